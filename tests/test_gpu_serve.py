"""Serving: continuous batching of decode requests (ccs_server_*).

Each served result must be bit-identical to the same request decoded alone,
whatever else shares its rounds; admission must respect the memory pool; a
request that can never fit is refused."""
import ctypes
import random
import time

import numpy as np
import pytest

from paper_1508_01256_gb300 import inputs
from gpu_util import device_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ccs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_01256_gb300 import build, ccs
    build.build()
    return ccs


def _requests(ccs, probs):
    import torch
    reqs = []
    for p in probs:
        csc, ptr, cols, y = device_problem(ccs, p)
        x_hat = torch.full((p.n,), float("nan"), dtype=torch.float64, device="cuda")
        r = torch.full((p.m,), float("nan"), dtype=torch.float64, device="cuda")
        hist = torch.full((101,), -1, dtype=torch.int64, device="cuda")
        reqs.append((csc, ptr, cols, y, x_hat, r, hist))
    return reqs


def _check_same_as_alone(ccs, reqs, infos):
    for (csc, ptr, cols, y, x_hat, r, hist), info in zip(reqs, infos):
        alone = ccs.decode_parallel_l0(csc, ptr, cols, y)
        res = info.result
        assert res.error == 0
        assert (res.status, res.iterations, res.r0_final) == \
            (alone.status, alone.iterations, alone.r0_final)
        assert np.array_equal(x_hat.cpu().numpy(), alone.x_hat.cpu().numpy())
        assert np.array_equal(r.cpu().numpy(), alone.r.cpu().numpy())
        assert hist[:res.iterations + 1].cpu().tolist() == alone.r0_hist


@pytest.mark.parametrize("iters_per_round", [1, 3])
def test_served_results_equal_alone(ccs, iters_per_round):
    """Mixed sizes arriving at random times join running rounds; every result
    equals the request decoded alone."""
    probs = inputs.batch_problems(24, seed=17 + iters_per_round, log2n_hi=17.0, ds=(7, 9))
    reqs = _requests(ccs, probs)
    rng = random.Random(5)
    arrivals = np.cumsum([rng.uniform(0, 0.002) for _ in reqs])
    with ccs.Server(512 << 20, max_batch=8, iters_per_round=iters_per_round) as srv:
        infos = ccs.serve_poisson(srv, reqs, arrivals)
        st = srv.stats()
    assert st["completed"] == len(reqs) and st["error"] == 0
    assert st["peak_inflight"] <= 8
    assert all(i.done_s >= i.admit_s >= i.submit_s for i in infos)
    _check_same_as_alone(ccs, reqs, infos)


def test_admission_by_memory_budget(ccs):
    """A pool that holds about two requests' state at a time: the rest wait,
    every request still completes with the alone result, and the state in use
    never exceeds the pool."""
    probs = [inputs.make_problem(200000, 20000, 7, 2000, 300 + i) for i in range(6)]
    reqs = _requests(ccs, probs)
    one = ccs.ccs_workspace_size(ccs.OP_DECODE, 200000, 20000, 7)
    pool = int(2.5 * one) + (64 << 10)  # room for two states and the launch header
    with ccs.Server(pool, max_batch=16, iters_per_round=2) as srv:
        infos = ccs.serve_poisson(srv, reqs, [0.0] * len(reqs))
        st = srv.stats()
    assert st["completed"] == 6 and st["peak_inflight"] <= 2
    assert st["peak_bytes"] <= pool
    assert max(i.admit_s for i in infos) > min(i.done_s for i in infos)  # someone waited
    _check_same_as_alone(ccs, reqs, infos)


def test_refuses_request_that_cannot_fit(ccs):
    import torch
    p = inputs.make_problem(300000, 50000, 7, 100, 9)
    csc, ptr, cols, y = device_problem(ccs, p)
    x_hat = torch.empty(p.n, dtype=torch.float64, device="cuda")
    r = torch.empty(p.m, dtype=torch.float64, device="cuda")
    with ccs.Server(2 << 20, max_batch=4) as srv:  # the request needs ~3.7 MB of state
        with pytest.raises(ccs.CcsError) as ei:
            srv.submit(csc, ptr, cols, y, x_hat, r)
        assert ei.value.code == ccs.CCS_EBUDGET
        # a request without an output array is stopped by the binding before
        # any pointer leaves it ...
        with pytest.raises(TypeError):
            srv.submit(csc, ptr, cols, y, x_hat, None)
        # ... and, through the C ABI directly, refused by the library with
        # CCS_EINVAL, without disturbing the server
        small = inputs.make_problem(4096, 410, 7, 41, 10)
        s_csc, s_ptr, s_cols, s_y = device_problem(ccs, small)
        s_x = torch.empty(small.n, dtype=torch.float64, device="cuda")
        s_r = torch.empty(small.m, dtype=torch.float64, device="cuda")
        desc = ccs.problem(s_csc, s_ptr, s_cols, s_y, s_x, s_r)
        desc.r = None  # null output pointer
        ticket = ctypes.c_int64(-1)
        rc = ccs.lib().ccs_server_submit(srv._h, ctypes.byref(desc), ctypes.byref(ticket))
        assert rc == ccs.CCS_EINVAL and ticket.value == -1
        assert srv.stats()["error"] == 0
        # the server still decodes a good request afterwards
        info = srv.wait(srv.submit(s_csc, s_ptr, s_cols, s_y, s_x, s_r))
        alone = ccs.decode_parallel_l0(s_csc, s_ptr, s_cols, s_y)
        assert info.result.error == 0 and info.result.status == alone.status
        assert torch.equal(s_x, alone.x_hat) and torch.equal(s_r, alone.r)


def test_poll_reports_busy_then_done(ccs):
    probs = [inputs.plain_small(seed=s) for s in range(3)]
    reqs = _requests(ccs, probs)
    with ccs.Server(256 << 20, max_batch=4, iters_per_round=1) as srv:
        tickets = [srv.submit(*q) for q in reqs]
        infos = []
        deadline = time.time() + 30
        for t in tickets:
            while True:
                info = srv.poll(t)
                if info is not None:
                    infos.append(info)
                    break
                assert time.time() < deadline
                time.sleep(0.001)
        with pytest.raises(ccs.CcsError):
            srv.poll(999999)
    _check_same_as_alone(ccs, reqs, infos)


def test_serve_stream_ring_results_equal_alone(ccs):
    """Open-loop stream over a ring of output slots (the serving load sweep's
    driver): 48 requests cycle through 6 distinct problems and 12 output
    slots; each slot's final contents equal its problem decoded alone, and
    every result's (status, iterations, final ||r||_0) does too."""
    import torch
    probs = inputs.batch_problems(6, seed=99, log2n_hi=16.0, ds=(7, 9))
    reqs = _requests(ccs, probs)
    D, R, count = len(reqs), 12, 48
    outs = [(torch.full_like(reqs[s % D][4], float("nan")),
             torch.full_like(reqs[s % D][5], float("nan"))) for s in range(R)]

    def request_of(q):
        return tuple(reqs[q % D][:4]) + outs[q % R]

    arrivals = np.cumsum(np.random.default_rng(3).exponential(0.0002, size=count))
    with ccs.Server(512 << 20, max_batch=8, iters_per_round=2) as srv:
        infos, waited = ccs.serve_stream(srv, request_of, count, arrivals, R)
    alone = [ccs.decode_parallel_l0(*reqs[p][:4]) for p in range(D)]
    for q, info in enumerate(infos):
        a = alone[q % D]
        assert info.result.error == 0
        assert (info.result.status, info.result.iterations, info.result.r0_final) == \
            (a.status, a.iterations, a.r0_final)
    for s in range(R):
        a = alone[s % D]
        assert torch.equal(outs[s][0], a.x_hat) and torch.equal(outs[s][1], a.r)


def _seeded_inputs(orc, shapes, seed):
    """Host y of each (n, m, d, k) problem from the oracle's own expander and
    measurement (the server draws the same A from the seed on the device)."""
    out = []
    for q, (n, m, d, k) in enumerate(shapes):
        p = inputs.make_problem(n, m, d, k, seed + q)
        A = orc.make_expander(n, m, d, p.a_seed)
        out.append((p, A, orc.measure(A, m, p.x)))
    return out


def test_seeded_requests_equal_the_oracle(ccs, orc):
    """Seeded requests (A drawn by the server into its pool, y from the host,
    results copied back to the host) served in one mix with device requests:
    every seeded result, x_hat, r and the ||r||_0 history, is bit-identical
    to the oracle's decode of the same A and y; the device requests still
    equal their decodes alone."""
    shapes = [(4096, 410, 7, 41), (20000, 2000, 9, 400), (3000, 300, 7, 90),
              (12000, 120, 7, 12), (8000, 2400, 9, 480), (5000, 500, 7, 150)]
    seeded = _seeded_inputs(orc, shapes, 4100)
    dev_probs = inputs.batch_problems(6, seed=23, log2n_hi=15.0, ds=(7, 9))
    dev_reqs = _requests(ccs, dev_probs)
    outs = [(np.full(p.n, np.nan), np.full(p.m, np.nan), np.full(101, -1, dtype=np.int64))
            for p, _, _ in seeded]
    with ccs.Server(512 << 20, max_batch=8, iters_per_round=2) as srv:
        tickets = []
        for (p, _, y), (xo, ro, ho), dq in zip(seeded, outs, dev_reqs):
            tickets.append(srv.submit_seeded(p.n, p.m, p.d, p.a_seed, y, xo, ro, ho))
            tickets.append(srv.submit(*dq))
        infos = [srv.wait(t) for t in tickets]
        st = srv.stats()
    assert st["completed"] == 12 and st["error"] == 0
    for q, ((p, A, y), (xo, ro, ho)) in enumerate(zip(seeded, outs)):
        res = infos[2 * q].result
        ref = orc.parallel_l0(A, p.m, y)
        assert res.error == 0
        assert (res.status, res.iterations, res.r0_final) == \
            (ref["status"], ref["iterations"], ref["r0_final"])
        assert np.array_equal(xo.view(np.int64), ref["x_hat"].view(np.int64))
        assert np.array_equal(ro.view(np.int64), ref["r"].view(np.int64))
        assert ho[:res.iterations + 1].tolist() == list(ref["r0_hist"])
    _check_same_as_alone(ccs, dev_reqs, infos[1::2])


def test_seeded_admission_bounds_the_pool(ccs, orc):
    """A pool that holds two seeded requests (A, y, outputs and state
    included): the others wait; the pool's peak use stays within it; every
    result equals the oracle's."""
    shapes = [(60000, 6000, 7, 600)] * 5
    seeded = _seeded_inputs(orc, shapes, 5200)
    one = ccs.ccs_seeded_request_bytes(60000, 6000, 7, 100)
    assert one > 2 * 60000 * 7 * 4  # CSC and CSR are part of it
    pool = 2 * one + (1 << 20)
    outs = [np.full(p.n, np.nan) for p, _, _ in seeded]
    with ccs.Server(pool, max_batch=8, iters_per_round=1) as srv:
        tickets = [srv.submit_seeded(p.n, p.m, p.d, p.a_seed, y, xo)
                   for (p, _, y), xo in zip(seeded, outs)]
        infos = [srv.wait(t) for t in tickets]
        st = srv.stats()
        with pytest.raises(ccs.CcsError) as ei:  # can never fit
            srv.submit_seeded(600000, 60000, 7, 1, np.zeros(60000), np.zeros(600000))
        assert ei.value.code == ccs.CCS_EBUDGET
    assert st["peak_inflight"] <= 2 and st["peak_bytes"] <= pool - (1 << 20) + 256
    assert max(i.admit_s for i in infos) > min(i.done_s for i in infos)
    for (p, A, y), xo, info in zip(seeded, outs, infos):
        ref = orc.parallel_l0(A, p.m, y)
        assert info.result.status == ref["status"]
        assert np.array_equal(xo, ref["x_hat"])


def test_seeded_nonzero_outputs_equal_the_oracle(ccs, orc):
    """Seeded requests that ask for x_hat as its nonzeros: the count equals
    the oracle's, the indices come back ascending with their values bit for
    bit; with a list too short for every nonzero the count is still exact
    and the entries returned are nonzeros of the oracle's x_hat."""
    shapes = [(4096, 410, 7, 41), (20000, 2000, 9, 400), (30000, 300, 7, 90),
              (12000, 1200, 7, 360)]
    seeded = _seeded_inputs(orc, shapes, 6100)
    caps = [1000, 1000, 1000, 7]
    outs = [(np.zeros(c, dtype=np.int64), np.zeros(c), np.full(1, -1, dtype=np.int64))
            for c in caps]
    with ccs.Server(512 << 20, max_batch=8, iters_per_round=2) as srv:
        tickets = [srv.submit_seeded(p.n, p.m, p.d, p.a_seed, y, None, nonzeros=nz)
                   for (p, _, y), nz in zip(seeded, outs)]
        infos = [srv.wait(t) for t in tickets]
        with pytest.raises(ValueError):
            srv.submit_seeded(4096, 410, 7, 1, np.zeros(410))  # neither output form
    for (p, A, y), (idx, val, nnz), cap, info in zip(seeded, outs, caps, infos):
        ref = orc.parallel_l0(A, p.m, y)
        assert info.result.error == 0 and info.result.status == ref["status"]
        want = np.nonzero(ref["x_hat"])[0]
        assert nnz[0] == want.size
        got = idx[:min(cap, want.size)]
        assert np.all(np.diff(got) > 0)
        assert np.array_equal(val[:got.size].view(np.int64), ref["x_hat"][got].view(np.int64))
        if want.size <= cap:
            assert np.array_equal(got, want)
        else:
            assert np.isin(got, want).all()
