"""The decode entry point that allocates nothing.

Callers that cannot allocate device memory while they decode (a reserved
memory budget, a real-time loop, buffers handed out by a host) use
ccs_decode_parallel_l0_noalloc: no caller workspace, the scratch is one
library-held static device array shared by every call.  Its results must be
the same as the ordinary entry point's, bit for bit, on consecutive calls
(the shared scratch keeps the previous call's contents and must not leak
into the next).  This file is collected last so that a run stopping at the
first failure has already run every other test; it also passes on its own in
a fresh process.
"""
import numpy as np
import pytest

from paper_1508_01256_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ccs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_01256_gb300 import build, ccs
    build.build()
    return ccs


def _device(ccs, p):
    import torch
    csc, ptr, cols = ccs.make_expander(p.n, p.m, p.d, p.a_seed)
    y = ccs.measure(ptr, cols, torch.from_numpy(p.x).cuda(), p.m, p.d)
    return csc, ptr, cols, y


def _noalloc(ccs, p, csc, ptr, cols, y):
    import torch
    x_hat = torch.full((p.n,), float("nan"), dtype=torch.float64, device="cuda")
    r = torch.full((p.m,), float("nan"), dtype=torch.float64, device="cuda")
    hist = torch.full((101,), -1, dtype=torch.int64, device="cuda")
    res = ccs.ccs_decode_parallel_l0_noalloc(p.n, p.m, p.d, csc, ptr, cols, y, x_hat, r, hist,
                                             ccs.params())
    return res, x_hat, r, hist


def test_noalloc_matches_workspace_entry_point_on_consecutive_calls(ccs):
    # two different problems, then the first again: each call must equal the
    # ordinary entry point's result although the scratch still holds the
    # previous call's state
    probs = [inputs.plain_at_scale(seed=3), inputs.plain_small(seed=4),
             inputs.plain_at_scale(seed=3)]
    for p in probs:
        csc, ptr, cols, y = _device(ccs, p)
        ref = ccs.decode_parallel_l0(csc, ptr, cols, y)
        for _ in range(2):
            res, x_hat, r, hist = _noalloc(ccs, p, csc, ptr, cols, y)
            assert (res.status, res.iterations, res.r0_final, res.error) == \
                (ref.status, ref.iterations, ref.r0_final, ref.error)
            assert np.array_equal(x_hat.cpu().numpy(), ref.x_hat.cpu().numpy())
            assert np.array_equal(r.cpu().numpy(), ref.r.cpu().numpy())
            assert hist[:res.iterations + 1].cpu().tolist() == ref.r0_hist


def test_noalloc_takes_no_device_memory(ccs):
    """After a first call (which looks up the scratch's device address), more
    calls leave the device's free memory exactly where it was: neither the
    library nor the driver hands out memory for them."""
    import torch
    p = inputs.plain_at_scale(seed=5)
    csc, ptr, cols, y = _device(ccs, p)
    x_hat = torch.empty(p.n, dtype=torch.float64, device="cuda")
    r = torch.empty(p.m, dtype=torch.float64, device="cuda")
    hist = torch.empty(101, dtype=torch.int64, device="cuda")
    ccs.ccs_decode_parallel_l0_noalloc(p.n, p.m, p.d, csc, ptr, cols, y, x_hat, r, hist,
                                       ccs.params())
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        ccs.ccs_decode_parallel_l0_noalloc(p.n, p.m, p.d, csc, ptr, cols, y, x_hat, r, hist,
                                           ccs.params())
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before


def test_noalloc_checks_tensor_arguments(ccs):
    """Tensors handed to the binding are checked before a pointer reaches the
    library: a short history or a wrong-sized output is refused on the host."""
    import torch
    p = inputs.plain_small(seed=6)
    csc, ptr, cols, y = _device(ccs, p)
    x_hat = torch.empty(p.n, dtype=torch.float64, device="cuda")
    r = torch.empty(p.m, dtype=torch.float64, device="cuda")
    short_hist = torch.empty(10, dtype=torch.int64, device="cuda")
    with pytest.raises(ValueError):
        ccs.ccs_decode_parallel_l0_noalloc(p.n, p.m, p.d, csc, ptr, cols, y, x_hat, r,
                                           short_hist, ccs.params(max_iter=100))
    with pytest.raises(ValueError):
        ccs.ccs_decode_parallel_l0_noalloc(p.n, p.m, p.d, csc, ptr, cols, y, x_hat[:-1], r,
                                           None, ccs.params())


def test_noalloc_rejects_sizes_beyond_its_scratch(ccs):
    n, m, d = 2 ** 22, 2 ** 19, 7
    assert ccs.ccs_workspace_size(ccs.OP_DECODE, n, m, d) > ccs.ccs_noalloc_scratch_bytes()
    with pytest.raises(ccs.CcsError) as ei:
        ccs.ccs_decode_parallel_l0_noalloc(n, m, d, 16, 16, 16, 16, 16, 16, None, ccs.params())
    assert ei.value.code == ccs.CCS_EINVAL and "scratch" in str(ei.value)
