"""Host-side checks of libccs that need no GPU: the library builds for
sm_103a, exports every entry point that include/ccs.h declares, sizes its
workspaces and rejects bad arguments before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ccs():
    from paper_1508_01256_gb300 import build, ccs
    build.build()
    return ccs


def _declared():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"CCS_API\s+[\w\s\*]+?\b(ccs_\w+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(ccs):
    names = _declared()
    assert len(names) >= 13
    lib = ctypes.CDLL(ccs.LIB_PATH)
    for name in names:
        assert hasattr(lib, name), name


def test_version_and_status_strings(ccs):
    l = ccs.lib()
    assert l.ccs_version() >= 10000
    assert l.ccs_status_string(0) == b"CCS_OK"
    assert l.ccs_status_string(4) == b"CCS_ETIMEOUT"


def test_params_defaults(ccs):
    p = ccs.params()
    assert (p.alpha, p.max_iter, p.score_mode, p.engine, p.watchdog_ms) == (2, 100, 0, 0, 0)


def test_workspace_sizes(ccs):
    a = ccs.ccs_workspace_size(ccs.OP_DECODE, 4096, 410, 7)
    b = ccs.ccs_workspace_size(ccs.OP_DECODE, 2 ** 20, 2 ** 17, 7)
    assert 0 < a < b
    assert ccs.ccs_workspace_size(ccs.OP_MAKE_EXPANDER, 4096, 410, 7) > 410 * 4
    for bad in [(0, 10, 3), (10, 0, 3), (10, 5, 0), (10, 5, 6), (10, 40, 17), (2 ** 28, 10 ** 6, 9)]:
        assert ccs.ccs_workspace_size(ccs.OP_DECODE, *bad) == 0


def test_batch_workspace_covers_every_problem(ccs):
    """One shared header plus every problem's arrays: more than either
    problem alone needs, less than two separate workspaces."""
    probs = [ccs.Problem(4096, 410, 7, 0), ccs.Problem(1000, 100, 5, 0)]
    total = ccs.ccs_batch_workspace_size(probs)
    a = ccs.ccs_workspace_size(ccs.OP_DECODE, 4096, 410, 7)
    b = ccs.ccs_workspace_size(ccs.OP_DECODE, 1000, 100, 5)
    assert max(a, b) < total < a + b + (1 << 20)
    assert ccs.ccs_batch_workspace_size([ccs.Problem(10, 5, 6, 0)]) == 0


def test_bad_arguments_rejected_before_device_work(ccs):
    l = ccs.lib()
    # sizes
    rc = l.ccs_make_expander(10, 5, 17, 1, 1, 1, 1, 1, 1 << 20, None)
    assert rc == ccs.CCS_EINVAL and b"d=17" in l.ccs_last_error()
    rc = l.ccs_measure(10, 5, 6, 1, 1, 1, 1, None)
    assert rc == ccs.CCS_EINVAL
    # alpha outside [2, d], unknown score mode, negative max_iter
    for kw in (dict(alpha=1), dict(alpha=8), dict(score_mode=5), dict(max_iter=-1),
               dict(engine=9), dict(watchdog_ms=-3)):
        p = ccs.params(**kw)
        out = ccs.Result()
        rc = l.ccs_decode_parallel_l0(100, 20, 7, 1, 1, 1, 1, 1, 1, None, ctypes.byref(p),
                                      ctypes.byref(out), 1, 1 << 30, None)
        assert rc == ccs.CCS_EINVAL, kw
    # workspace too small
    p = ccs.params()
    out = ccs.Result()
    rc = l.ccs_decode_parallel_l0(100, 20, 7, 1, 1, 1, 1, 1, 1, None, ctypes.byref(p),
                                  ctypes.byref(out), 1, 16, None)
    assert rc == ccs.CCS_ENOMEM and b"workspace" in l.ccs_last_error()
    # null pointers
    rc = l.ccs_decode_parallel_l0(100, 20, 7, None, 1, 1, 1, 1, 1, None, ctypes.byref(p),
                                  ctypes.byref(out), 1, 1 << 30, None)
    assert rc == ccs.CCS_EINVAL
    # server configurations (checked before the device is touched): a pool
    # off a 256-byte boundary, no batch slot, a pool too small for the header
    h = ctypes.c_void_p()
    for pool, nbytes, maxb, want in ((0x100008, 1 << 30, 8, ccs.CCS_EINVAL),
                                     (0x100000, 1 << 30, 0, ccs.CCS_EINVAL),
                                     (0x100000, 4096, 512, ccs.CCS_EBUDGET)):
        cfg = ccs.ServerConfig(pool, nbytes, maxb, 2, ccs.params())
        assert l.ccs_server_create(ctypes.byref(cfg), None, ctypes.byref(h)) == want, pool
        assert not h.value


def test_misaligned_arrays_rejected_before_device_work(ccs):
    """Device pointers off their alignment (a bulk copy from csc_rows wants 16
    bytes, binary64 and int64 arrays 8, csr_cols 4, workspaces 256) are
    refused on the host with CCS_EINVAL, naming the array, before any device
    work: on the device they would fault."""
    l = ccs.lib()
    A = 0x10000000  # aligned fake device addresses, 1 MiB apart
    ptrs = dict(csc=A, ptr=A + (1 << 20), cols=A + (2 << 20), y=A + (3 << 20),
                x_hat=A + (4 << 20), r=A + (5 << 20), hist=A + (6 << 20))
    ws = A + (64 << 20)
    p = ccs.params()
    out = ccs.Result()

    def decode(**bad):
        q = dict(ptrs, **{k: v for k, v in bad.items() if k != "ws"})
        return l.ccs_decode_parallel_l0(100, 20, 7, q["csc"], q["ptr"], q["cols"], q["y"],
                                        q["x_hat"], q["r"], q["hist"], ctypes.byref(p),
                                        ctypes.byref(out), bad.get("ws", ws), 1 << 30, None)

    for bad, name in ((dict(csc=A + 8), b"csc_rows"), (dict(ptr=A + (1 << 20) + 4), b"csr_ptr"),
                      (dict(cols=A + (2 << 20) + 2), b"csr_cols"), (dict(y=A + (3 << 20) + 4), b"y"),
                      (dict(x_hat=A + (4 << 20) + 1), b"x_hat"), (dict(r=A + (5 << 20) + 4), b"r"),
                      (dict(hist=A + (6 << 20) + 4), b"r0_hist"), (dict(ws=ws + 128), b"ws")):
        assert decode(**bad) == ccs.CCS_EINVAL, bad
        assert name + b" is not on a" in l.ccs_last_error(), bad
    # a batch names the problem
    good = ccs.Problem(100, 20, 7, 0, ptrs["csc"], ptrs["ptr"], ptrs["cols"], ptrs["y"],
                       ptrs["x_hat"], ptrs["r"], None)
    bad = ccs.Problem(100, 20, 7, 0, ptrs["csc"], ptrs["ptr"], ptrs["cols"], ptrs["y"],
                      ptrs["x_hat"] + 4, ptrs["r"], None)
    arr = (ccs.Problem * 2)(good, bad)
    res = (ccs.Result * 2)()
    rc = l.ccs_decode_batch(arr, 2, ctypes.byref(p), res, ws, 1 << 30, None)
    assert rc == ccs.CCS_EINVAL and b"problem 1: x_hat" in l.ccs_last_error()
    rc = l.ccs_decode_batch(arr, 1, ctypes.byref(p), res, ws + 64, 1 << 30, None)
    assert rc == ccs.CCS_EINVAL and b"ws" in l.ccs_last_error()
    # set-up calls
    rc = l.ccs_measure(100, 20, 7, ptrs["ptr"], ptrs["cols"], ptrs["x_hat"] + 4, ptrs["y"], None)
    assert rc == ccs.CCS_EINVAL and b"ccs_measure: x is not" in l.ccs_last_error()
    rc = l.ccs_make_expander(100, 20, 7, 1, ptrs["csc"], ptrs["ptr"], ptrs["cols"], ws + 16,
                             1 << 30, None)
    assert rc == ccs.CCS_EINVAL and b"ws" in l.ccs_last_error()
    rc = l.ccs_unscale(100, ptrs["y"], ptrs["r"] + 2, ptrs["x_hat"], None)
    assert rc == ccs.CCS_EINVAL and b"ccs_unscale: z" in l.ccs_last_error()


def test_binding_refuses_host_tensors():
    """The binding hands tensors' addresses to the device as pointers, so a
    host tensor is refused before any library call (on the device its
    address would be an illegal access)."""
    import torch
    from paper_1508_01256_gb300 import ccs
    n, m, d = 40, 12, 3
    csc = torch.zeros((n, d), dtype=torch.int32)
    ptr = torch.zeros(m + 1, dtype=torch.int64)
    cols = torch.zeros(n * d, dtype=torch.int32)
    y = torch.zeros(m, dtype=torch.float64)
    x_hat = torch.zeros(n, dtype=torch.float64)
    r = torch.zeros(m, dtype=torch.float64)
    with pytest.raises(TypeError, match="csc_rows must be a CUDA tensor"):
        ccs.problem(csc, ptr, cols, y, x_hat, r)
    with pytest.raises(TypeError, match="CUDA tensor"):
        ccs.decode_parallel_l0(csc, ptr, cols, y)
    with pytest.raises(TypeError, match="CUDA tensor"):
        ccs.decode_parallel_l0(csc, ptr, cols, y, out=(x_hat, r, None))
    with pytest.raises(TypeError, match="csc_rows must be a CUDA tensor of shape"):
        ccs.problem(cols, ptr, cols, y, x_hat, r)  # not [n, d]


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1508_01256_gb300 import ccs
    monkeypatch.setattr(ccs, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(ccs, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        ccs.lib()
