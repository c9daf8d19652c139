"""Thin ctypes binding of libccs (include/ccs.h).

Argument marshalling only: every step of the decode runs in the CUDA
library.  PyTorch supplies device memory (tensors) and the stream.  If the
library is missing, importing works but every call raises: there is no CPU
fallback.

The ``ccs_*`` functions mirror the C ABI one to one (tensors stand in for
device pointers).  ``make_expander``, ``measure``, ``decode_parallel_l0`` and
``decode_batch`` are conveniences that allocate outputs and workspaces with
torch and call the ``ccs_*`` functions.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libccs.so")

CCS_OK, CCS_EINVAL, CCS_ENOMEM, CCS_ECUDA, CCS_ETIMEOUT, CCS_EBUDGET, CCS_EBUSY = range(7)
CONVERGED, STALLED, MAX_ITER = 0, 1, 2
STATUS_NAMES = {CONVERGED: "converged", STALLED: "stalled", MAX_ITER: "max_iter"}
SCORE_L0_DECREASE, SCORE_COUNT = 0, 1
ENGINE_AUTO, ENGINE_HOST_LOOP, ENGINE_PERSISTENT = 0, 1, 3
RESIDUAL_EXACT, RESIDUAL_ORDERED = 0, 1
OP_MAKE_EXPANDER, OP_DECODE = 0, 1


class CcsError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str):
        super().__init__(f"{where}: {_STATUS.get(code, code)}: {detail}")
        self.code = code


_STATUS = {0: "CCS_OK", 1: "CCS_EINVAL", 2: "CCS_ENOMEM", 3: "CCS_ECUDA",
           4: "CCS_ETIMEOUT", 5: "CCS_EBUDGET", 6: "CCS_EBUSY"}


class Params(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_int32), ("max_iter", ctypes.c_int32),
                ("score_mode", ctypes.c_int32), ("engine", ctypes.c_int32),
                ("watchdog_ms", ctypes.c_int32), ("debug_flags", ctypes.c_int32),
                ("schedule", ctypes.c_int32), ("shifted", ctypes.c_int32)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("r0_final", ctypes.c_int64), ("error", ctypes.c_int32),
                ("row_driven", ctypes.c_int32), ("row_entries", ctypes.c_int64),
                ("residual_form", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("m", ctypes.c_int32), ("d", ctypes.c_int32),
                ("reserved", ctypes.c_int32),
                ("csc_rows", ctypes.c_void_p), ("csr_ptr", ctypes.c_void_p),
                ("csr_cols", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("x_hat", ctypes.c_void_p), ("r", ctypes.c_void_p),
                ("r0_hist", ctypes.c_void_p)]


class SeededRequest(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("m", ctypes.c_int32), ("d", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("a_seed", ctypes.c_uint64),
                ("y", ctypes.c_void_p), ("x_hat", ctypes.c_void_p), ("r", ctypes.c_void_p),
                ("r0_hist", ctypes.c_void_p), ("x_idx", ctypes.c_void_p),
                ("x_val", ctypes.c_void_p), ("x_cap", ctypes.c_int64),
                ("x_nnz", ctypes.c_void_p)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("pool", ctypes.c_void_p), ("pool_bytes", ctypes.c_size_t),
                ("max_batch", ctypes.c_int32), ("iters_per_round", ctypes.c_int32),
                ("params", Params)]


class TicketInfo(ctypes.Structure):
    _fields_ = [("result", Result), ("submit_s", ctypes.c_double),
                ("admit_s", ctypes.c_double), ("done_s", ctypes.c_double),
                ("rounds", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in ("submitted", "admitted", "completed", "rounds",
                                              "peak_inflight", "peak_bytes", "bytes_in_use",
                                              "pending", "inflight")] + \
               [("error", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None

K_INIT, K_SCORE, K_RESIDUAL, K_FINISH, K_PERSISTENT, K_COUNT = 0, 1, 2, 3, 4, 8
KERNEL_NAMES = {K_INIT: "init", K_SCORE: "score", K_RESIDUAL: "residual",
                K_FINISH: "finish", K_PERSISTENT: "persistent", 5: "score.fingerprints",
                6: "score.stream", 7: "score.queue"}


class KernelTime(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


def lib() -> ctypes.CDLL:
    """Load libccs.so (built in-tree by ``paper_1508_01256_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_1508_01256_gb300.build`")
        l = ctypes.CDLL(LIB_PATH)
        P, i32, i64, u64, sz = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                ctypes.c_uint64, ctypes.c_size_t)
        l.ccs_params_init.argtypes = [ctypes.POINTER(Params)]
        l.ccs_params_init.restype = None
        l.ccs_status_string.argtypes = [ctypes.c_int]
        l.ccs_status_string.restype = ctypes.c_char_p
        l.ccs_last_error.argtypes = []
        l.ccs_last_error.restype = ctypes.c_char_p
        l.ccs_version.restype = ctypes.c_int
        l.ccs_workspace_size.argtypes = [i32, i32, i32, i32]
        l.ccs_workspace_size.restype = sz
        l.ccs_batch_workspace_size.argtypes = [ctypes.POINTER(Problem), i32]
        l.ccs_batch_workspace_size.restype = sz
        l.ccs_make_expander.argtypes = [i32, i32, i32, u64, P, P, P, P, sz, P]
        l.ccs_measure.argtypes = [i32, i32, i32, P, P, P, P, P]
        l.ccs_column_scales.argtypes = [i32, u64, P, P]
        l.ccs_measure_scaled.argtypes = [i32, i32, i32, P, P, P, P, P, P]
        l.ccs_unscale.argtypes = [i32, P, P, P, P]
        l.ccs_decode_parallel_l0.argtypes = [i32, i32, i32, P, P, P, P, P, P, P,
                                             ctypes.POINTER(Params), ctypes.POINTER(Result),
                                             P, sz, P]
        l.ccs_decode_batch.argtypes = [ctypes.POINTER(Problem), i32, ctypes.POINTER(Params),
                                       ctypes.POINTER(Result), P, sz, P]
        l.ccs_decode_parallel_l0_async.argtypes = [i32, i32, i32, P, P, P, P, P, P, P,
                                                   ctypes.POINTER(Params), P, P, sz, P]
        l.ccs_decode_batch_async.argtypes = [ctypes.POINTER(Problem), i32, ctypes.POINTER(Params),
                                             P, P, sz, P]
        l.ccs_autotune.argtypes = [ctypes.POINTER(Problem), i32, ctypes.POINTER(Params), P, sz, P,
                                   ctypes.POINTER(i32)]
        l.ccs_autotune.restype = ctypes.c_int
        l.ccs_autotune_reset.argtypes = []
        l.ccs_autotune_reset.restype = None
        l.ccs_autotune_get.argtypes = [i32, i32, ctypes.POINTER(i32)]
        l.ccs_autotune_get.restype = ctypes.c_int
        l.ccs_autotune_save.argtypes = [ctypes.c_char_p]
        l.ccs_autotune_save.restype = ctypes.c_int
        l.ccs_autotune_load.argtypes = [ctypes.c_char_p]
        l.ccs_autotune_load.restype = ctypes.c_int
        l.ccs_decode_parallel_l0_noalloc.argtypes = [i32, i32, i32, P, P, P, P, P, P, P,
                                                     ctypes.POINTER(Params),
                                                     ctypes.POINTER(Result), P]
        l.ccs_decode_parallel_l0_noalloc.restype = ctypes.c_int
        l.ccs_noalloc_scratch_bytes.argtypes = []
        l.ccs_noalloc_scratch_bytes.restype = sz
        l.ccs_server_create.argtypes = [ctypes.POINTER(ServerConfig), P, ctypes.POINTER(P)]
        l.ccs_server_submit.argtypes = [P, ctypes.POINTER(Problem), ctypes.POINTER(i64)]
        l.ccs_server_submit_seeded.argtypes = [P, ctypes.POINTER(SeededRequest),
                                               ctypes.POINTER(i64)]
        l.ccs_seeded_request_bytes.argtypes = [i32, i32, i32, i32, i64]
        l.ccs_seeded_request_bytes.restype = sz
        l.ccs_server_poll.argtypes = [P, i64, ctypes.POINTER(TicketInfo)]
        l.ccs_server_wait.argtypes = [P, i64, ctypes.POINTER(TicketInfo), i32]
        l.ccs_server_stats_get.argtypes = [P, ctypes.POINTER(ServerStats)]
        l.ccs_server_destroy.argtypes = [P]
        for name in ("ccs_server_create", "ccs_server_submit", "ccs_server_submit_seeded",
                     "ccs_server_poll",
                     "ccs_server_wait", "ccs_server_stats_get", "ccs_server_destroy"):
            getattr(l, name).restype = ctypes.c_int
        l.ccs_batch_graph_create.argtypes = [ctypes.POINTER(Problem), i32, ctypes.POINTER(Params),
                                             P, P, sz, ctypes.POINTER(P)]
        l.ccs_graph_launch.argtypes = [P, P]
        l.ccs_graph_destroy.argtypes = [P]
        for name in ("ccs_batch_graph_create", "ccs_graph_launch", "ccs_graph_destroy"):
            getattr(l, name).restype = ctypes.c_int
        l.ccs_profile_begin.argtypes = []
        l.ccs_profile_end.argtypes = [ctypes.POINTER(KernelTime)]
        l.ccs_profile_phases.argtypes = [i32, ctypes.POINTER(ctypes.c_double)]
        l.ccs_profile_phases.restype = ctypes.c_int
        l.ccs_launch_count.argtypes = []
        l.ccs_launch_count.restype = ctypes.c_int64
        for name in ("ccs_make_expander", "ccs_measure", "ccs_decode_parallel_l0",
                     "ccs_decode_batch", "ccs_profile_begin", "ccs_profile_end",
                     "ccs_decode_parallel_l0_async", "ccs_decode_batch_async"):
            getattr(l, name).restype = ctypes.c_int
        _lib = l
        return l


def _check(rc: int, where: str):
    if rc != CCS_OK:
        raise CcsError(rc, where, lib().ccs_last_error().decode(errors="replace"))


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream):
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _need(t, dtype, numel, name, at_least=False):
    """t must be a contiguous CUDA tensor of `dtype` with `numel` elements
    (or at least that many): the library takes its address as a device
    pointer, so anything else would be read or written out of bounds."""
    import torch
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
        raise TypeError(f"{name} must be a CUDA tensor")
    short = t.numel() < numel if at_least else t.numel() != numel
    if t.dtype != dtype or not t.is_contiguous() or short:
        raise ValueError(f"{name}: need contiguous {dtype} with {'at least ' if at_least else ''}"
                         f"{numel} elements, got {t.dtype} {tuple(t.shape)}")


def _need_problem(csc_rows, csr_ptr, csr_cols, y, x_hat, r, r0_hist, max_iter, outputs=True):
    """The arrays of one problem (shapes from csc_rows [n, d] and y [m]);
    outputs=False skips x_hat, r and r0_hist (allocated by this module)."""
    import torch
    if not isinstance(csc_rows, torch.Tensor) or csc_rows.dim() != 2:
        raise TypeError("csc_rows must be a CUDA tensor of shape [n, d]")
    n, d = csc_rows.shape
    if not isinstance(y, torch.Tensor):
        raise TypeError("y must be a CUDA tensor")
    m = y.numel()
    _need(csc_rows, torch.int32, n * d, "csc_rows")
    _need(csr_ptr, torch.int64, m + 1, "csr_ptr")
    _need(csr_cols, torch.int32, n * d, "csr_cols")
    _need(y, torch.float64, m, "y")
    if not outputs:
        return n, m, d
    _need(x_hat, torch.float64, n, "x_hat")
    _need(r, torch.float64, m, "r")
    if r0_hist is not None:
        _need(r0_hist, torch.int64, max_iter + 1 if max_iter is not None else 1, "r0_hist",
              at_least=True)
    return n, m, d


def _need_abi_arrays(where, n, m, d, csc_rows, csr_ptr, csr_cols, y, x_hat, r, r0_hist,
                     p: Params | None):
    """The one-to-one decode calls take tensors or raw device addresses (ints,
    passed through as the C ABI would take them).  Tensors are checked like
    the conveniences' arrays, and against the sizes n, m, d given, so that a
    short output never reaches the kernel."""
    import torch
    arrays = (csc_rows, csr_ptr, csr_cols, y, x_hat, r)
    if not any(isinstance(a, torch.Tensor) for a in arrays + (r0_hist,)):
        return
    max_iter = p.max_iter if p is not None else 100
    if isinstance(csc_rows, torch.Tensor) and csc_rows.dim() == 1:
        csc_rows = csc_rows.view(-1, d) if csc_rows.numel() % max(d, 1) == 0 else csc_rows
    got = _need_problem(csc_rows, csr_ptr, csr_cols, y, x_hat, r, r0_hist, max_iter)
    if got != (n, m, d):
        raise ValueError(f"{where}: arrays are for n, m, d = {got}, not {(n, m, d)}")


def params(alpha=2, max_iter=100, score_mode=SCORE_L0_DECREASE, engine=ENGINE_AUTO,
           watchdog_ms=0, debug_flags=0, schedule=0, shifted=False) -> Params:
    p = Params()
    lib().ccs_params_init(ctypes.byref(p))
    p.alpha, p.max_iter, p.score_mode, p.engine, p.watchdog_ms, p.debug_flags = (
        alpha, max_iter, score_mode, engine, watchdog_ms, debug_flags)
    p.schedule = schedule
    p.shifted = int(shifted)
    return p


# ---- one-to-one ABI calls ---------------------------------------------------

def ccs_workspace_size(op: int, n: int, m: int, d: int) -> int:
    return int(lib().ccs_workspace_size(op, n, m, d))


def ccs_batch_workspace_size(probs) -> int:
    arr = (Problem * len(probs))(*probs)
    return int(lib().ccs_batch_workspace_size(arr, len(probs)))


def ccs_make_expander(n, m, d, seed, csc_rows, csr_ptr, csr_cols, ws, stream=None):
    _check(lib().ccs_make_expander(n, m, d, seed & (2**64 - 1), _ptr(csc_rows),
                                   _ptr(csr_ptr), _ptr(csr_cols), _ptr(ws),
                                   ws.numel() * ws.element_size(), _stream(stream)),
           "ccs_make_expander")


def ccs_measure(n, m, d, csr_ptr, csr_cols, x, y, stream=None):
    _check(lib().ccs_measure(n, m, d, _ptr(csr_ptr), _ptr(csr_cols), _ptr(x), _ptr(y),
                             _stream(stream)), "ccs_measure")


def ccs_decode_parallel_l0(n, m, d, csc_rows, csr_ptr, csr_cols, y, x_hat, r, r0_hist,
                           p: Params | None, ws, stream=None) -> Result:
    _need_abi_arrays("ccs_decode_parallel_l0", n, m, d, csc_rows, csr_ptr, csr_cols, y, x_hat,
                     r, r0_hist, p)
    out = Result()
    rc = lib().ccs_decode_parallel_l0(
        n, m, d, _ptr(csc_rows), _ptr(csr_ptr), _ptr(csr_cols), _ptr(y), _ptr(x_hat), _ptr(r),
        _ptr(r0_hist), ctypes.byref(p) if p is not None else None, ctypes.byref(out),
        _ptr(ws), ws.numel() * ws.element_size(), _stream(stream))
    _check(rc, "ccs_decode_parallel_l0")
    return out


def ccs_decode_parallel_l0_async(n, m, d, csc_rows, csr_ptr, csr_cols, y, x_hat, r, r0_hist,
                                 p: Params | None, out_dev, ws, stream=None):
    """Enqueue a decode; its ccs_result lands in the device buffer out_dev
    (a tensor of >= RESULT_BYTES bytes, or a device address)."""
    _need_abi_arrays("ccs_decode_parallel_l0_async", n, m, d, csc_rows, csr_ptr, csr_cols, y,
                     x_hat, r, r0_hist, p)
    rc = lib().ccs_decode_parallel_l0_async(
        n, m, d, _ptr(csc_rows), _ptr(csr_ptr), _ptr(csr_cols), _ptr(y), _ptr(x_hat), _ptr(r),
        _ptr(r0_hist), ctypes.byref(p) if p is not None else None, _ptr(out_dev),
        _ptr(ws), ws.numel() * ws.element_size(), _stream(stream))
    _check(rc, "ccs_decode_parallel_l0_async")


def ccs_decode_batch_async(probs, p: Params | None, out_dev, ws, stream=None):
    cnt = len(probs)
    arr = (Problem * cnt)(*probs)
    rc = lib().ccs_decode_batch_async(arr, cnt, ctypes.byref(p) if p is not None else None,
                                      _ptr(out_dev), _ptr(ws), ws.numel() * ws.element_size(),
                                      _stream(stream))
    _check(rc, "ccs_decode_batch_async")


def lddsr_alpha(d: int) -> int:
    """Parallel-LDDSR (Sec. 4.3.2): LDDSR accepts (j, omega) when more than d/2
    of j's rows hold omega; with the match-count score (Alg. 8) that is
    alpha = floor(d/2) + 1 and score_mode = SCORE_COUNT."""
    return d // 2 + 1


def ccs_autotune(probs, p: Params | None, ws, stream=None) -> list:
    """Time every launch shape per launch group of this batch and record the
    fastest in the library's table; returns the shape picked per group."""
    cnt = len(probs)
    arr = (Problem * cnt)(*probs)
    tuned = (ctypes.c_int32 * 4)()
    rc = lib().ccs_autotune(arr, cnt, ctypes.byref(p) if p is not None else None, _ptr(ws),
                            ws.numel() * ws.element_size(), _stream(stream), tuned)
    _check(rc, "ccs_autotune")
    return [int(t) for t in tuned]


def ccs_autotune_reset() -> None:
    lib().ccs_autotune_reset()


def ccs_autotune_get(dmax: int, fits: bool) -> int:
    """The recorded launch shape of a class on the current device (0: none)."""
    out = ctypes.c_int32()
    _check(lib().ccs_autotune_get(dmax, int(fits), ctypes.byref(out)), "ccs_autotune_get")
    return int(out.value)


def ccs_autotune_save(path: str) -> None:
    _check(lib().ccs_autotune_save(os.fsencode(path)), "ccs_autotune_save")


def ccs_autotune_load(path: str) -> None:
    _check(lib().ccs_autotune_load(os.fsencode(path)), "ccs_autotune_load")


RESULT_BYTES = ctypes.sizeof(Result)


def result_buffer(count: int, device="cuda"):
    """Device buffer for `count` ccs_result records."""
    import torch
    return torch.zeros(count * RESULT_BYTES, dtype=torch.uint8, device=device)


def results_from_device(buf, count: int) -> list[Result]:
    raw = bytes(buf[:count * RESULT_BYTES].cpu().numpy().tobytes())
    return [Result.from_buffer_copy(raw, i * RESULT_BYTES) for i in range(count)]


def ccs_decode_parallel_l0_noalloc(n, m, d, csc_rows, csr_ptr, csr_cols, y, x_hat, r, r0_hist,
                                   p: Params | None, stream=None) -> Result:
    """The decode without a caller workspace (library-held static scratch).
    Tensors are checked like every other decode's arrays; ints are raw device
    addresses, passed through unchecked as in C."""
    _need_abi_arrays("ccs_decode_parallel_l0_noalloc", n, m, d, csc_rows, csr_ptr, csr_cols, y,
                     x_hat, r, r0_hist, p)
    out = Result()
    rc = lib().ccs_decode_parallel_l0_noalloc(
        n, m, d, _ptr(csc_rows), _ptr(csr_ptr), _ptr(csr_cols), _ptr(y), _ptr(x_hat), _ptr(r),
        _ptr(r0_hist), ctypes.byref(p) if p is not None else None, ctypes.byref(out),
        _stream(stream))
    _check(rc, "ccs_decode_parallel_l0_noalloc")
    return out


def ccs_seeded_request_bytes(n: int, m: int, d: int, max_iter: int = 100, x_cap: int = 0) -> int:
    return int(lib().ccs_seeded_request_bytes(n, m, d, max_iter, x_cap))


def ccs_noalloc_scratch_bytes() -> int:
    return int(lib().ccs_noalloc_scratch_bytes())


def ccs_decode_batch(probs, p: Params | None, ws, stream=None) -> list[Result]:
    cnt = len(probs)
    arr = (Problem * cnt)(*probs)
    outs = (Result * cnt)()
    rc = lib().ccs_decode_batch(arr, cnt, ctypes.byref(p) if p is not None else None, outs,
                                _ptr(ws), ws.numel() * ws.element_size(), _stream(stream))
    _check(rc, "ccs_decode_batch")
    return list(outs)


def ccs_profile_begin():
    _check(lib().ccs_profile_begin(), "ccs_profile_begin")


def ccs_profile_end() -> dict:
    """{kernel name: (launches, total_ms)} for the kernels timed since begin."""
    arr = (KernelTime * K_COUNT)()
    _check(lib().ccs_profile_end(arr), "ccs_profile_end")
    return {KERNEL_NAMES.get(k, str(k)): (int(arr[k].launches), float(arr[k].total_ms))
            for k in range(K_COUNT) if arr[k].launches}


def ccs_profile_phases(iteration: int):
    """(score_us, residual_us, fp_us, stream_us, queue_us) of one iteration of
    the last profiled persistent launch, or None."""
    arr = (ctypes.c_double * 5)()
    if lib().ccs_profile_phases(iteration, arr) != CCS_OK:
        return None
    return tuple(arr)


def ccs_launch_count() -> int:
    return int(lib().ccs_launch_count())


# ---- conveniences -------------------------------------------------------------

def workspace(nbytes: int, device="cuda"):
    import torch
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def make_expander(n: int, m: int, d: int, seed: int, device="cuda", stream=None):
    """(csc_rows[n, d] int32, csr_ptr[m+1] int64, csr_cols[n*d] int32) on device."""
    import torch
    csc = torch.empty((n, d), dtype=torch.int32, device=device)
    ptr = torch.empty(m + 1, dtype=torch.int64, device=device)
    cols = torch.empty(n * d, dtype=torch.int32, device=device)
    ws = workspace(ccs_workspace_size(OP_MAKE_EXPANDER, n, m, d), device)
    ccs_make_expander(n, m, d, seed, csc, ptr, cols, ws, stream)
    return csc, ptr, cols


def measure(csr_ptr, csr_cols, x, m: int, d: int, stream=None):
    import torch
    n = x.numel()
    _need(csr_ptr, torch.int64, m + 1, "csr_ptr")
    _need(csr_cols, torch.int32, n * d, "csr_cols")
    _need(x, torch.float64, n, "x")
    y = torch.empty(m, dtype=torch.float64, device=x.device)
    ccs_measure(n, m, d, csr_ptr, csr_cols, x, y, stream)
    return y


def column_scales(n: int, seed: int, device="cuda", stream=None):
    """One i.i.d. scale per column on [1, 2), grid 2^-20 (Sec. 4.3.3)."""
    import torch
    s = torch.empty(n, dtype=torch.float64, device=device)
    _check(lib().ccs_column_scales(n, ctypes.c_uint64(seed), _ptr(s), _stream(stream)),
           "ccs_column_scales")
    return s


def measure_scaled(csr_ptr, csr_cols, scales, x, m: int, d: int, stream=None):
    """y = A diag(scales) x."""
    import torch
    n = x.numel()
    _need(csr_ptr, torch.int64, m + 1, "csr_ptr")
    _need(csr_cols, torch.int32, n * d, "csr_cols")
    _need(scales, torch.float64, n, "scales")
    _need(x, torch.float64, n, "x")
    y = torch.empty(m, dtype=torch.float64, device=x.device)
    _check(lib().ccs_measure_scaled(n, m, d, _ptr(csr_ptr), _ptr(csr_cols), _ptr(scales),
                                    _ptr(x), _ptr(y), _stream(stream)), "ccs_measure_scaled")
    return y


def unscale(scales, z, stream=None):
    """x = z / scales, the signal from the decode z of a scaled measurement."""
    import torch
    _need(z, torch.float64, scales.numel(), "z")
    x = torch.empty_like(z)
    _check(lib().ccs_unscale(scales.numel(), _ptr(scales), _ptr(z), _ptr(x), _stream(stream)),
           "ccs_unscale")
    return x


class DecodeOutput(dict):
    __getattr__ = dict.__getitem__


def decode_parallel_l0(csc_rows, csr_ptr, csr_cols, y, alpha=2, max_iter=100,
                       score_mode=SCORE_L0_DECREASE, engine=ENGINE_AUTO, history=True,
                       ws=None, out=None, stream=None, watchdog_ms=0,
                       debug_flags=0, schedule=0, shifted=False) -> DecodeOutput:
    """Parallel-l0 (Alg. 2) on one problem; returns x_hat, r (device tensors),
    r0_hist (host list), status, iterations, r0_final."""
    import torch
    if out is None:
        if not isinstance(y, torch.Tensor) or y.device.type != "cuda":
            raise TypeError("y must be a CUDA tensor")
        dev, m = y.device, y.numel()
        x_hat = torch.empty(csc_rows.shape[0], dtype=torch.float64, device=dev)
        r = torch.empty(m, dtype=torch.float64, device=dev)
        hist = torch.full((max_iter + 1,), -1, dtype=torch.int64, device=dev) if history else None
    else:
        x_hat, r, hist = out
    n, m, d = _need_problem(csc_rows, csr_ptr, csr_cols, y, x_hat, r, hist, max_iter,
                            outputs=out is not None)
    if ws is None:
        ws = workspace(ccs_workspace_size(OP_DECODE, n, m, d), y.device)
    elif not isinstance(ws, torch.Tensor) or ws.device.type != "cuda" or not ws.is_contiguous():
        raise TypeError("ws must be a contiguous CUDA tensor")
    p = params(alpha, max_iter, score_mode, engine, watchdog_ms, debug_flags, schedule, shifted)
    res = ccs_decode_parallel_l0(n, m, d, csc_rows, csr_ptr, csr_cols, y, x_hat, r, hist, p,
                                 ws, stream)
    h = hist[:res.iterations + 1].cpu().tolist() if hist is not None else None
    return DecodeOutput(x_hat=x_hat, r=r, r0_hist=h, status=res.status,
                        iterations=res.iterations, r0_final=res.r0_final, error=res.error,
                        row_driven=res.row_driven, row_entries=res.row_entries,
                        residual_form=res.residual_form)


def problem(csc_rows, csr_ptr, csr_cols, y, x_hat, r, r0_hist=None,
            max_iter: int | None = None) -> Problem:
    """Descriptor of one problem for the batch, graph and server calls.
    Every array is checked (CUDA, dtype, contiguous, size); r0_hist needs
    max_iter + 1 entries when max_iter is given, else at least one."""
    n, m, d = _need_problem(csc_rows, csr_ptr, csr_cols, y, x_hat, r, r0_hist, max_iter)
    return Problem(n, m, d, 0, _ptr(csc_rows), _ptr(csr_ptr), _ptr(csr_cols),
                   _ptr(y), _ptr(x_hat), _ptr(r), _ptr(r0_hist))


def decode_batch(items, alpha=2, max_iter=100, score_mode=SCORE_L0_DECREASE,
                 engine=ENGINE_AUTO, history=False, ws=None, stream=None, debug_flags=0,
                 shifted=False):
    """items: list of (csc_rows, csr_ptr, csr_cols, y).  Returns a list of
    DecodeOutput, one per problem, from a single ccs_decode_batch call."""
    import torch
    probs, outs = [], []
    for csc, ptr, cols, y in items:
        n, d = csc.shape
        m = y.numel()
        x_hat = torch.empty(n, dtype=torch.float64, device=y.device)
        r = torch.empty(m, dtype=torch.float64, device=y.device)
        hist = torch.full((max_iter + 1,), -1, dtype=torch.int64, device=y.device) \
            if history else None
        outs.append((x_hat, r, hist))
        probs.append(problem(csc, ptr, cols, y, x_hat, r, hist, max_iter))
    if ws is None:
        ws = workspace(ccs_batch_workspace_size(probs), items[0][3].device)
    p = params(alpha, max_iter, score_mode, engine, debug_flags=debug_flags, shifted=shifted)
    res = ccs_decode_batch(probs, p, ws, stream)
    result = []
    for (x_hat, r, hist), rr in zip(outs, res):
        h = hist[:rr.iterations + 1].cpu().tolist() if hist is not None else None
        result.append(DecodeOutput(x_hat=x_hat, r=r, r0_hist=h, status=rr.status,
                                   iterations=rr.iterations, r0_final=rr.r0_final,
                                   error=rr.error, residual_form=rr.residual_form))
    return result


# ---- CUDA graph of a batched decode ----------------------------------------------

class BatchGraph:
    """A batched decode captured once (ccs_batch_graph_create), replayed by
    launch().  Keeps the problems' tensors, workspace and result buffer."""

    def __init__(self, probs, p: Params | None = None, device="cuda"):
        self.probs = list(probs)
        arr = (Problem * len(self.probs))(*self.probs)
        self.ws = workspace(ccs_batch_workspace_size(self.probs), device)
        self.results = result_buffer(len(self.probs), device)
        self._h = ctypes.c_void_p()
        _check(lib().ccs_batch_graph_create(arr, len(self.probs),
                                            ctypes.byref(p) if p is not None else None,
                                            _ptr(self.results), _ptr(self.ws),
                                            self.ws.numel(), ctypes.byref(self._h)),
               "ccs_batch_graph_create")

    def launch(self, stream=None):
        _check(lib().ccs_graph_launch(self._h, _stream(stream)), "ccs_graph_launch")

    def read_results(self):
        return results_from_device(self.results, len(self.probs))

    def close(self):
        if self._h:
            lib().ccs_graph_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- serving -------------------------------------------------------------------

class Server:
    """Continuous-batching decode server (ccs_server_* in include/ccs.h).

    `pool_bytes` of device memory (a torch tensor held here) is the budget
    for request state.  Requests are (csc_rows, csr_ptr, csr_cols, y, x_hat,
    r[, r0_hist]) device tensors that must stay alive until collected."""

    def __init__(self, pool_bytes: int, max_batch: int = 512, iters_per_round: int = 2,
                 alpha=2, max_iter=100, score_mode=SCORE_L0_DECREASE, device="cuda",
                 stream=None):
        import torch
        self.pool = torch.empty(int(pool_bytes), dtype=torch.uint8, device=device)
        cfg = ServerConfig(self.pool.data_ptr(), int(pool_bytes), max_batch, iters_per_round,
                           params(alpha, max_iter, score_mode))
        self._h = ctypes.c_void_p()
        self._stream = torch.cuda.Stream(device=device) if stream is None else stream
        self.max_iter = max_iter
        _check(lib().ccs_server_create(ctypes.byref(cfg), self._stream.cuda_stream,
                                       ctypes.byref(self._h)), "ccs_server_create")
        self._keep = {}

    def submit(self, csc_rows, csr_ptr, csr_cols, y, x_hat, r, r0_hist=None) -> int:
        pb = problem(csc_rows, csr_ptr, csr_cols, y, x_hat, r, r0_hist, self.max_iter)
        t = ctypes.c_int64()
        _check(lib().ccs_server_submit(self._h, ctypes.byref(pb), ctypes.byref(t)),
               "ccs_server_submit")
        self._keep[t.value] = (csc_rows, csr_ptr, csr_cols, y, x_hat, r, r0_hist)
        return t.value

    def submit_seeded(self, n: int, m: int, d: int, a_seed: int, y, x_hat=None, r=None,
                      r0_hist=None, nonzeros=None) -> int:
        """A request whose A the server draws from `a_seed` into its pool
        (ccs_server_submit_seeded).  y, x_hat, r, r0_hist are HOST numpy
        arrays (float64 m, float64 n, float64 m, int64 >= max_iter + 1),
        kept alive here until the result is collected.  nonzeros = (idx
        int64[cap], val float64[cap], nnz int64[1]) asks for x_hat as its
        nonzero entries instead of (or besides) the dense x_hat."""
        import numpy as np

        def need(a, dtype, size, name, at_least=False):
            if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags.c_contiguous \
                    or (a.size < size if at_least else a.size != size):
                raise ValueError(f"{name}: need a contiguous {np.dtype(dtype)} numpy array "
                                 f"of {'at least ' if at_least else ''}{size} elements")
        need(y, np.float64, m, "y")
        if x_hat is None and nonzeros is None:
            raise ValueError("need x_hat or nonzeros")
        if x_hat is not None:
            need(x_hat, np.float64, n, "x_hat")
        if r is not None:
            need(r, np.float64, m, "r")
        if r0_hist is not None:
            need(r0_hist, np.int64, self.max_iter + 1, "r0_hist", at_least=True)
        cap, nz_args = 0, (None, None, 0, None)
        if nonzeros is not None:
            idx, val, nnz = nonzeros
            cap = idx.size if isinstance(idx, np.ndarray) else 0
            if cap < 1:
                raise ValueError("nonzeros: idx needs at least one entry")
            need(idx, np.int64, cap, "nonzeros idx")
            need(val, np.float64, cap, "nonzeros val")
            need(nnz, np.int64, 1, "nonzeros nnz")
            nz_args = (idx.ctypes.data, val.ctypes.data, cap, nnz.ctypes.data)
        req = SeededRequest(n, m, d, 0, a_seed & (2 ** 64 - 1), y.ctypes.data,
                            x_hat.ctypes.data if x_hat is not None else None,
                            r.ctypes.data if r is not None else None,
                            r0_hist.ctypes.data if r0_hist is not None else None, *nz_args)
        t = ctypes.c_int64()
        _check(lib().ccs_server_submit_seeded(self._h, ctypes.byref(req), ctypes.byref(t)),
               "ccs_server_submit_seeded")
        self._keep[t.value] = (y, x_hat, r, r0_hist, nonzeros)
        return t.value

    def poll(self, ticket: int):
        info = TicketInfo()
        rc = lib().ccs_server_poll(self._h, ticket, ctypes.byref(info))
        if rc == CCS_EBUSY:
            return None
        _check(rc, "ccs_server_poll")
        self._keep.pop(ticket, None)
        return info

    def wait(self, ticket: int, timeout_ms: int = 60000):
        info = TicketInfo()
        rc = lib().ccs_server_wait(self._h, ticket, ctypes.byref(info), timeout_ms)
        if rc == CCS_EBUSY:
            return None
        _check(rc, "ccs_server_wait")
        self._keep.pop(ticket, None)
        return info

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().ccs_server_stats_get(self._h, ctypes.byref(st)), "ccs_server_stats_get")
        return {f: getattr(st, f) for f, _ in ServerStats._fields_ if f != "reserved"}

    def close(self):
        if self._h:
            rc = lib().ccs_server_destroy(self._h)
            self._h = ctypes.c_void_p()
            _check(rc, "ccs_server_destroy")

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def serve_poisson(server: Server, requests, arrivals_s, timeout_ms: int = 120000):
    """Submit requests[i] at time arrivals_s[i] (seconds from now) and collect
    every result.  Returns a list of TicketInfo in submission order."""
    import time
    tickets, infos = [], [None] * len(requests)
    done = threading.Event()

    def collect():
        i = 0
        while i < len(requests):
            if i >= len(tickets):
                time.sleep(0.0001)
                continue
            info = server.wait(tickets[i], timeout_ms)
            if info is None:
                raise RuntimeError(f"request {i} not finished within {timeout_ms} ms")
            infos[i] = info
            i += 1
        done.set()

    th = threading.Thread(target=collect, daemon=True)
    th.start()
    t0 = time.perf_counter()
    for req, at in zip(requests, arrivals_s):
        delay = t0 + at - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        tickets.append(server.submit(*req))
    th.join()
    return infos


def serve_stream(server: Server, request_of, count: int, arrivals_s, ring: int,
                 timeout_ms: int = 120000):
    """Open-loop serving of `count` requests: request q, the tuple
    `request_of(q)`, is submitted at arrivals_s[q] (seconds from now).
    `request_of` may hand out output buffers from a ring of `ring` slots
    (requests q and q + ring share one), so request q is submitted only once
    request q - ring has been collected.  Returns (TicketInfo list in
    submission order, number of submissions that waited for their slot)."""
    import time
    tickets, infos = [], [None] * count
    state = {"collected": 0, "error": None}

    def collect():
        try:
            i = 0
            while i < count:
                if i >= len(tickets):
                    time.sleep(0.0001)
                    continue
                info = server.wait(tickets[i], timeout_ms)
                if info is None:
                    raise RuntimeError(f"request {i} not finished within {timeout_ms} ms")
                infos[i] = info
                i += 1
                state["collected"] = i
        except BaseException as e:  # re-raised on the submitting thread
            state["error"] = e

    th = threading.Thread(target=collect, daemon=True)
    th.start()
    waited = 0
    t0 = time.perf_counter()
    for q in range(count):
        delay = t0 + arrivals_s[q] - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        if q >= ring and state["collected"] <= q - ring:
            waited += 1
            limit = time.perf_counter() + timeout_ms / 1000.0
            while state["collected"] <= q - ring and state["error"] is None:
                if time.perf_counter() > limit:
                    raise RuntimeError(f"slot of request {q} not free within {timeout_ms} ms")
                time.sleep(0.00005)
        if state["error"] is not None:
            break
        tickets.append(server.submit(*request_of(q)))
    th.join()
    if state["error"] is not None:
        raise state["error"]
    return infos, waited


def serve_seeded(server: Server, requests, arrivals_s, on_done, timeout_ms: int = 120000,
                 sampler=None, sample_every_s: float = 0.002, nonzeros_cap=None):
    """Open-loop serving of seeded requests: requests[q] = (n, m, d, a_seed,
    y host array) is submitted at arrivals_s[q] (seconds from now) with a
    fresh host x_hat buffer -- or, with nonzeros_cap(q) given, fresh
    (idx, val, nnz) buffers for x_hat's nonzeros; when its result arrives
    (collected in submission order) on_done(q, info, out) is called (out:
    the x_hat array, or the (idx, val, nnz) tuple) and the buffers are
    released.  With `sampler` (a list), (t, inflight, pending, bytes_in_use)
    from ccs_server_stats is appended every `sample_every_s` while requests
    are outstanding.  Returns the TicketInfo list in submission order."""
    import time

    import numpy as np
    count = len(requests)
    tickets, bufs, infos = [], {}, [None] * count
    state = {"error": None, "done": False}

    def collect():
        try:
            for i in range(count):
                while i >= len(tickets):
                    if state["error"] is not None:
                        return
                    time.sleep(0.0001)
                info = server.wait(tickets[i], timeout_ms)
                if info is None:
                    raise RuntimeError(f"request {i} not finished within {timeout_ms} ms")
                infos[i] = info
                on_done(i, info, bufs.pop(i))
        except BaseException as e:  # re-raised on the submitting thread
            state["error"] = e
        finally:
            state["done"] = True

    def sample(t0):
        while not state["done"]:
            st = server.stats()
            sampler.append((time.perf_counter() - t0, st["inflight"], st["pending"],
                            st["bytes_in_use"]))
            time.sleep(sample_every_s)

    th = threading.Thread(target=collect, daemon=True)
    th.start()
    t0 = time.perf_counter()
    ts = None
    if sampler is not None:
        ts = threading.Thread(target=sample, args=(t0,), daemon=True)
        ts.start()
    for q, (n, m, d, a_seed, y) in enumerate(requests):
        delay = t0 + arrivals_s[q] - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        if state["error"] is not None:
            break
        if nonzeros_cap is None:
            x = np.empty(n, dtype=np.float64)
            bufs[q] = x
            tickets.append(server.submit_seeded(n, m, d, a_seed, y, x))
        else:
            cap = max(1, int(nonzeros_cap(q)))
            nz = (np.empty(cap, dtype=np.int64), np.empty(cap, dtype=np.float64),
                  np.zeros(1, dtype=np.int64))
            bufs[q] = nz
            tickets.append(server.submit_seeded(n, m, d, a_seed, y, None, nonzeros=nz))
    th.join()
    if ts is not None:
        ts.join()
    if state["error"] is not None:
        raise state["error"]
    return infos
