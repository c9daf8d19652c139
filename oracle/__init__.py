"""CPU oracle for expander l0-decoding -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does; it
shares no code with it.  The oracle is plain single-threaded C
(``ccs_oracle.c``) compiled with gcc, IEEE binary64, ``-ffp-contract=off``;
this module compiles it on first use and wraps it with ctypes.

Every routine follows Mendoza-Smith & Tanner, "Expander l0-decoding":
Alg. 1 (Serial-l0), Alg. 2 (Parallel-l0), the selection rule Eq. (15) and the
score of Alg. 8, with the readings listed at the top of ``ccs_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ccs_oracle.c")
_HDR = os.path.join(_HERE, "ccs_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libccs_oracle.so")

SCORE_L0_DECREASE = 0
SCORE_COUNT = 1
CONVERGED, STALLED, MAX_ITER = 0, 1, 2
STATUS_NAMES = {CONVERGED: "converged", STALLED: "stalled", MAX_ITER: "max_iter"}

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, -O2, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    fresh = os.path.exists(_SO) and all(
        os.path.getmtime(_SO) >= os.path.getmtime(f) for f in (_SRC, _HDR))
    if fresh and not force:
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _SO)
    return _SO


class Outcome(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("r0_final", ctypes.c_int64)]


TRACE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                            ctypes.POINTER(ctypes.c_uint8),
                            ctypes.POINTER(ctypes.c_double))

_P = ctypes.c_void_p


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # CCS_ORACLE_LIB names another build of ccs_oracle.c to load: the
            # planted-mistake test runs the pins against broken copies
            l = ctypes.CDLL(os.environ.get("CCS_ORACLE_LIB") or build())
            i32, i64, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
            l.oracle_splitmix64_next.argtypes = [ctypes.POINTER(u64)]
            l.oracle_splitmix64_next.restype = u64
            l.oracle_make_expander.argtypes = [i32, i32, i32, u64, _P]
            l.oracle_transpose.argtypes = [i32, i32, i32, _P, _P, _P]
            l.oracle_column_scales.argtypes = [i32, u64, _P]
            l.oracle_measure_scaled.argtypes = [i32, _P, _P, _P, _P, _P]
            l.oracle_unscale.argtypes = [i32, _P, _P, _P]
            l.oracle_measure.argtypes = [i32, _P, _P, _P, _P]
            l.oracle_residual.argtypes = [i32, _P, _P, _P, _P, _P]
            l.oracle_l0.argtypes = [i32, _P]
            l.oracle_l0.restype = i64
            l.oracle_score_column.argtypes = [i32, _P, _P, i32, i32, _P, _P, _P]
            l.oracle_score_column_shifted.argtypes = [i32, _P, _P, i32, i32, i32, _P, _P, _P]
            l.oracle_score_all.argtypes = [i32, i32, _P, _P, i32, i32, i32, _P, _P, _P]
            l.oracle_score_all.restype = i64
            l.oracle_parallel_l0.argtypes = [i32, i32, i32, _P, _P, i32, i32, i32, i32,
                                             _P, _P, _P, TRACE_FN, _P,
                                             ctypes.POINTER(Outcome)]
            l.oracle_serial_l0.argtypes = [i32, i32, i32, _P, _P, i32, i32, i32, i32,
                                           _P, _P, _P, ctypes.POINTER(Outcome)]
            _lib = l
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.c_void_p)


def splitmix64(seed: int, count: int) -> list[int]:
    st = ctypes.c_uint64(seed)
    return [lib().oracle_splitmix64_next(ctypes.byref(st)) for _ in range(count)]


def make_expander(n: int, m: int, d: int, seed: int) -> np.ndarray:
    """CSC row indices, shape (n, d), int32, each column ascending (R5)."""
    rows = np.empty((n, d), dtype=np.int32)
    rc = lib().oracle_make_expander(n, m, d, seed, _ptr(rows))
    if rc:
        raise ValueError(f"oracle_make_expander rejected n={n} m={m} d={d}")
    return rows


def transpose(csc_rows: np.ndarray, m: int):
    n, d = csc_rows.shape
    ptr = np.empty(m + 1, dtype=np.int64)
    cols = np.empty(n * d, dtype=np.int32)
    rc = lib().oracle_transpose(n, m, d, _ptr(np.ascontiguousarray(csc_rows)),
                                _ptr(ptr), _ptr(cols))
    if rc:
        raise ValueError("oracle_transpose failed")
    return ptr, cols


def measure(csc_rows: np.ndarray, m: int, x: np.ndarray) -> np.ndarray:
    ptr, cols = transpose(csc_rows, m)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(m, dtype=np.float64)
    lib().oracle_measure(m, _ptr(ptr), _ptr(cols), _ptr(x), _ptr(y))
    return y


def column_scales(n: int, seed: int) -> np.ndarray:
    """Column scales of Sec. 4.3.3 (reading R12): s_j on [1, 2), grid 2^-20."""
    s = np.empty(n, dtype=np.float64)
    if lib().oracle_column_scales(n, ctypes.c_uint64(seed), _ptr(s)):
        raise ValueError("oracle_column_scales: bad arguments")
    return s


def measure_scaled(csc_rows: np.ndarray, m: int, s: np.ndarray, x: np.ndarray) -> np.ndarray:
    """y = A diag(s) x, ordered row sums of the products s_j x_j."""
    ptr, cols = transpose(csc_rows, m)
    y = np.empty(m, dtype=np.float64)
    lib().oracle_measure_scaled(m, _ptr(ptr), _ptr(cols),
                                _ptr(np.ascontiguousarray(s, dtype=np.float64)),
                                _ptr(np.ascontiguousarray(x, dtype=np.float64)), _ptr(y))
    return y


def unscale(s: np.ndarray, z: np.ndarray) -> np.ndarray:
    x = np.empty(s.size, dtype=np.float64)
    lib().oracle_unscale(s.size, _ptr(np.ascontiguousarray(s, dtype=np.float64)),
                         _ptr(np.ascontiguousarray(z, dtype=np.float64)), _ptr(x))
    return x


def residual(csc_rows: np.ndarray, m: int, y: np.ndarray, x_hat: np.ndarray):
    ptr, cols = transpose(csc_rows, m)
    r = np.empty(m, dtype=np.float64)
    lib().oracle_residual(m, _ptr(ptr), _ptr(cols),
                          _ptr(np.ascontiguousarray(y, dtype=np.float64)),
                          _ptr(np.ascontiguousarray(x_hat, dtype=np.float64)),
                          _ptr(r))
    return r


def l0(r: np.ndarray) -> int:
    r = np.ascontiguousarray(r, dtype=np.float64)
    return int(lib().oracle_l0(r.size, _ptr(r)))


def score_column(values_rows: np.ndarray, r: np.ndarray, alpha: int = 2,
                 score_mode: int = SCORE_L0_DECREASE):
    rows = np.ascontiguousarray(values_rows, dtype=np.int32)
    r = np.ascontiguousarray(r, dtype=np.float64)
    om = ctypes.c_double()
    sc = ctypes.c_int32()
    ct = ctypes.c_int32()
    acc = lib().oracle_score_column(rows.size, _ptr(rows), _ptr(r), alpha,
                                    score_mode, ctypes.byref(om), ctypes.byref(sc),
                                    ctypes.byref(ct))
    return bool(acc), om.value, sc.value, ct.value


def score_column_shifted(values_rows: np.ndarray, r: np.ndarray, pos: int, alpha: int = 2,
                         score_mode: int = SCORE_L0_DECREASE):
    """Shifted score (Sec. 4.3.1): the candidate is r at row pos of the column."""
    rows = np.ascontiguousarray(values_rows, dtype=np.int32)
    r = np.ascontiguousarray(r, dtype=np.float64)
    om = ctypes.c_double()
    sc = ctypes.c_int32()
    ct = ctypes.c_int32()
    acc = lib().oracle_score_column_shifted(rows.size, _ptr(rows), _ptr(r), pos, alpha,
                                            score_mode, ctypes.byref(om), ctypes.byref(sc),
                                            ctypes.byref(ct))
    if acc < 0:
        raise ValueError("oracle_score_column_shifted: bad arguments")
    return bool(acc), om.value, sc.value, ct.value


def score_all(csc_rows: np.ndarray, r: np.ndarray, alpha: int = 2,
              score_mode: int = SCORE_L0_DECREASE, shift_pos: int = -1):
    n, d = csc_rows.shape
    acc = np.empty(n, dtype=np.uint8)
    om = np.empty(n, dtype=np.float64)
    sc = np.empty(n, dtype=np.int32)
    lib().oracle_score_all(n, d, _ptr(np.ascontiguousarray(csc_rows)),
                           _ptr(np.ascontiguousarray(r, dtype=np.float64)), alpha,
                           score_mode, shift_pos, _ptr(acc), _ptr(om), _ptr(sc))
    return acc.astype(bool), om, sc


def parallel_l0(csc_rows: np.ndarray, m: int, y: np.ndarray, alpha: int = 2,
                max_iter: int = 100, score_mode: int = SCORE_L0_DECREASE,
                trace: bool = False, shifted: bool = False):
    """Alg. 2 (shifted: the variant of Sec. 4.3.1).  Returns dict(x_hat, r,
    r0_hist, status, iterations, r0_final[, trace])."""
    n, d = csc_rows.shape
    x_hat = np.empty(n, dtype=np.float64)
    r = np.empty(m, dtype=np.float64)
    hist = np.full(max_iter + 1, -1, dtype=np.int64)
    out = Outcome()
    steps = []

    def _cb(_ctx, it, nn, acc_p, om_p):
        acc = np.ctypeslib.as_array(acc_p, shape=(nn,)).astype(bool)
        om = np.ctypeslib.as_array(om_p, shape=(nn,))
        idx = np.nonzero(acc)[0]
        steps.append((int(it), idx.copy(), om[idx].copy()))

    cb = TRACE_FN(_cb) if trace else TRACE_FN()
    rc = lib().oracle_parallel_l0(n, m, d, _ptr(np.ascontiguousarray(csc_rows)),
                                  _ptr(np.ascontiguousarray(y, dtype=np.float64)),
                                  alpha, max_iter, score_mode, int(shifted), _ptr(x_hat),
                                  _ptr(r), _ptr(hist), cb, None, ctypes.byref(out))
    if rc:
        raise ValueError(f"oracle_parallel_l0 failed ({rc})")
    res = dict(x_hat=x_hat, r=r, r0_hist=hist[:out.iterations + 1].copy(),
               status=out.status, iterations=out.iterations, r0_final=out.r0_final)
    if trace:
        res["trace"] = steps
    return res


def serial_l0(csc_rows: np.ndarray, m: int, y: np.ndarray, alpha: int = 2,
              max_iter: int = 100, score_mode: int = SCORE_L0_DECREASE,
              shifted: bool = False):
    """Alg. 1, one sweep over j = 0..n-1 per iteration."""
    n, d = csc_rows.shape
    x_hat = np.empty(n, dtype=np.float64)
    r = np.empty(m, dtype=np.float64)
    hist = np.full(max_iter + 1, -1, dtype=np.int64)
    out = Outcome()
    rc = lib().oracle_serial_l0(n, m, d, _ptr(np.ascontiguousarray(csc_rows)),
                                _ptr(np.ascontiguousarray(y, dtype=np.float64)),
                                alpha, max_iter, score_mode, int(shifted), _ptr(x_hat),
                                _ptr(r), _ptr(hist), ctypes.byref(out))
    if rc:
        raise ValueError(f"oracle_serial_l0 failed ({rc})")
    return dict(x_hat=x_hat, r=r, r0_hist=hist[:out.iterations + 1].copy(),
                status=out.status, iterations=out.iterations, r0_final=out.r0_final)
