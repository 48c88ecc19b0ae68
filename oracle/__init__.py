"""FP64 CPU oracle for FastConv and the multi-scale TTC pipeline (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import this package.  It shares no code with the CUDA library and never
imports it.  The arithmetic lives in ``oracle.c`` (plain C, double precision,
compiled by :func:`build` with ``gcc -O2 -ffp-contract=off``); this module only
marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

FLAG_SINGULAR = 1
FLAG_C_ZERO = 2
FLAG_RECEDING = 4

SUM_NAMES = ("ExEx", "ExEy", "EyEy", "GEx", "GEy", "GG", "ExEt", "EyEt", "GEt", "EtEt")

RESULT_DTYPE = np.dtype([
    ("sums", np.float64, (10,)),
    ("abssums", np.float64, (10,)),
    ("A", np.float64), ("B", np.float64), ("C", np.float64),
    ("ttc", np.float64), ("x0", np.float64), ("y0", np.float64),
    ("resid", np.float64),
    ("n", np.int64),
    ("level", np.int32), ("flags", np.int32),
])

_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``_build/liboracle.so`` (host compiler, no GPU)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                        _SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            lib.oracle_fastconv_nd.argtypes = [_f64p, _i64p, ctypes.c_int, _f64p, _i64p, _f64p, _f64p]
            lib.oracle_fastconv_points.argtypes = [_f64p, _i64p, ctypes.c_int, _f64p, _i64p, _i64p,
                                                   ctypes.c_int64, _f64p, _f64p]
            lib.oracle_conv_out_dims.argtypes = [ctypes.c_int, _i64p, _i64p, _i64p]
            lib.oracle_downsample.argtypes = [_f64p, ctypes.c_int, ctypes.c_int, _f64p]
            lib.oracle_derivatives.argtypes = [_f64p, _f64p, ctypes.c_int, ctypes.c_int, _f64p, _f64p, _f64p]
            lib.oracle_gradient.argtypes = [_f64p, ctypes.c_int, ctypes.c_int, _f64p, _f64p]
            lib.oracle_sums.argtypes = [_f64p, _f64p, _f64p, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_double, _f64p, _f64p]
            lib.oracle_solve.argtypes = [_f64p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
            lib.oracle_ttc_pair.argtypes = [_f64p, _f64p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_void_p]
            lib.oracle_select_level.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
            assert lib.oracle_result_size() == RESULT_DTYPE.itemsize, "oracle_result layout mismatch"
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a: np.ndarray, t=_f64p):
    return a.ctypes.data_as(t)


def conv_out_dims(dims, kdims) -> tuple:
    return tuple(int(n) + int(k) - 1 for n, k in zip(dims, kdims))


def fastconv_nd(E, k, with_abs: bool = False):
    """Full n-D convolution of E with k (Eq. conv2, full extent), FP64.

    Returns ``out`` or ``(out, |E| conv |k|)`` when ``with_abs``.
    """
    E = _f64(E)
    k = _f64(k)
    if E.ndim != k.ndim or E.ndim < 1:
        raise ValueError("E and k must have the same rank >= 1")
    lib = _load()
    dims = np.array(E.shape, dtype=np.int64)
    kd = np.array(k.shape, dtype=np.int64)
    out = np.empty(conv_out_dims(E.shape, k.shape), dtype=np.float64)
    oabs = np.empty_like(out) if with_abs else None
    rc = lib.oracle_fastconv_nd(_p(E), _p(dims, _i64p), E.ndim, _p(k), _p(kd, _i64p), _p(out),
                                _p(oabs) if with_abs else None)
    if rc != 0:
        raise ValueError(f"oracle_fastconv_nd failed ({rc})")
    return (out, oabs) if with_abs else out


def fastconv_points(E, k, points):
    """Full convolution at the given output linear indices: (values, abs-values)."""
    E = _f64(E)
    k = _f64(k)
    lib = _load()
    dims = np.array(E.shape, dtype=np.int64)
    kd = np.array(k.shape, dtype=np.int64)
    pts = np.ascontiguousarray(np.asarray(points, dtype=np.int64))
    out = np.empty(pts.shape[0], dtype=np.float64)
    oabs = np.empty_like(out)
    rc = lib.oracle_fastconv_points(_p(E), _p(dims, _i64p), E.ndim, _p(k), _p(kd, _i64p),
                                    _p(pts, _i64p), pts.shape[0], _p(out), _p(oabs))
    if rc != 0:
        raise ValueError(f"oracle_fastconv_points failed ({rc})")
    return out, oabs


def downsample(img):
    img = _f64(img)
    H, W = img.shape
    out = np.empty((H // 2, W // 2), dtype=np.float64)
    _load().oracle_downsample(_p(img), H, W, _p(out))
    return out


def gradient(E):
    """Gradient magnitude and direction of one image (Sec. II, Eq. Emag, Eq. Eangle),
    each (H-1) x (W-1)."""
    E = _f64(E)
    H, W = E.shape
    mag = np.empty((H - 1, W - 1), dtype=np.float64)
    ang = np.empty((H - 1, W - 1), dtype=np.float64)
    _load().oracle_gradient(_p(E), H, W, _p(mag), _p(ang))
    return mag, ang


def derivatives(E0, E1):
    """(Ex, Ey, Et), each (H-1) x (W-1)."""
    E0 = _f64(E0)
    E1 = _f64(E1)
    H, W = E0.shape
    outs = [np.empty((H - 1, W - 1), dtype=np.float64) for _ in range(3)]
    _load().oracle_derivatives(_p(E0), _p(E1), H, W, *[_p(o) for o in outs])
    return tuple(outs)


def sums(Ex, Ey, Et, cx: float, cy: float):
    """(sums[10], abssums[10]) with G = x Ex + y Ey, x = j + 1/2 - cx, y = i + 1/2 - cy."""
    Ex, Ey, Et = _f64(Ex), _f64(Ey), _f64(Et)
    h, w = Ex.shape
    s = np.empty(10, dtype=np.float64)
    a = np.empty(10, dtype=np.float64)
    _load().oracle_sums(_p(Ex), _p(Ey), _p(Et), h, w, float(cx), float(cy), _p(s), _p(a))
    return s, a


def solve(s, mode: int = 1, level: int = 0):
    """Solve from ten sums: one RESULT_DTYPE record."""
    s = _f64(s)
    r = np.zeros(1, dtype=RESULT_DTYPE)
    _load().oracle_solve(_p(s), int(mode), int(level), r.ctypes.data)
    return r[0]


def ttc_pair(E0, E1, levels: int = 1, mode: int = 1) -> np.ndarray:
    """Whole chain for one frame pair: RESULT_DTYPE array of length ``levels``."""
    E0 = _f64(E0)
    E1 = _f64(E1)
    H, W = E0.shape
    res = np.zeros(levels, dtype=RESULT_DTYPE)
    rc = _load().oracle_ttc_pair(_p(E0), _p(E1), H, W, int(levels), int(mode), res.ctypes.data)
    if rc != 0:
        raise ValueError(f"oracle_ttc_pair: bad shape/levels ({rc})")
    return res


def select_level(results: np.ndarray, rule: int = 0) -> int:
    """Multi-scale selection (Sec. V-B) over per-level results of one pair."""
    r = np.ascontiguousarray(results, dtype=RESULT_DTYPE)
    return int(_load().oracle_select_level(r.ctypes.data, r.shape[0], int(rule)))


def _pair_job(job):
    prev, cur, levels, mode = job
    return ttc_pair(prev, cur, levels=levels, mode=mode)


def ttc_pairs_parallel(frames, npairs: int, levels: int, mode: int, workers: int):
    """ttc_pair on the first npairs consecutive pairs of `frames` (host array) spread over
    `workers` processes (spawned, so that a process that already uses the GPU can call
    it); returns (results, seconds of the timed pass).  A first untimed pass starts the
    processes and loads the library in each; for timing the baseline on all host cores."""
    import multiprocessing as mp
    import time

    build()
    jobs = [(frames[t], frames[t + 1], levels, mode) for t in range(npairs)]
    with mp.get_context("spawn").Pool(workers) as pool:
        pool.map(_pair_job, jobs[:workers], chunksize=1)
        t0 = time.perf_counter()
        out = pool.map(_pair_job, jobs, chunksize=1)
        dt = time.perf_counter() - t0
    return out, dt


def _list_job(job):
    a, b, levels, mode = job
    return ttc_pair(a, b, levels=levels, mode=mode)


def ttc_pairs_list(pairs, levels: int, mode: int, workers: int):
    """ttc_pair on every (E0, E1) host pair of `pairs` (frames of any sizes), spread over
    `workers` spawned processes (workers <= 1: in this process); returns the list of
    per-pair results in order and the seconds taken."""
    import time

    build()
    jobs = [(a, b, levels, mode) for a, b in pairs]
    t0 = time.perf_counter()
    if workers <= 1:
        out = [_list_job(j) for j in jobs]
    else:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as pool:
            out = pool.map(_list_job, jobs, chunksize=1)
    return out, time.perf_counter() - t0

