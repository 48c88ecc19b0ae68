"""GB300 (sm_103a) FastConv and multi-scale time-to-contact, Python binding.

Paper: "Accelerated Convolutions for Efficient Multi-Scale Time to Contact
Computation in Julia" (Amini, Horn, Edelman).

This module only marshals arguments to the C ABI of ``libfastttc.so`` (declared in
``include/fastttc.h``): torch tensors supply device memory and the current CUDA
stream; every step of the computation runs in the library's CUDA kernels.  There
is no CPU fallback: if the library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np
import torch

from . import build as _build

__all__ = [
    "FtError", "lib", "load", "fastconv_out_dims", "fastconv_nd", "fastconv_check", "fastconv_separable", "fastconv_fft",
    "FftPlan", "fastconv",
    "factor_kernel", "ttc_derivatives", "gradient",
    "ttc_solve_noalloc",
    "TtcContext", "RESULT_DTYPE", "results_to_numpy", "select_level",
    "MODE_TTC", "MODE_FOE", "FLAG_SINGULAR", "FLAG_C_ZERO", "FLAG_RECEDING", "MAX_LEVELS",
    "MAX_NDIM",
]

MODE_TTC, MODE_FOE = 0, 1
DTYPE_U8, DTYPE_F32 = 0, 1
FLAG_SINGULAR, FLAG_C_ZERO, FLAG_RECEDING, FLAG_TIMEOUT, FLAG_BOUNDS = 1, 2, 4, 8, 16
ERR_TIMEOUT = 6
MAX_LEVELS = 7
MAX_NDIM = 8

# mirror of ttc_level_result (152 bytes)
RESULT_DTYPE = np.dtype([
    ("sums", np.float64, (10,)),
    ("A", np.float64), ("B", np.float64), ("C", np.float64),
    ("ttc", np.float64), ("x0", np.float64), ("y0", np.float64),
    ("resid", np.float64),
    ("n", np.int64),
    ("level", np.int32), ("flags", np.int32),
])
assert RESULT_DTYPE.itemsize == 152

# mirror of ttc_served (one report of the serving runtime)
SERVED_DTYPE = np.dtype([
    ("records", RESULT_DTYPE, (7,)),
    ("t_arrival", np.float64), ("seq", np.int64),
    ("stream", np.int32), ("status", np.int32), ("level", np.int32), ("pad", np.int32),
])
assert SERVED_DTYPE.itemsize == 1096

_lib = None
_i64p = ctypes.POINTER(ctypes.c_int64)
_vp = ctypes.c_void_p


class PairDesc(ctypes.Structure):
    """Mirror of ttc_pair_desc."""
    _fields_ = [("prev", ctypes.c_void_p), ("cur", ctypes.c_void_p), ("H", ctypes.c_int), ("W", ctypes.c_int),
                ("pitch_bytes", ctypes.c_int64), ("prev_pyramid", ctypes.c_void_p), ("cur_pyramid", ctypes.c_void_p)]


class FtError(RuntimeError):
    def __init__(self, status: int, what: str):
        name = _lib.ft_status_string(status).decode() if _lib is not None else str(status)
        extra = ""
        if _lib is not None and status == 5:
            extra = ": " + _lib.ft_last_cuda_error().decode()
        super().__init__(f"{what} failed with {name}{extra}")
        self.status = status


def load(path: Optional[str] = None):
    """Load libfastttc.so (built in-tree by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(path)
    st = ctypes.c_int
    L.ft_status_string.argtypes = [ctypes.c_int]
    L.ft_status_string.restype = ctypes.c_char_p
    L.ft_last_cuda_error.argtypes = []
    L.ft_last_cuda_error.restype = ctypes.c_char_p
    L.ft_version.restype = ctypes.c_int
    L.fastconv_out_dims.argtypes = [ctypes.c_int, _i64p, _i64p, _i64p]
    L.fastconv_out_dims.restype = st
    L.fastconv_nd.argtypes = [_vp, _i64p, ctypes.c_int, _vp, _i64p, _vp, _vp]
    L.fastconv_nd.restype = st
    L.fastconv_nd_typed.argtypes = [_vp, ctypes.c_int, _i64p, ctypes.c_int, _vp, _i64p, _vp, _vp, _vp]
    L.fastconv_nd_typed.restype = st
    L.fastconv_fft_plan_create.argtypes = [_i64p, ctypes.c_int, _i64p, ctypes.POINTER(_vp),
                                           ctypes.POINTER(ctypes.c_size_t)]
    L.fastconv_fft_plan_create.restype = st
    L.fastconv_fft_plan_destroy.argtypes = [_vp]
    L.fastconv_fft_plan_destroy.restype = None
    L.fastconv_fft_plan_workspace.argtypes = [_vp]
    L.fastconv_fft_plan_workspace.restype = ctypes.c_size_t
    L.fastconv_fft.argtypes = [_vp, _vp, _vp, _vp, _vp, ctypes.c_size_t, _vp]
    L.fastconv_fft.restype = st
    L.fastconv_prefers_fft.argtypes = [_i64p, ctypes.c_int, _i64p]
    L.fastconv_prefers_fft.restype = ctypes.c_int
    L.ft_test_stall_tma_waits.argtypes = [ctypes.c_int]
    L.ft_test_stall_tma_waits.restype = None
    L.fastconv_check.argtypes = [_vp]
    L.fastconv_check.restype = st
    L.fastconv_separable.argtypes = [_vp, _i64p, ctypes.c_int, ctypes.POINTER(_vp), _i64p, _vp, _vp, _vp]
    L.fastconv_separable.restype = st
    L.fastconv_factor.argtypes = [ctypes.POINTER(ctypes.c_float), _i64p, ctypes.c_int, ctypes.c_double,
                                  ctypes.POINTER(ctypes.c_float)]
    L.fastconv_factor.restype = ctypes.c_int
    L.ttc_derivatives.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                  _vp, _vp, _vp, _vp, _vp]
    L.ttc_derivatives.restype = st
    L.ttc_gradient.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64, _vp, _vp, _vp]
    L.ttc_gradient.restype = st
    L.ttc_gradient_batch.argtypes = [_vp, ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int64, _vp, _vp, _vp]
    L.ttc_gradient_batch.restype = st
    L.ttc_ctx_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.ttc_ctx_create.restype = st
    L.ttc_ctx_destroy.argtypes = [_vp]
    L.ttc_ctx_destroy.restype = None
    L.ttc_ctx_workspace_bytes.argtypes = [_vp]
    L.ttc_ctx_workspace_bytes.restype = ctypes.c_size_t
    L.ttc_solve.argtypes = [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                            ctypes.c_int, ctypes.c_int, _vp, _vp]
    L.ttc_solve.restype = st
    L.ttc_solve_noalloc.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                    ctypes.c_int, ctypes.c_int, _vp, _vp]
    L.ttc_solve_noalloc.restype = st
    L.ttc_solve_sequence.argtypes = [_vp, _vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _vp, _vp]
    L.ttc_solve_sequence.restype = st
    L.ttc_solve_sequence_host.argtypes = L.ttc_solve_sequence.argtypes
    L.ttc_solve_sequence_host.restype = st
    L.ttc_ctx_reserve_host.argtypes = [_vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int64, ctypes.c_int]
    L.ttc_ctx_reserve_host.restype = st
    L.ttc_partial_sums.argtypes = [_vp, _vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int, ctypes.c_int64, ctypes.c_int, _vp]
    L.ttc_partial_sums.restype = st
    L.ttc_reduce_solve.argtypes = [_vp, ctypes.c_int, _vp, _vp]
    L.ttc_reduce_solve.restype = st
    L.ttc_ctx_set_level0_events.argtypes = [_vp, _vp, _vp]
    L.ttc_ctx_set_level0_events.restype = st
    L.ttc_ctx_last_launch_count.argtypes = [_vp]
    L.ttc_ctx_last_launch_count.restype = ctypes.c_int
    L.ttc_batch_prepare.argtypes = [_vp, ctypes.POINTER(PairDesc), ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp]
    L.ttc_batch_prepare.restype = st
    L.ttc_batch_run.argtypes = [_vp, ctypes.c_int, _vp, _vp]
    L.ttc_batch_run.restype = st
    L.ttc_batch_autotune.argtypes = [_vp, ctypes.c_int, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _vp]
    L.ttc_batch_autotune.restype = st
    L.ttc_pyramid_layout.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _i64p, _i64p, _i64p]
    L.ttc_pyramid_layout.restype = st
    L.ttc_batch_set_plan.argtypes = [_vp, ctypes.POINTER(ctypes.c_int), ctypes.c_int]
    L.ttc_batch_set_plan.restype = st
    L.ttc_server_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int64, ctypes.POINTER(ctypes.c_int)]
    L.ttc_server_create.restype = st
    L.ttc_server_destroy.argtypes = [_vp]
    L.ttc_server_destroy.restype = None
    L.ttc_server_stream_bytes.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _i64p]
    L.ttc_server_stream_bytes.restype = st
    L.ttc_server_admit.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L.ttc_server_admit.restype = st
    L.ttc_server_remove.argtypes = [_vp, ctypes.c_int]
    L.ttc_server_remove.restype = st
    L.ttc_server_submit.argtypes = [_vp, ctypes.c_int, _vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_double]
    L.ttc_server_submit.restype = st
    L.ttc_server_step.argtypes = [_vp, ctypes.c_int, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L.ttc_server_step.restype = st
    L.ttc_server_drive.argtypes = [_vp, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.POINTER(_vp), _i64p,
                                   ctypes.c_int, ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double)]
    L.ttc_server_drive.restype = st
    L.ttc_server_in_flight.argtypes = [_vp]
    L.ttc_server_in_flight.restype = ctypes.c_int
    L.ttc_server_ticks.argtypes = [_vp]
    L.ttc_server_ticks.restype = ctypes.c_int64
    L.ttc_server_waiting.argtypes = [_vp, ctypes.c_int]
    L.ttc_server_waiting.restype = ctypes.c_int
    L.ttc_server_bytes_in_use.argtypes = [_vp]
    L.ttc_server_bytes_in_use.restype = ctypes.c_int64
    L.ttc_server_launches.argtypes = [_vp]
    L.ttc_server_launches.restype = ctypes.c_int
    L.ttc_select_level.argtypes = [_vp, ctypes.c_int, ctypes.c_int]
    L.ttc_select_level.restype = ctypes.c_int
    _lib = L
    return L


def lib():
    return load()


def _check(status: int, what: str):
    if status != 0:
        raise FtError(status, what)


def _stream_ptr(t: torch.Tensor) -> int:
    return torch.cuda.current_stream(t.device).cuda_stream


def _cuda_device(device=None) -> torch.device:
    """A CUDA device with its index (the current device when none is given)."""
    d = torch.device(device) if device is not None else torch.device("cuda")
    if d.type != "cuda":
        raise ValueError("a CUDA device is needed")
    return d if d.index is not None else torch.device("cuda", torch.cuda.current_device())


def _require_cuda(t: torch.Tensor, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")


def _dims(seq: Sequence[int]):
    arr = (ctypes.c_int64 * len(seq))(*[int(v) for v in seq])
    return arr


# --------------------------------------------------------------------------- #
# FastConv
# --------------------------------------------------------------------------- #

def fastconv_out_dims(dims: Sequence[int], kdims: Sequence[int]) -> tuple:
    """Full-convolution output extent (host call into the library)."""
    L = load()
    nd = len(dims)
    if len(kdims) != nd:
        raise ValueError("dims and kdims must have the same length")
    out = (ctypes.c_int64 * max(nd, 1))()
    _check(L.fastconv_out_dims(nd, _dims(dims), _dims(kdims), out), "fastconv_out_dims")
    return tuple(int(out[i]) for i in range(nd))


CONV_DTYPES = {torch.uint8: 0, torch.float32: 1, torch.int16: 2, torch.float16: 3, torch.bfloat16: 4}


def fastconv_nd(x: torch.Tensor, k: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Full n-D convolution of x with k (Eq. conv2 read as the full linear convolution).

    x: float32, uint8, int16, float16 or bfloat16 (widened to FP32 exactly); k and the
    output are float32."""
    L = load()
    _require_cuda(x, "x")
    _require_cuda(k, "k")
    if x.dtype not in CONV_DTYPES or k.dtype != torch.float32:
        raise ValueError("fastconv_nd takes a float32 kernel and a float32, uint8, int16, float16 or "
                         "bfloat16 input")
    if x.dim() != k.dim():
        raise ValueError("x and k must have the same rank")
    x = x.contiguous()
    k = k.contiguous()
    od = fastconv_out_dims(x.shape, k.shape)
    if out is None:
        out = torch.empty(od, dtype=torch.float32, device=x.device)
    elif tuple(out.shape) != od or not out.is_contiguous() or out.dtype != torch.float32:
        raise ValueError("out has the wrong shape, dtype or layout")
    if x.dtype == torch.float32:
        _check(L.fastconv_nd(x.data_ptr(), _dims(x.shape), x.dim(), k.data_ptr(), _dims(k.shape),
                             out.data_ptr(), _stream_ptr(x)), "fastconv_nd")
        return out
    args = (x.data_ptr(), CONV_DTYPES[x.dtype], _dims(x.shape), x.dim(), k.data_ptr(), _dims(k.shape),
            out.data_ptr())
    st = L.fastconv_nd_typed(*args, None, _stream_ptr(x))
    if st == 4:                         # this request converts the input first: give it room
        scratch = torch.empty(x.shape, dtype=torch.float32, device=x.device)
        st = L.fastconv_nd_typed(*args, scratch.data_ptr(), _stream_ptr(x))
        out._fastconv_scratch = scratch  # alive until the caller drops `out`
    _check(st, "fastconv_nd_typed")
    return out


class FftPlan:
    """cuFFT transforms for one (input shape, kernel shape) on one device
    (fastconv_fft_plan_create: the call that allocates); calls with it allocate nothing
    but the workspace the caller passes or that the plan keeps for the default stream."""

    def __init__(self, shape, kshape, device=None):
        L = load()
        self.device = _cuda_device(device)
        self.shape, self.kshape = tuple(int(v) for v in shape), tuple(int(v) for v in kshape)
        if len(self.shape) != len(self.kshape):
            raise ValueError("shape and kshape must have the same rank")
        h = _vp()
        nbytes = ctypes.c_size_t(0)
        with torch.cuda.device(self.device):
            _check(L.fastconv_fft_plan_create(_dims(self.shape), len(self.shape), _dims(self.kshape), ctypes.byref(h),
                                              ctypes.byref(nbytes)), "fastconv_fft_plan_create")
        self._h = h
        self.workspace_bytes = int(nbytes.value)

    def new_workspace(self) -> torch.Tensor:
        return torch.empty(self.workspace_bytes, dtype=torch.uint8, device=self.device)

    def __call__(self, x: torch.Tensor, k: torch.Tensor, out: Optional[torch.Tensor] = None,
                 workspace: Optional[torch.Tensor] = None) -> torch.Tensor:
        L = load()
        _require_cuda(x, "x")
        _require_cuda(k, "k")
        if x.dtype != torch.float32 or k.dtype != torch.float32:
            raise ValueError("float32 tensors")
        if tuple(x.shape) != self.shape or tuple(k.shape) != self.kshape or x.device != self.device:
            raise ValueError("x and k do not match the plan")
        x = x.contiguous()
        k = k.contiguous()
        od = tuple(n + m - 1 for n, m in zip(self.shape, self.kshape))
        out = torch.empty(od, dtype=torch.float32, device=x.device) if out is None else out
        if tuple(out.shape) != od or not out.is_contiguous() or out.dtype != torch.float32:
            raise ValueError("out has the wrong shape, dtype or layout")
        if workspace is None:
            workspace = self.new_workspace()
        with torch.cuda.device(self.device):
            _check(L.fastconv_fft(self._h, x.data_ptr(), k.data_ptr(), out.data_ptr(), workspace.data_ptr(),
                                  workspace.numel() * workspace.element_size(), _stream_ptr(x)), "fastconv_fft")
        out._fastconv_workspace = workspace        # alive until the caller drops `out`
        return out

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().fastconv_fft_plan_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_fft_plans = {}


def fastconv_fft(x: torch.Tensor, k: torch.Tensor, out: Optional[torch.Tensor] = None,
                 workspace: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Full convolution by FFT (ranks 1-3, float32), for large kernels.  Keeps one
    FftPlan per (device, shapes) in this module: the first call of a shape creates it."""
    _require_cuda(x, "x")
    _require_cuda(k, "k")
    if x.dtype != torch.float32 or k.dtype != torch.float32 or x.dim() != k.dim():
        raise ValueError("float32 tensors of one rank")
    key = (x.device, tuple(x.shape), tuple(k.shape))
    plan = _fft_plans.get(key)
    if plan is None:
        plan = _fft_plans[key] = FftPlan(x.shape, k.shape, x.device)
    if workspace is not None and workspace.numel() * workspace.element_size() < plan.workspace_bytes:
        workspace = None
    return plan(x, k, out=out, workspace=workspace)


def fastconv(x: torch.Tensor, k: torch.Tensor, method: str = "auto") -> torch.Tensor:
    """FastConv with the paper's switch: the direct path, or the FFT path for kernels at
    or above the measured crossover (method "auto"); "direct" or "fft" force one."""
    L = load()
    if method == "auto":
        use_fft = x.dtype == torch.float32 and bool(L.fastconv_prefers_fft(_dims(x.shape), x.dim(), _dims(k.shape)))
        method = "fft" if use_fft else "direct"
    if method == "fft":
        return fastconv_fft(x, k)
    if method == "direct":
        return fastconv_nd(x, k)
    raise ValueError("method is auto, direct or fft")


def fastconv_separable(x: torch.Tensor, factors, out: Optional[torch.Tensor] = None,
                       scratch: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Full convolution of x with the outer product of the 1-D factors (one per axis)."""
    L = load()
    _require_cuda(x, "x")
    if x.dtype != torch.float32 or len(factors) != x.dim():
        raise ValueError("float32 input and one factor per axis")
    fs = []
    for f in factors:
        _require_cuda(f, "factor")
        if f.dtype != torch.float32 or f.dim() != 1:
            raise ValueError("factors are 1-D float32 tensors")
        fs.append(f.contiguous())
    x = x.contiguous()
    kdims = [f.numel() for f in fs]
    od = fastconv_out_dims(x.shape, kdims)
    if out is None:
        out = torch.empty(od, dtype=torch.float32, device=x.device)
    if scratch is None and x.dim() >= 2:
        scratch = torch.empty(od, dtype=torch.float32, device=x.device)
    ptrs = (_vp * len(fs))(*[f.data_ptr() for f in fs])
    _check(L.fastconv_separable(x.data_ptr(), _dims(x.shape), x.dim(), ptrs, _dims(kdims), out.data_ptr(),
                                scratch.data_ptr() if scratch is not None else None, _stream_ptr(x)),
           "fastconv_separable")
    return out


def factor_kernel(k, rel_tol: float = 1e-6):
    """Host rank-1 test: the per-axis factors of a separable kernel, or None."""
    L = load()
    k = np.ascontiguousarray(np.asarray(k.cpu() if isinstance(k, torch.Tensor) else k, dtype=np.float32))
    kd = list(k.shape)
    f = np.empty(sum(kd), dtype=np.float32)
    r = L.fastconv_factor(k.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), _dims(kd), k.ndim, float(rel_tol),
                          f.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    if r < 0:
        raise ValueError("invalid kernel for fastconv_factor")
    if r == 0:
        return None
    return list(np.split(f, np.cumsum(kd)[:-1]))


def fastconv_check(device=None):
    """Synchronise the current stream; raise FtError if a FastConv wait gave up since the last check."""
    L = load()
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    _check(L.fastconv_check(torch.cuda.current_stream(dev).cuda_stream), "fastconv_check")


# --------------------------------------------------------------------------- #
# Time to contact
# --------------------------------------------------------------------------- #

def _frame_args(t: torch.Tensor):
    if t.dtype == torch.uint8:
        return DTYPE_U8, 1
    if t.dtype == torch.float32:
        return DTYPE_F32, 4
    raise ValueError("frames must be uint8 or float32")


def ttc_derivatives(prev: torch.Tensor, cur: torch.Tensor, with_G: bool = True):
    """Level-0 Ex, Ey, Et (and G), each (H-1, W-1) float32."""
    L = load()
    _require_cuda(prev, "prev")
    _require_cuda(cur, "cur")
    if prev.shape != cur.shape or prev.dtype != cur.dtype or prev.dim() != 2:
        raise ValueError("prev and cur must be 2-D tensors of one shape and dtype")
    if prev.stride(1) != 1 or cur.stride(1) != 1 or prev.stride(0) != cur.stride(0):
        raise ValueError("rows must be contiguous with one common pitch")
    dt, es = _frame_args(prev)
    H, W = prev.shape
    outs = [torch.empty((max(H - 1, 0), max(W - 1, 0)), dtype=torch.float32, device=prev.device)
            for _ in range(4 if with_G else 3)]
    G = outs[3].data_ptr() if with_G else None
    _check(L.ttc_derivatives(prev.data_ptr(), cur.data_ptr(), dt, H, W, prev.stride(0) * es,
                             outs[0].data_ptr(), outs[1].data_ptr(), outs[2].data_ptr(), G,
                             _stream_ptr(prev)), "ttc_derivatives")
    return tuple(outs)


def gradient(image: torch.Tensor, with_mag: bool = True, with_dir: bool = True):
    """Gradient magnitude and direction (Sec. II, Eq. Emag, Eq. Eangle) of one image (2-D)
    or of a batch of images (3-D, one launch): float32 tensors of shape (..., H-1, W-1)
    (None for an output not asked for)."""
    L = load()
    _require_cuda(image, "image")
    if image.dim() not in (2, 3) or image.stride(-1) != 1:
        raise ValueError("image must be 2-D (or a 3-D batch) with contiguous rows")
    if not (with_mag or with_dir):
        raise ValueError("ask for at least one output")
    dt, es = _frame_args(image)
    H, W = image.shape[-2:]
    n = image.shape[0] if image.dim() == 3 else 1
    shape = (n, H - 1, W - 1) if image.dim() == 3 else (H - 1, W - 1)
    mag = torch.empty(shape, dtype=torch.float32, device=image.device) if with_mag else None
    ang = torch.empty(shape, dtype=torch.float32, device=image.device) if with_dir else None
    if n == 0:
        return mag, ang
    stride = image.stride(0) * es if image.dim() == 3 else 0
    _check(L.ttc_gradient_batch(image.data_ptr(), n, stride, dt, H, W, image.stride(-2) * es,
                                mag.data_ptr() if mag is not None else None,
                                ang.data_ptr() if ang is not None else None, _stream_ptr(image)),
           "ttc_gradient_batch")
    return mag, ang


def results_to_numpy(t: torch.Tensor) -> np.ndarray:
    """Device/host byte tensor of ttc_level_result records -> numpy structured array."""
    a = t.detach().to("cpu").contiguous().numpy()
    return a.view(RESULT_DTYPE).reshape(-1)


def pyramid_layout(H: int, W: int, levels: int, dtype=torch.uint8) -> dict:
    """Layout of one frame's pyramid block (levels 1 .. levels-1): offsets, pitches, bytes."""
    L = load()
    dt = DTYPE_U8 if dtype == torch.uint8 else DTYPE_F32 if dtype == torch.float32 else None
    if dt is None:
        raise ValueError("frames are uint8 or float32")
    n = max(int(levels), 1)
    off = (ctypes.c_int64 * n)()
    pit = (ctypes.c_int64 * n)()
    nbytes = ctypes.c_int64(0)
    _check(L.ttc_pyramid_layout(int(H), int(W), int(levels), dt, off, pit, ctypes.byref(nbytes)),
           "ttc_pyramid_layout")
    return {"offsets": list(off), "pitches": list(pit), "bytes": int(nbytes.value)}


def select_level(results: np.ndarray, rule: int = 0) -> int:
    """Multi-scale selection (Sec. V-B) over one pair's per-level results (host)."""
    L = load()
    r = np.ascontiguousarray(results, dtype=RESULT_DTYPE)
    v = L.ttc_select_level(r.ctypes.data, r.shape[0], int(rule))
    if v == -2:
        raise ValueError("invalid arguments to ttc_select_level")
    return int(v)


def ttc_solve_noalloc(prev: torch.Tensor, cur: torch.Tensor, levels: int = 1, mode: int = MODE_FOE,
                      out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """One frame pair through ttc_solve_noalloc (library allocates no device memory).

    For callers that cannot allocate device memory once running; the library's fixed
    scratch array is shared by all calls, so calls must not overlap on the GPU.
    """
    L = load()
    _require_cuda(prev, "prev")
    _require_cuda(cur, "cur")
    if prev.shape != cur.shape or prev.dtype != cur.dtype or prev.dim() != 2:
        raise ValueError("prev and cur must be 2-D tensors of one shape and dtype")
    if prev.stride(1) != 1 or cur.stride(1) != 1 or prev.stride(0) != cur.stride(0):
        raise ValueError("rows must be contiguous with one common pitch")
    dt, es = _frame_args(prev)
    H, W = prev.shape
    if out is None:
        out = torch.empty(levels * RESULT_DTYPE.itemsize, dtype=torch.uint8, device=prev.device)
    if cur.device != prev.device or not out.is_cuda or out.device != prev.device:
        raise ValueError("prev, cur and out must be on one CUDA device")
    # the library uses the scratch array of the current device: make it prev's
    with torch.cuda.device(prev.device):
        _check(L.ttc_solve_noalloc(prev.data_ptr(), cur.data_ptr(), dt, H, W, prev.stride(0) * es, int(levels),
                                   int(mode), out.data_ptr(), _stream_ptr(prev)), "ttc_solve_noalloc")
    return out


class TtcContext:
    """Owns the library's partial-sum workspace (ttc_ctx) for requests up to a size."""

    def __init__(self, max_H: int, max_W: int, max_levels: int = 5, max_pairs: int = 1,
                 device: Optional[torch.device] = None):
        L = load()
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.max = (max_H, max_W, max_levels, max_pairs)
        h = _vp()
        with torch.cuda.device(self.device):
            _check(L.ttc_ctx_create(ctypes.byref(h), max_H, max_W, max_levels, max_pairs), "ttc_ctx_create")
        self._h = h
        self._staging = None

    @property
    def workspace_bytes(self) -> int:
        return int(load().ttc_ctx_workspace_bytes(self._h))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().ttc_ctx_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_level0_events(self, start: Optional[torch.cuda.Event], end: Optional[torch.cuda.Event]):
        """Record `start`/`end` around the level-0 pass of later calls (None, None: off)."""
        L = load()
        sp = start.cuda_event if start is not None else None
        ep = end.cuda_event if end is not None else None
        _check(L.ttc_ctx_set_level0_events(self._h, sp, ep), "ttc_ctx_set_level0_events")

    @property
    def last_launch_count(self) -> int:
        """Kernels launched by the last solve, sequence or partial-sums call (a
        ttc_reduce_solve after ttc_partial_sums adds one)."""
        return int(load().ttc_ctx_last_launch_count(self._h))

    def new_results(self, n: int) -> torch.Tensor:
        return torch.empty(n * RESULT_DTYPE.itemsize, dtype=torch.uint8, device=self.device)

    def solve(self, prev: torch.Tensor, cur: torch.Tensor, levels: int = 1, mode: int = MODE_FOE,
              out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """One frame pair -> byte tensor of `levels` ttc_level_result records (device)."""
        L = load()
        _require_cuda(prev, "prev")
        _require_cuda(cur, "cur")
        if prev.shape != cur.shape or prev.dtype != cur.dtype or prev.dim() != 2:
            raise ValueError("prev and cur must be 2-D tensors of one shape and dtype")
        if prev.stride(1) != 1 or cur.stride(1) != 1 or prev.stride(0) != cur.stride(0):
            raise ValueError("rows must be contiguous with one common pitch")
        dt, es = _frame_args(prev)
        H, W = prev.shape
        out = self.new_results(levels) if out is None else out
        _check(L.ttc_solve(self._h, prev.data_ptr(), cur.data_ptr(), dt, H, W, prev.stride(0) * es,
                           int(levels), int(mode), out.data_ptr(), _stream_ptr(prev)), "ttc_solve")
        return out

    def _seq_args(self, frames: torch.Tensor):
        if frames.dim() != 3 or frames.stride(2) != 1:
            raise ValueError("frames must be (T, H, W) with contiguous rows")
        dt, es = _frame_args(frames)
        T, H, W = frames.shape
        return dt, es, T, H, W

    def solve_sequence(self, frames: torch.Tensor, levels: int = 1, mode: int = MODE_FOE,
                       out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """T frames -> (T-1) * levels records.

        With CUDA frames the records stay on the device (asynchronous).  With host
        frames (ideally pinned) the library uploads them in chunks that overlap the
        compute and returns the records in a host tensor (ttc_solve_sequence_host), on
        the current stream; keep `frames` alive until the stream is synchronised.
        """
        L = load()
        dt, es, T, H, W = self._seq_args(frames)
        n = (T - 1) * levels
        if not frames.is_cuda:
            if out is None:
                out = torch.empty(n * RESULT_DTYPE.itemsize, dtype=torch.uint8, pin_memory=True)
            elif out.is_cuda or out.numel() * out.element_size() < n * RESULT_DTYPE.itemsize:
                raise ValueError("out must be a host tensor of (T-1) * levels records")
            stream = torch.cuda.current_stream(self.device).cuda_stream
            self.reserve_host(frames, levels)
            _check(L.ttc_solve_sequence_host(self._h, frames.data_ptr(), frames.stride(0) * es, T, dt, H, W,
                                             frames.stride(1) * es, int(levels), int(mode), out.data_ptr(), stream),
                   "ttc_solve_sequence_host")
            self._host_frames = frames          # referenced until the next call
            return out
        out = self.new_results(n) if out is None else out
        _check(L.ttc_solve_sequence(self._h, frames.data_ptr(), frames.stride(0) * es, T, dt, H, W,
                                    frames.stride(1) * es, int(levels), int(mode), out.data_ptr(),
                                    _stream_ptr(frames)), "ttc_solve_sequence")
        return out

    def reserve_host(self, frames: torch.Tensor, levels: int = 1):
        """Size the context's host-sequence buffers for `frames` (T, H, W) on the host
        (ttc_ctx_reserve_host: allocates only when they must grow)."""
        L = load()
        dt, es, T, H, W = self._seq_args(frames)
        with torch.cuda.device(self.device):
            _check(L.ttc_ctx_reserve_host(self._h, frames.stride(0) * es, T, dt, H, W, frames.stride(1) * es,
                                          int(levels)), "ttc_ctx_reserve_host")

    @staticmethod
    def host_upload_bytes(T: int, frame_bytes: int, max_pairs: int) -> int:
        """Bytes ttc_solve_sequence_host copies to the device for T frames."""
        chunk = min(64, max_pairs, T - 1)
        nchunks = -(-(T - 1) // chunk)
        return (T - 1 + nchunks) * frame_bytes

    def batch_prepare(self, pairs, levels: int = 1):
        """Prepare a batch of independent pairs of any sizes.

        Each entry is (prev, cur) or (prev, cur, prev_pyramid, cur_pyramid): 2-D frame
        tensors, and optional uint8 device blocks of ``pyramid_layout(...)['bytes']``
        bytes (None: that frame's pyramid stays in the context workspace).  The tensors
        must stay alive and in place while the batch is run.
        """
        L = load()
        if len(pairs) == 0:
            raise ValueError("empty batch")
        descs = (PairDesc * len(pairs))()
        dt0 = None
        for i, entry in enumerate(pairs):
            a, b = entry[0], entry[1]
            pa, pb = (entry[2], entry[3]) if len(entry) > 2 else (None, None)
            for blk, what in ((pa, "prev_pyramid"), (pb, "cur_pyramid")):
                if blk is not None:
                    _require_cuda(blk, what)
            _require_cuda(a, "prev")
            _require_cuda(b, "cur")
            if a.shape != b.shape or a.dtype != b.dtype or a.dim() != 2:
                raise ValueError("each pair: 2-D tensors of one shape and dtype")
            if a.stride(1) != 1 or b.stride(1) != 1 or a.stride(0) != b.stride(0):
                raise ValueError("rows must be contiguous with one common pitch")
            dt, es = _frame_args(a)
            if dt0 is None:
                dt0 = dt
            elif dt != dt0:
                raise ValueError("all pairs of a batch have one dtype")
            descs[i] = PairDesc(a.data_ptr(), b.data_ptr(), a.shape[0], a.shape[1], a.stride(0) * es,
                                pa.data_ptr() if pa is not None else None, pb.data_ptr() if pb is not None else None)
        self._batch = (len(pairs), levels, pairs)          # keeps the frames referenced
        _check(L.ttc_batch_prepare(self._h, descs, len(pairs), dt0, int(levels), _stream_ptr(pairs[0][0])),
               "ttc_batch_prepare")

    def batch_run(self, mode: int = MODE_FOE, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Run the prepared batch: npairs * levels records, out[p * levels + l] (device)."""
        L = load()
        n, levels, _ = self._batch
        out = self.new_results(n * levels) if out is None else out
        _check(L.ttc_batch_run(self._h, int(mode), out.data_ptr(), _stream_ptr(out)), "ttc_batch_run")
        return out

    def batch_autotune(self, mode: int = MODE_FOE, reps: int = 3, out: Optional[torch.Tensor] = None) -> list:
        """Pick 64- or 16-row tiles per level by timing the prepared batch; returns rows per level."""
        L = load()
        n, levels, _ = self._batch
        out = self.new_results(n * levels) if out is None else out
        rows = (ctypes.c_int * levels)()
        _check(L.ttc_batch_autotune(self._h, int(mode), out.data_ptr(), int(reps), rows, _stream_ptr(out)),
               "ttc_batch_autotune")
        return [int(rows[i]) for i in range(levels)]

    def batch_set_plan(self, rows_per_tile=None, levels: Optional[int] = None):
        """Fix the tile height (16 or 64 rows) per level for later prepares; None: automatic."""
        L = load()
        if rows_per_tile is None:
            _check(L.ttc_batch_set_plan(self._h, None, int(levels or 1)), "ttc_batch_set_plan")
            return
        arr = (ctypes.c_int * len(rows_per_tile))(*[int(r) for r in rows_per_tile])
        _check(L.ttc_batch_set_plan(self._h, arr, len(rows_per_tile)), "ttc_batch_set_plan")

    def partial_sums(self, frames: torch.Tensor, levels: int = 1):
        """Stage 1 only (fused pyramid/stencil/products/tile reduction)."""
        L = load()
        _require_cuda(frames, "frames")
        dt, es, T, H, W = self._seq_args(frames)
        _check(L.ttc_partial_sums(self._h, frames.data_ptr(), frames.stride(0) * es, T, dt, H, W,
                                  frames.stride(1) * es, int(levels), _stream_ptr(frames)), "ttc_partial_sums")

    def reduce_solve(self, out: torch.Tensor, mode: int = MODE_FOE):
        """Stage 2 only (FP64 merge + solve) for the last partial_sums call."""
        L = load()
        _check(L.ttc_reduce_solve(self._h, int(mode), out.data_ptr(), _stream_ptr(out)), "ttc_reduce_solve")
        return out
