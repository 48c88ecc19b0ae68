"""The checked build of the TTC passes (FASTTTC_CHECK=1 at build time, FT_CHECK in the
sources): every frame read and every pyramid store is compared with the extent its call
gave, and one outside it is skipped and reported as FT_FLAG_BOUNDS in the records.  On
valid inputs nothing is reported and the records are bitwise those of the release build,
on every pass: the copy-engine level 0, the load-based levels (padded context images,
caller pyramid blocks, float frames) and unaligned frames."""
import ctypes

import numpy as np
import pytest
import torch

import paper_1612_08825_gb300 as ft
import scenes
from paper_1612_08825_gb300 import build as ftbuild

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")
_vp = ctypes.c_void_p


@pytest.fixture(scope="module")
def checked():
    C = ctypes.CDLL(ftbuild.build_checked_ttc())
    C.ttc_ctx_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    C.ttc_ctx_destroy.argtypes = [_vp]
    C.ttc_solve_sequence.argtypes = [_vp, _vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _vp, _vp]
    C.ttc_batch_prepare.argtypes = [_vp, ctypes.POINTER(ft.PairDesc), ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp]
    C.ttc_batch_run.argtypes = [_vp, ctypes.c_int, _vp, _vp]
    C.ttc_pyramid_layout.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp,
                                     ctypes.POINTER(ctypes.c_int64)]
    return C


def _ctx(C, H, W, levels, pairs):
    h = _vp()
    assert C.ttc_ctx_create(ctypes.byref(h), H, W, levels, pairs) == 0
    return h


def _no_bounds(rec):
    assert np.all((rec["flags"] & ft.FLAG_BOUNDS) == 0)


@pytest.mark.parametrize("H,W,T,dtype,pad", [
    (270, 481, 6, torch.uint8, 0),        # copy-engine level 0 (pitch 496), padded level images
    (133, 259, 5, torch.uint8, 3),        # unaligned pitch: load-based level 0 with checked loads
    (128, 200, 4, torch.float32, 0),      # float frames
])
def test_checked_sequence_equals_release(checked, H, W, T, dtype, pad):
    sc = scenes.tilted_plane_scene(H=H, W=W, seed=H + W, m=16, quantize=dtype == torch.uint8)
    fr = scenes.render_sequence(sc, T, device=DEV)
    pitch = -(-(W + pad) // 16) * 16 if pad == 0 else W + pad
    buf = torch.zeros((T, H, pitch), dtype=dtype, device=DEV)
    buf[:, :, :W] = fr
    frames = buf[:, :, :W]
    levels = 4
    ref = ft.TtcContext(H, W, levels, T - 1)
    want = ft.results_to_numpy(ref.solve_sequence(frames, levels=levels, mode=1))
    es = frames.element_size()
    h = _ctx(checked, H, W, levels, T - 1)
    out = torch.empty((T - 1) * levels * ft.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=DEV)
    st = checked.ttc_solve_sequence(h, frames.data_ptr(), frames.stride(0) * es, T, 0 if dtype == torch.uint8 else 1,
                                    H, W, frames.stride(1) * es, levels, 1, out.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
    assert st == 0
    got = ft.results_to_numpy(out)
    _no_bounds(got)
    assert got.tobytes() == want.tobytes()
    checked.ttc_ctx_destroy(h)
    ref.close()


def test_checked_batch_with_caller_pyramids_equals_release(checked):
    sizes = [(120, 160), (243, 337), (480, 640), (67, 301)]
    levels = 4
    pairs, descs = [], (ft.PairDesc * len(sizes))()
    for i, (H, W) in enumerate(sizes):
        sc = scenes.tilted_plane_scene(H=H, W=W, seed=40 + i, m=16)
        fr = scenes.render_sequence(sc, 2, device=DEV)
        lay = ft.pyramid_layout(H, W, levels)
        blocks = [torch.zeros(lay["bytes"], dtype=torch.uint8, device=DEV) for _ in range(2)]
        pairs.append((fr[0], fr[1], blocks[0], blocks[1]))
        descs[i] = ft.PairDesc(fr[0].data_ptr(), fr[1].data_ptr(), H, W, W, blocks[0].data_ptr(), blocks[1].data_ptr())
    ref = ft.TtcContext(480, 640, levels, len(sizes))
    ref.batch_prepare(pairs, levels=levels)
    want = ft.results_to_numpy(ref.batch_run(mode=1))
    h = _ctx(checked, 480, 640, levels, len(sizes))
    s = torch.cuda.current_stream().cuda_stream
    assert checked.ttc_batch_prepare(h, descs, len(sizes), 0, levels, s) == 0
    out = torch.empty(len(sizes) * levels * ft.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=DEV)
    assert checked.ttc_batch_run(h, 1, out.data_ptr(), s) == 0
    got = ft.results_to_numpy(out)
    _no_bounds(got)
    assert got.tobytes() == want.tobytes()
    checked.ttc_ctx_destroy(h)
    ref.close()
