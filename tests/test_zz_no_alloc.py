"""ttc_solve_noalloc against ttc_solve and the FP64 oracle, through the C ABI.

ttc_solve_noalloc serves callers that must not allocate device memory once they are
running (hard real-time loops, safety-certified software, plug-ins inside a process
that owns all device memory): its scratch is a fixed array inside the library.  Its
results must equal those of ttc_solve with a context, on consecutive calls that reuse
the same scratch.  This file is collected last so that a failure here comes after
every other test has run.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_1612_08825_gb300 as ft
import scenes
from _tol import SUM_REL, SUM_REL_F32, check_record

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")
REL = 1e-5      # the relative tolerance of the parity tests


def _close(got, ref):
    assert int(got["flags"]) == int(ref["flags"]) and int(got["n"]) == int(ref["n"])
    assert np.all(np.abs(got["sums"] - ref["sums"]) <= REL * np.abs(ref["sums"]) + 1e-300)
    for k in ("A", "B", "C", "ttc", "x0", "y0", "resid"):
        g, r = float(got[k]), float(ref[k])
        if np.isnan(r):
            assert np.isnan(g)
        else:
            assert abs(g - r) <= REL * abs(r) + 1e-12, (k, g, r)


@pytest.mark.parametrize("mode", [ft.MODE_TTC, ft.MODE_FOE])
@pytest.mark.parametrize("H,W,levels,quantize", [(1080, 1920, 5, True), (150, 333, 4, True), (128, 128, 3, False)])
def test_noalloc_matches_context_solve_and_oracle_on_two_calls(H, W, levels, quantize, mode):
    L = ft.load()
    sc = scenes.tilted_plane_scene(H=H, W=W, seed=H + W, quantize=quantize)
    fr = scenes.render_sequence(sc, 3, device=DEV)
    host = fr.cpu().numpy().astype(np.float64)
    dt, es = (0, 1) if quantize else (1, 4)
    rel = SUM_REL if quantize else SUM_REL_F32
    ctx = ft.TtcContext(H, W, levels, 1)
    stream = torch.cuda.current_stream().cuda_stream
    for t in range(2):                                   # two calls in a row, different pairs
        a, b = fr[t], fr[t + 1]
        ref = ft.results_to_numpy(ctx.solve(a, b, levels=levels, mode=mode))
        out = torch.empty(levels * ft.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=DEV)
        st = L.ttc_solve_noalloc(a.data_ptr(), b.data_ptr(), dt, H, W, a.stride(0) * es, levels,
                                 mode, out.data_ptr(), stream)
        assert st == 0, L.ft_status_string(st)
        got = ft.results_to_numpy(out)
        orc = oracle.ttc_pair(host[t], host[t + 1], levels=levels, mode=mode)
        for l in range(levels):
            _close(got[l], ref[l])
            check_record(got[l], orc[l], mode, l, rel=rel)
    ctx.close()


def test_noalloc_rejects_requests_beyond_its_scratch():
    L = ft.load()
    big = torch.zeros((2048, 4096), dtype=torch.uint8, device=DEV)
    out = torch.empty(5 * ft.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=DEV)
    st = L.ttc_solve_noalloc(big.data_ptr(), big.data_ptr(), 0, 2048, 4096, 4096, 5, 1, out.data_ptr(),
                             torch.cuda.current_stream().cuda_stream)
    assert st == 4          # FT_ERR_WORKSPACE
