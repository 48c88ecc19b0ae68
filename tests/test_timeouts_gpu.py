"""Bounded waits of the copy-engine-fed kernels, exercised without any fault: the test
switch makes every barrier expect 16 bytes more than its copies deliver, so each wait
gives up after about 2 s of GPU clock; the kernels report it through their status words
and return, and the same context and library work normally afterwards."""
import numpy as np
import pytest
import torch

import oracle
import paper_1612_08825_gb300 as ft
import scenes

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")


def _stalled(fn):
    L = ft.load()
    L.ft_test_stall_tma_waits(1)
    try:
        return fn()
    finally:
        torch.cuda.synchronize()
        L.ft_test_stall_tma_waits(0)


def test_ttc_level0_timeout_is_flagged_and_the_context_recovers():
    # nine 1080p pairs: enough tiles for 64-row level-0 tiles, hence the TMA-fed pass
    sc = scenes.tilted_plane_scene(H=1080, W=1920, seed=41)
    fr = scenes.render_sequence(sc, 10, device=DEV)
    ctx = ft.TtcContext(1080, 1920, 2, 9)
    ref = ft.results_to_numpy(ctx.solve_sequence(fr, levels=2, mode=1))
    assert not np.any(ref["flags"] & ft.FLAG_TIMEOUT)
    bad = _stalled(lambda: ft.results_to_numpy(ctx.solve_sequence(fr, levels=2, mode=1)))
    assert np.all(bad["flags"] & ft.FLAG_TIMEOUT)
    again = ft.results_to_numpy(ctx.solve_sequence(fr, levels=2, mode=1))
    assert again.tobytes() == ref.tobytes()
    ctx.close()


def test_fastconv_timeout_is_reported_and_the_next_call_is_correct():
    E = scenes.uniform_array((8, 256, 512), seed=3)
    k = scenes.normal_array((1, 7, 7), seed=4)
    x, kk = torch.from_numpy(E).to(DEV), torch.from_numpy(k).to(DEV)
    ft.fastconv_check()                                   # clear any earlier state
    with pytest.raises(ft.FtError) as err:
        _stalled(lambda: (ft.fastconv_nd(x, kk), ft.fastconv_check()))
    assert err.value.status == ft.ERR_TIMEOUT
    ft.fastconv_check()                                   # the word was cleared by the report
    got = ft.fastconv_nd(x, kk)
    ft.fastconv_check()
    pts = np.random.default_rng(1).integers(0, got.numel(), 500).astype(np.int64)
    ref, rabs = oracle.fastconv_points(E, k, pts)
    g = got.cpu().numpy().reshape(-1)[pts].astype(np.float64)
    assert np.all(np.abs(g - ref) <= 1e-5 * rabs + 1e-30)
