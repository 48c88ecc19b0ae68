"""Batches of independent frame pairs of different sizes (work-list launches) vs the
FP64 oracle, the single-pair entry point, and themselves (alone vs in the mix, graph
replay)."""
import numpy as np
import pytest
import torch

import oracle
import paper_1612_08825_gb300 as ft
import scenes
from _tol import check_record

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")
LEVELS = 3


def _make_pairs(sizes, seed0=100, unaligned_every=0):
    pairs, host = [], []
    for i, (H, W) in enumerate(sizes):
        sc = scenes.tilted_plane_scene(H=H, W=W, seed=seed0 + i, m=16, pmin=3.0, pmax=40.0)
        a = scenes.render(sc, 1.0)
        b = scenes.render(sc, 2.0)
        host.append((a.numpy(), b.numpy()))
        if unaligned_every and i % unaligned_every == 0:
            buf = torch.zeros((2, H, W + 3), dtype=torch.uint8, device=DEV)     # odd pitch
            buf[0, :, :W] = a.to(DEV)
            buf[1, :, :W] = b.to(DEV)
            pairs.append((buf[0, :, :W], buf[1, :, :W]))
        else:
            pairs.append((a.to(DEV), b.to(DEV)))
    return pairs, host


SIZES = [(120, 160), (135, 241), (300, 517), (64, 64), (271, 399), (33, 700), (480, 640), (17, 19), (250, 260)]


def test_batch_matches_oracle_and_single_pairs():
    pairs, host = _make_pairs(SIZES, unaligned_every=4)
    ctx = ft.TtcContext(480, 700, LEVELS, len(pairs))
    ctx.batch_prepare(pairs, levels=LEVELS)
    got = ft.results_to_numpy(ctx.batch_run(mode=1)).reshape(len(pairs), LEVELS)
    single = ft.TtcContext(480, 700, LEVELS, 1)
    for i, (a, b) in enumerate(host):
        ref = oracle.ttc_pair(a, b, levels=LEVELS, mode=1)
        one = ft.results_to_numpy(single.solve(pairs[i][0], pairs[i][1], levels=LEVELS, mode=1))
        for l in range(LEVELS):
            check_record(got[i, l], ref[l], 1, l)
            check_record(one[l], ref[l], 1, l)
    ctx.close()
    single.close()


def test_batch_result_same_alone_and_in_the_mix():
    pairs, _ = _make_pairs(SIZES, seed0=300)
    ctx = ft.TtcContext(480, 700, LEVELS, len(pairs))
    ctx.batch_prepare(pairs, levels=LEVELS)
    rows = ctx.batch_autotune(mode=1, reps=1)          # fixes the tile plan on this context
    assert all(r in (16, 64) for r in rows)
    mix = ft.results_to_numpy(ctx.batch_run(mode=1)).reshape(len(pairs), LEVELS)
    for i in (0, 2, 7):
        ctx.batch_prepare([pairs[i]], levels=LEVELS)
        alone = ft.results_to_numpy(ctx.batch_run(mode=1))
        assert alone.tobytes() == mix[i].tobytes()      # same plan: bitwise
    # a different plan (fresh context, automatic choice): within tolerance
    other = ft.TtcContext(480, 700, LEVELS, 1)
    for i in (1, 4):
        other.batch_prepare([pairs[i]], levels=LEVELS)
        r = ft.results_to_numpy(other.batch_run(mode=1))
        for l in range(LEVELS):
            assert np.allclose(r[l]["sums"], mix[i, l]["sums"], rtol=1e-5, atol=0)
    ctx.close()
    other.close()


def test_batch_graph_replay():
    pairs, _ = _make_pairs(SIZES[:5], seed0=500)
    ctx = ft.TtcContext(480, 700, LEVELS, len(pairs))
    ctx.batch_prepare(pairs, levels=LEVELS)
    out = ctx.new_results(len(pairs) * LEVELS)
    ref = ctx.batch_run(mode=1).clone()
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        ctx.batch_run(mode=1, out=out)                  # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ctx.batch_run(mode=1, out=out)
    out.zero_()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert out.cpu().numpy().tobytes() == ref.cpu().numpy().tobytes()
    ctx.close()


def _uneven_full_scale(n, seed):
    """n pairs drawn like the 512-pair uneven workload (W 160-1920, H 120-1080, per-pair
    depth and speed), with the first two forced to 1920 x 1080 and 160 x 120."""
    specs = scenes.uneven_pair_sizes(n, seed=seed)
    specs[0] = (1080, 1920) + specs[0][2:]
    specs[1] = (120, 160) + specs[1][2:]
    pairs, host = [], []
    for i, (h, w, z0, sp) in enumerate(specs):
        sc = scenes.tilted_plane_scene(H=h, W=w, seed=seed + 1000 + i, Z0=z0, speed=sp)
        fr = scenes.render_sequence(sc, 2, device=DEV)
        pairs.append((fr[0], fr[1]))
        host.append((fr[0].cpu().numpy(), fr[1].cpu().numpy()))
    return pairs, host


@pytest.mark.parametrize("plan", ["autotuned", "forced"])
def test_batch_full_scale_uneven_pairs_vs_oracle(plan):
    """24 pairs of the uneven workload at full scale (up to 1920 x 1080), 5 levels, FOE:
    every record against the FP64 oracle, under the autotuned tile plan and under the
    plan 64, 64, 64, 64, 16 rows per level."""
    levels = 5
    pairs, host = _uneven_full_scale(24, seed=4242)
    ctx = ft.TtcContext(1080, 1920, levels, len(pairs))
    if plan == "forced":
        ctx.batch_set_plan([64, 64, 64, 64, 16])
    ctx.batch_prepare(pairs, levels=levels)
    out = ctx.new_results(len(pairs) * levels)
    if plan == "autotuned":
        rows = ctx.batch_autotune(mode=1, reps=1, out=out)
        assert all(r in (16, 64) for r in rows)
    got = ft.results_to_numpy(ctx.batch_run(mode=1, out=out)).reshape(len(pairs), levels)
    for i, (a, b) in enumerate(host):
        ref = oracle.ttc_pair(a, b, levels=levels, mode=1)
        for l in range(levels):
            check_record(got[i, l], ref[l], 1, l)
    ctx.close()


def test_batch_errors():
    ctx = ft.TtcContext(100, 100, 2, 2)
    a = torch.zeros((100, 100), dtype=torch.uint8, device=DEV)
    big = torch.zeros((200, 100), dtype=torch.uint8, device=DEV)
    with pytest.raises(ft.FtError):
        ctx.batch_prepare([(big, big)], levels=2)              # larger than the context
    with pytest.raises(ft.FtError):
        ctx.batch_prepare([(a, a)] * 3, levels=2)              # more pairs than the context
    tiny = torch.zeros((3, 3), dtype=torch.uint8, device=DEV)
    with pytest.raises(ft.FtError):
        ctx.batch_prepare([(tiny, tiny)], levels=2)            # level 1 would be 1 x 1
    ctx.close()
