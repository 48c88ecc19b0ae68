"""Time-to-contact / FOE pipeline through the C ABI vs the FP64 oracle.

Bars: uint8 derivatives bitwise; sums within 1e-5 of the oracle's sum of |terms|;
flags identical; A, B, C, TTC and FOE within the bounds that the sum tolerance
implies through the solve (tests/_tol.py).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1612_08825_gb300 as ft
import scenes
from _tol import SUM_REL_F32, check_record

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")


def _pair(sc, t=0.0):
    a = scenes.render(sc, t)
    b = scenes.render(sc, t + 1.0)
    return a, b


# --------------------------------------------------------------------------- #
# derivatives (debug surface)
# --------------------------------------------------------------------------- #

@pytest.mark.parametrize("H,W", [(2, 2), (5, 7), (67, 133), (130, 300)])
def test_derivatives_uint8_bitwise(H, W):
    sc = scenes.tilted_plane_scene(H=H, W=W, seed=H + W, m=16, pmin=3.0, pmax=20.0)
    a, b = _pair(sc)
    Ex, Ey, Et, G = ft.ttc_derivatives(a.to(DEV), b.to(DEV))
    torch.cuda.synchronize()
    rx, ry, rt = oracle.derivatives(a.numpy(), b.numpy())
    np.testing.assert_array_equal(Ex.cpu().numpy().astype(np.float64), rx)
    np.testing.assert_array_equal(Ey.cpu().numpy().astype(np.float64), ry)
    np.testing.assert_array_equal(Et.cpu().numpy().astype(np.float64), rt)
    # G = x Ex + y Ey, FP32: within 2 ulp-scale of |x Ex| + |y Ey|
    yy, xx = np.meshgrid(np.arange(H - 1) + 0.5 - (H - 1) / 2, np.arange(W - 1) + 0.5 - (W - 1) / 2,
                         indexing="ij")
    gref = xx * rx + yy * ry
    bound = 2.0 ** -22 * (np.abs(xx * rx) + np.abs(yy * ry))
    assert np.all(np.abs(G.cpu().numpy() - gref) <= bound + 1e-30)


def test_derivatives_float32_and_pitch():
    sc = scenes.fronto_parallel_scene(H=37, W=51, seed=2)
    a, b = _pair(sc, 3.0)
    # frames inside wider buffers: pitch != width
    buf = torch.zeros((2, 37, 60), dtype=torch.float32, device=DEV)
    buf[0, :, :51] = a.to(DEV)
    buf[1, :, :51] = b.to(DEV)
    Ex, Ey, Et = ft.ttc_derivatives(buf[0, :, :51], buf[1, :, :51], with_G=False)
    torch.cuda.synchronize()
    rx, ry, rt = oracle.derivatives(a.double().numpy(), b.double().numpy())
    for got, ref in ((Ex, rx), (Ey, ry), (Et, rt)):
        assert np.all(np.abs(got.cpu().numpy() - ref) <= 4 * 2.0 ** -24 * 2.0)


# --------------------------------------------------------------------------- #
# the fused multi-level solve
# --------------------------------------------------------------------------- #

CASES = [
    # H, W, levels, seed: several tiles (64 x 128 cubes), ragged tails, odd sizes
    (96, 160, 3, 1), (150, 333, 4, 2), (200, 260, 5, 3), (67, 129, 2, 4), (129, 257, 6, 5),
    (2, 2, 1, 6), (3, 300, 1, 7), (300, 3, 1, 8), (256, 256, 7, 9), (65, 130, 1, 10),
]


@pytest.mark.parametrize("H,W,levels,seed", CASES)
@pytest.mark.parametrize("mode", [0, 1])
def test_solve_uint8_matches_oracle(H, W, levels, seed, mode):
    sc = scenes.tilted_plane_scene(H=H, W=W, seed=seed, m=24, pmin=3.0, pmax=40.0)
    a, b = _pair(sc, 2.0)
    ctx = ft.TtcContext(H, W, levels, 1)
    got = ft.results_to_numpy(ctx.solve(a.to(DEV), b.to(DEV), levels=levels, mode=mode))
    ref = oracle.ttc_pair(a.numpy(), b.numpy(), levels=levels, mode=mode)
    for l in range(levels):
        check_record(got[l], ref[l], mode, l)
    ctx.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_solve_float32_c0_sequence(mode):
    """C0-like: 32 float32 128x128 frames of a fronto-parallel plane, all 31 pairs."""
    sc = scenes.fronto_parallel_scene(H=128, W=128, seed=0, Z0=10.0, speed=0.1)
    fr = scenes.render_sequence(sc, 32)
    ctx = ft.TtcContext(128, 128, 3, 31)
    got = ft.results_to_numpy(ctx.solve_sequence(fr.to(DEV), levels=3, mode=mode)).reshape(31, 3)
    for t in range(31):
        ref = oracle.ttc_pair(fr[t].double().numpy(), fr[t + 1].double().numpy(), levels=3, mode=mode)
        for l in range(3):
            check_record(got[t, l], ref[l], mode, l, rel=SUM_REL_F32)
    ctx.close()


def test_sequence_equals_single_pairs_bitwise():
    sc = scenes.tilted_plane_scene(H=140, W=270, seed=12, m=16)
    fr = scenes.render_sequence(sc, 5).to(DEV)
    ctx = ft.TtcContext(140, 270, 4, 4)
    seq = ft.results_to_numpy(ctx.solve_sequence(fr, levels=4, mode=1)).reshape(4, 4)
    for t in range(4):
        one = ft.results_to_numpy(ctx.solve(fr[t], fr[t + 1], levels=4, mode=1))
        assert one.tobytes() == seq[t].tobytes()
    again = ft.results_to_numpy(ctx.solve_sequence(fr, levels=4, mode=1)).reshape(4, 4)
    assert again.tobytes() == seq.tobytes()
    ctx.close()


@pytest.mark.parametrize("T,H,W,dtype,pinned,max_pairs", [
    (150, 1080, 1920, torch.uint8, True, 149),      # three chunks (64, 64, 21), TMA level 0
    (40, 243, 337, torch.uint8, False, 39),         # one chunk, pageable frames, odd sizes
    (70, 96, 160, torch.float32, True, 20),         # chunks limited by the context (20, 20, 20, 9)
])
def test_host_sequence_equals_device_sequence_bitwise(T, H, W, dtype, pinned, max_pairs):
    """Host frames in chunks whose uploads overlap the compute give bitwise the records
    of the device-frame call (tile plans of the whole sequence)."""
    sc = scenes.tilted_plane_scene(H=H, W=W, seed=T, m=16, quantize=dtype == torch.uint8)
    fr = scenes.render_sequence(sc, T, device=DEV)
    ctx = ft.TtcContext(H, W, 4, max_pairs)
    if max_pairs >= T - 1:
        dev = ft.results_to_numpy(ctx.solve_sequence(fr, levels=4, mode=1)).reshape(T - 1, 4)
    else:
        # the device reference in pieces of the context's size, tile plan of the whole sequence
        big = ft.TtcContext(H, W, 4, T - 1)
        dev = ft.results_to_numpy(big.solve_sequence(fr, levels=4, mode=1)).reshape(T - 1, 4)
        big.close()
    host = fr.cpu()
    if pinned:
        host = host.pin_memory()
    got = ctx.solve_sequence(host, levels=4, mode=1)
    torch.cuda.synchronize()
    assert not got.is_cuda
    got = ft.results_to_numpy(got).reshape(T - 1, 4)
    assert got.tobytes() == dev.tobytes()
    again = ft.results_to_numpy(ctx.solve_sequence(host, levels=4, mode=1)).reshape(T - 1, 4)
    torch.cuda.synchronize()
    assert again.tobytes() == dev.tobytes()
    ctx.close()


def test_host_sequence_errors():
    ctx = ft.TtcContext(64, 64, 2, 4)
    fr = torch.zeros((3, 64, 64), dtype=torch.uint8)
    with pytest.raises(ValueError):
        ctx.solve_sequence(fr, levels=2, out=torch.empty(10, dtype=torch.uint8))
    L = ft.load()
    import ctypes
    out = torch.empty(2 * 2 * ft.RESULT_DTYPE.itemsize, dtype=torch.uint8)
    # frame stride shorter than a frame
    assert L.ttc_solve_sequence_host(ctx._h, fr.data_ptr(), 64 * 32, 3, 0, 64, 64, 64, 2, 1, out.data_ptr(),
                                     None) == 2
    assert L.ttc_solve_sequence_host(ctx._h, fr.data_ptr(), 64 * 64, 1, 0, 64, 64, 64, 2, 1, out.data_ptr(),
                                     None) == 2
    assert L.ttc_solve_sequence_host(ctx._h, None, 64 * 64, 3, 0, 64, 64, 64, 2, 1, out.data_ptr(), None) == 1
    ctx.close()


def test_two_stage_api_equals_one_call():
    sc = scenes.tilted_plane_scene(H=100, W=150, seed=13, m=16)
    fr = scenes.render_sequence(sc, 3).to(DEV)
    ctx = ft.TtcContext(100, 150, 3, 2)
    one = ft.results_to_numpy(ctx.solve_sequence(fr, levels=3, mode=1))
    ctx.partial_sums(fr, levels=3)
    out = ctx.new_results(6)
    ctx.reduce_solve(out, mode=1)
    assert ft.results_to_numpy(out).tobytes() == one.tobytes()
    ctx.close()


def test_unaligned_pitch_uint8():
    H, W = 90, 201
    sc = scenes.tilted_plane_scene(H=H, W=W, seed=14, m=16)
    a, b = _pair(sc)
    buf = torch.zeros((2, H, W + 3), dtype=torch.uint8, device=DEV)     # odd pitch: scalar loads
    buf[0, :, :W] = a.to(DEV)
    buf[1, :, :W] = b.to(DEV)
    ctx = ft.TtcContext(H, W, 3, 1)
    got = ft.results_to_numpy(ctx.solve(buf[0, :, :W], buf[1, :, :W], levels=3, mode=1))
    ref = oracle.ttc_pair(a.numpy(), b.numpy(), levels=3, mode=1)
    for l in range(3):
        check_record(got[l], ref[l], 1, l)
    ctx.close()


def test_ramp_scene_exact_ttc_float32():
    """Linear texture, fronto-parallel: C = W/Z at t + 1/2 at every level (Sec. V-A model)."""
    H, W = 130, 260
    fr = scenes.ramp_sequence(H, W, Z0=10.0, speed=0.1, a=0.3, b=-0.2, c=0.5, f=float(W)).astype(np.float32)
    ctx = ft.TtcContext(H, W, 4, 1)
    got = ft.results_to_numpy(ctx.solve(torch.from_numpy(fr[0]).to(DEV), torch.from_numpy(fr[1]).to(DEV),
                                        levels=4, mode=0))
    ref = oracle.ttc_pair(fr[0].astype(np.float64), fr[1].astype(np.float64), levels=4, mode=0)
    expect = 0.1 / (10.0 - 0.05)
    for l in range(4):
        check_record(got[l], ref[l], 0, l, rel=SUM_REL_F32)
        assert abs(got[l]["C"] - expect) < 1e-3 * expect     # float32 frames: rounding of E
    ctx.close()


def test_degenerate_identical_and_constant_frames():
    sc = scenes.tilted_plane_scene(H=64, W=96, seed=15, m=16)
    a, _ = _pair(sc)
    ctx = ft.TtcContext(64, 96, 2, 1)
    got = ft.results_to_numpy(ctx.solve(a.to(DEV), a.to(DEV), levels=2, mode=1))
    ref = oracle.ttc_pair(a.numpy(), a.numpy(), levels=2, mode=1)
    for l in range(2):
        assert got[l]["flags"] == ref[l]["flags"] == ft.FLAG_C_ZERO
        assert got[l]["ttc"] == np.inf and np.isnan(got[l]["x0"])
    c = torch.full((64, 96), 77, dtype=torch.uint8, device=DEV)
    got = ft.results_to_numpy(ctx.solve(c, c, levels=2, mode=1))
    assert all(int(r["flags"]) == ft.FLAG_SINGULAR for r in got)
    ctx.close()


def test_receding_flag():
    sc = scenes.fronto_parallel_scene(H=64, W=64, seed=16, quantize=True, pmin=8, pmax=24)
    a, b = _pair(sc, 1.0)
    ctx = ft.TtcContext(64, 64, 1, 1)
    got = ft.results_to_numpy(ctx.solve(b.to(DEV), a.to(DEV), levels=1, mode=0))     # time reversed
    ref = oracle.ttc_pair(b.numpy(), a.numpy(), levels=1, mode=0)
    check_record(got[0], ref[0], 0, 0)
    assert got[0]["flags"] == ft.FLAG_RECEDING and got[0]["ttc"] < 0
    ctx.close()


def test_errors():
    ctx = ft.TtcContext(64, 64, 3, 1)
    z = torch.zeros((64, 64), dtype=torch.uint8, device=DEV)
    with pytest.raises(ft.FtError):                  # level 6 would be 2 x 2 > context levels
        ctx.solve(z, z, levels=6, mode=1)
    small = torch.zeros((8, 8), dtype=torch.uint8, device=DEV)
    with pytest.raises(ft.FtError):                  # 8 >> 3 = 1 < 2
        ctx.solve(small, small, levels=4, mode=1)
    big = torch.zeros((200, 200), dtype=torch.uint8, device=DEV)
    with pytest.raises(ft.FtError):                  # more tiles than the context holds
        ctx.solve(big, big, levels=1, mode=1)
    with pytest.raises(ft.FtError):
        ctx.solve(z, z, levels=1, mode=5)
    ctx.close()


def test_full_size_1080p_five_levels():
    """1920x1080 uint8 tilted-plane pairs (the 1080p multi-scale workload), 5 levels, FOE."""
    sc = scenes.tilted_plane_scene(H=1080, W=1920, seed=2020)
    fr = scenes.render_sequence(sc, 3, device=DEV)
    ctx = ft.TtcContext(1080, 1920, 5, 2)
    got = ft.results_to_numpy(ctx.solve_sequence(fr, levels=5, mode=1)).reshape(2, 5)
    host = fr.cpu().numpy()
    for t in range(2):
        ref = oracle.ttc_pair(host[t], host[t + 1], levels=5, mode=1)
        for l in range(5):
            check_record(got[t, l], ref[l], 1, l)
    ctx.close()


def test_full_size_video_large_tile_paths():
    """35 consecutive 1080p pairs: all five levels in one launch of the all-levels kernel
    (strips cut into units of three tiles, so units below the top of a strip run the
    prologue), then the merge/solve; sampled pairs against the oracle, and the
    single-pair entry point (one-tile units) bitwise equal to the video."""
    sc = scenes.tilted_plane_scene(H=1080, W=1920, seed=2031)
    fr = scenes.render_sequence(sc, 36, device=DEV)
    ctx = ft.TtcContext(1080, 1920, 5, 35)
    got = ft.results_to_numpy(ctx.solve_sequence(fr, levels=5, mode=1)).reshape(35, 5)
    # the all-levels kernel and the merge/solve
    assert ctx.last_launch_count == 2
    host = fr.cpu().numpy()
    for t in (0, 17, 34):
        ref = oracle.ttc_pair(host[t], host[t + 1], levels=5, mode=1)
        for l in range(5):
            check_record(got[t, l], ref[l], 1, l)
        one = ft.results_to_numpy(ctx.solve(fr[t], fr[t + 1], levels=5, mode=1))
        assert one.tobytes() == got[t].tobytes()
    ctx.close()


def _gradient_check(E, got_mag, got_dir, integer):
    """|E| to 1.2e-7 relative for uint8 (Ex, Ey exact), direction to 5e-7 rad (the
    kernel's arctangent: minimax polynomial after the octant reduction, worst case
    4.4e-7 rad with the FP32 rounding of t, pi/2 and pi; uint8 images give millions of
    exact (Ex, Ey) pairs, octant boundaries and axes included); float frames add the
    FP32 rounding of the differences, 1e-6 of the block's absolute sum, propagated to
    the direction through 1/|E|."""
    mag, ang = oracle.gradient(E)
    E = np.asarray(E, np.float64)
    blk = np.abs(E[:-1, :-1]) + np.abs(E[:-1, 1:]) + np.abs(E[1:, :-1]) + np.abs(E[1:, 1:])
    dm = np.abs(got_mag.astype(np.float64) - mag)
    bound_m = 1.2e-7 * mag + (0.0 if integer else 1e-6 * blk)
    assert np.all(dm <= bound_m + 1e-30), float(np.max(dm - bound_m))
    d = np.abs(np.angle(np.exp(1j * (got_dir.astype(np.float64) - ang))))
    ok = mag > 0
    bound_d = 5e-7 + (np.zeros_like(mag) if integer else 1e-6 * blk / np.maximum(mag, 1e-300))
    assert np.all(d[ok] <= bound_d[ok]), float(np.max(d[ok] - bound_d[ok]))
    assert np.all(np.abs(got_dir) <= np.float32(np.pi))


def test_gradient_matches_oracle_uint8_full_size():
    sc = scenes.tilted_plane_scene(H=1080, W=1920, seed=21)
    img = scenes.render(sc, 3.0)
    mag, ang = ft.gradient(img.to(DEV))
    _gradient_check(img.numpy(), mag.cpu().numpy(), ang.cpu().numpy(), True)


@pytest.mark.parametrize("H,W,pad,offset", [(37, 53, 3, 0), (2, 2, 0, 0), (9, 300, 0, 1), (70, 33, 5, 1)])
def test_gradient_odd_shapes_pitch_and_dtypes(H, W, pad, offset):
    rng = np.random.default_rng(H * W)
    for integer in (True, False):
        E = (rng.integers(0, 256, (H, W)) if integer else rng.standard_normal((H, W))).astype(
            np.uint8 if integer else np.float32)
        buf = torch.zeros((H * (W + pad) + offset,), dtype=torch.uint8 if integer else torch.float32, device=DEV)
        view = buf[offset:].view(H, W + pad)[:, :W]
        view.copy_(torch.from_numpy(E))
        mag, ang = ft.gradient(view)
        _gradient_check(E, mag.cpu().numpy(), ang.cpu().numpy(), integer)
    # one output only
    m_only, none = ft.gradient(view, with_dir=False)
    assert none is None and torch.equal(m_only, mag)


@pytest.mark.parametrize("dtype", ["u8", "f32"])
def test_gradient_batch_equals_single_images(dtype):
    """One launch over a batch (3-D input, image stride larger than the image) gives
    each image's outputs bitwise as the single-image call, and matches the oracle."""
    rng = np.random.default_rng(7)
    H, W, n = 37, 53, 5
    if dtype == "u8":
        big = torch.from_numpy(rng.integers(0, 256, (n, H + 3, W + 5), dtype=np.uint8)).to(DEV)
    else:
        big = torch.from_numpy(rng.random((n, H + 3, W + 5), dtype=np.float32)).to(DEV)
    batch = big[:, :H, :W]                      # row pitch W + 5, image stride (H + 3)(W + 5)
    mag, ang = ft.gradient(batch)
    assert mag.shape == (n, H - 1, W - 1)
    for k in range(n):
        m1, a1 = ft.gradient(batch[k])
        assert torch.equal(m1, mag[k]) and torch.equal(a1, ang[k])
        _gradient_check(batch[k].cpu().numpy(), mag[k].cpu().numpy(), ang[k].cpu().numpy(), dtype == "u8")


def test_gradient_batch_errors():
    L = ft.load()
    x = torch.zeros((3, 4, 4), dtype=torch.uint8, device=DEV)
    out = torch.empty((3, 3, 3), device=DEV)
    assert L.ttc_gradient_batch(x.data_ptr(), 0, 16, 0, 4, 4, 4, out.data_ptr(), None, None) == 2
    assert L.ttc_gradient_batch(x.data_ptr(), 3, 8, 0, 4, 4, 4, out.data_ptr(), None, None) == 2
    assert L.ttc_gradient_batch(x.data_ptr(), 70000, 16, 0, 4, 4, 4, out.data_ptr(), None, None) == 3
    assert L.ttc_gradient_batch(None, 3, 16, 0, 4, 4, 4, out.data_ptr(), None, None) == 1
    xf = torch.zeros((2, 4, 4), dtype=torch.float32, device=DEV)
    # float images 66 bytes apart: not a whole number of pixels
    assert L.ttc_gradient_batch(xf.data_ptr(), 2, 66, 1, 4, 4, 16, out.data_ptr(), None, None) == 2
    assert L.ttc_gradient_batch(x.data_ptr(), 3, 16, 0, 4, 4, 4, out.data_ptr(), None, None) == 0
    torch.cuda.synchronize()
    m, _ = ft.gradient(torch.zeros((0, 4, 4), dtype=torch.uint8, device=DEV), with_dir=False)
    assert m.shape == (0, 3, 3)


def test_gradient_errors():
    L = ft.load()
    x = torch.zeros((4, 4), dtype=torch.uint8, device=DEV)
    out = torch.empty((3, 3), device=DEV)
    assert L.ttc_gradient(x.data_ptr(), 0, 4, 4, 4, None, None, None) == 1
    assert L.ttc_gradient(x.data_ptr(), 0, 1, 4, 4, out.data_ptr(), None, None) == 2
    assert L.ttc_gradient(x.data_ptr(), 0, 4, 4, 3, out.data_ptr(), None, None) == 2
    assert L.ttc_gradient(x.data_ptr(), 7, 4, 4, 4, out.data_ptr(), None, None) == 1


def test_reserve_host_waits_only_for_its_own_context():
    """Growing one context's host-sequence buffers does not synchronise the device: a
    long kernel on another stream is still running when the reservation returns; both
    contexts then give bitwise the same records for the same host video."""
    H, W, levels = 96, 160, 3
    sc = scenes.tilted_plane_scene(H=H, W=W, seed=31, m=16)
    frames = scenes.render_sequence(sc, 24).pin_memory()
    a = ft.TtcContext(H, W, levels, 23)
    b = ft.TtcContext(H, W, levels, 23)
    b.reserve_host(frames[:4], levels=levels)              # small buffers first
    other = torch.cuda.Stream()
    with torch.cuda.stream(other):
        torch.cuda._sleep(int(2e9))                        # about a second of GPU clock
    b.reserve_host(frames, levels=levels)                  # grows: frees and allocates
    assert not other.query(), "the reservation waited for another stream's work"
    ra = ft.results_to_numpy(a.solve_sequence(frames, levels=levels, mode=1))
    rb = ft.results_to_numpy(b.solve_sequence(frames, levels=levels, mode=1))
    torch.cuda.synchronize()
    assert ra.tobytes() == rb.tobytes()
    dev = ft.results_to_numpy(a.solve_sequence(frames.to(DEV), levels=levels, mode=1))
    assert dev.tobytes() == ra.tobytes()
    a.close()
    b.close()


def test_host_sequence_needs_reserved_buffers():
    L = ft.load()
    H, W = 64, 96
    fr = torch.zeros((5, H, W), dtype=torch.uint8).pin_memory()
    ctx = ft.TtcContext(H, W, 2, 4)
    out = torch.empty(4 * 2 * ft.RESULT_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    st = L.ttc_solve_sequence_host(ctx._h, fr.data_ptr(), H * W, 5, 0, H, W, W, 2, 1, out.data_ptr(),
                                   torch.cuda.current_stream().cuda_stream)
    assert st == 4                                          # FT_ERR_WORKSPACE: nothing reserved
    ctx.reserve_host(fr, levels=2)
    st = L.ttc_solve_sequence_host(ctx._h, fr.data_ptr(), H * W, 5, 0, H, W, W, 2, 1, out.data_ptr(),
                                   torch.cuda.current_stream().cuda_stream)
    assert st == 0
    torch.cuda.synchronize()
    ctx.close()
