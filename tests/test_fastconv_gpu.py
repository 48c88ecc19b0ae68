"""FastConv (full n-D convolution) through the C ABI vs the FP64 oracle.

Error metric (stated for FP32 with fixed-order accumulation): every element obeys
    |y - y*| <= 1e-5 * (|E| conv |k|)[p],
the natural bound for a dot product, relative to the absolute-value convolution
(a plain relative error is ill-posed where y* ~ 0 for mixed-sign kernels).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1612_08825_gb300 as ft
import scenes

pytestmark = pytest.mark.gpu
REL = 1e-5


def _run(E: np.ndarray, k: np.ndarray, offset: int = 0) -> np.ndarray:
    dev = torch.device("cuda")
    if offset:
        buf = torch.zeros(E.size + offset, dtype=torch.float32, device=dev)
        x = buf[offset:].view(E.shape)
        x.copy_(torch.from_numpy(E))
    else:
        x = torch.from_numpy(E).to(dev)
    out = ft.fastconv_nd(x, torch.from_numpy(k).to(dev))
    ft.fastconv_check()             # no bounded wait gave up
    return out.cpu().numpy()


def _check_full(E, k, offset=0):
    got = _run(E, k, offset)
    ref, rabs = oracle.fastconv_nd(E, k, with_abs=True)
    assert got.shape == ref.shape
    err = np.abs(got.astype(np.float64) - ref)
    assert np.all(err <= REL * rabs + 1e-30), float(np.max(err / np.maximum(rabs, 1e-30)))
    return float(np.max(err / np.maximum(rabs, 1e-30)))


@pytest.mark.parametrize("shape,kshape", [
    ((1,), (1,)), ((17,), (5,)), ((3000,), (31,)), ((5,), (40,)),
    ((1, 1), (1, 1)), ((7, 9), (3, 3)), ((70, 300), (3, 3)), ((130, 261), (2, 2)),
    ((99, 257), (7, 7)), ((66, 140), (15, 15)), ((40, 37), (1, 6)), ((33, 50), (9, 1)),
    ((3, 4), (6, 9)),                        # kernel larger than the input
    ((5, 37, 45), (2, 3, 4)), ((9, 40, 33), (5, 5, 5)), ((4, 3, 20, 21), (2, 1, 3, 2)),
    ((6, 1, 300), (1, 1, 3)), ((5, 2, 132), (1, 2, 2)), ((4, 70, 264), (1, 3, 3)),   # batches, small kernels
    ((2, 2, 2, 2, 2, 2, 3, 5), (2, 1, 2, 1, 2, 1, 2, 3)),   # rank 8
])
def test_fastconv_small_shapes(shape, kshape):
    E = scenes.normal_array(shape, seed=sum(shape))
    k = scenes.normal_array(kshape, seed=100 + sum(kshape))
    _check_full(E, k)


@pytest.mark.parametrize("shape,kshape", [
    ((37, 256), (2, 2)), ((45, 257), (3, 3)), ((20, 130), (1, 3)), ((70, 253), (2, 2)),
    ((5, 33, 256), (2, 2, 2)), ((4, 19, 258), (2, 3, 3)), ((3, 70, 129), (2, 1, 2)),
    ((6, 40, 126), (1, 3, 3)),
])
def test_fastconv_streaming_narrow_last_strip(shape, kshape):
    """Outputs whose last 128-column strip has 1-4 columns (257, 259, 132, 254, 257, 260,
    130, 128 + 0): that strip is taken with a lane per output row; planes with one or
    two leading kernel taps, unaligned rows, pointer and image edges."""
    E = scenes.normal_array(shape, seed=sum(shape) + 1)
    k = scenes.normal_array(kshape, seed=200 + sum(kshape))
    _check_full(E, k)
    _check_full(E, k, offset=1)


@pytest.mark.parametrize("shape,kshape", [
    ((8, 40, 256), (5, 5, 5)), ((6, 70, 128), (1, 7, 7)), ((50, 1000), (15, 15)), ((4, 33, 264), (3, 4, 9)),
    ((5, 36, 384), (1, 6, 17)), ((70, 252), (9, 5)),
])
def test_fastconv_copy_engine_narrow_last_tile(shape, kshape):
    """FMA-bound kernels on the copy-engine path whose last 128-column output tile has few
    columns inside the output (260, 134, 272, 400 columns; 1014 and 256 as controls)."""
    E = scenes.normal_array(shape, seed=sum(shape) + 7)
    k = scenes.normal_array(kshape, seed=300 + sum(kshape))
    _check_full(E, k)


@pytest.mark.parametrize("kc", [5, 9, 17, 33, 65, 70])
def test_fastconv_every_padding_bucket_and_direct_fallback(kc):
    E = scenes.uniform_array((20, 150), seed=kc)
    k = scenes.normal_array((2, kc), seed=kc + 1)
    _check_full(E, k)


def test_fastconv_unaligned_input_and_odd_width():
    E = scenes.uniform_array((41, 203), seed=3)
    k = scenes.normal_array((3, 3), seed=4)
    _check_full(E, k, offset=1)          # input pointer not 16-byte aligned
    E = scenes.uniform_array((41, 200), seed=5)
    _check_full(E, k, offset=1)
    _check_full(E, k, offset=0)          # aligned, width multiple of 4 (vector path)


def test_fastconv_paper_masks_and_delta():
    # Sec. II derivative mask and Sec. III edge kernels on an image with a vertical edge
    img = np.zeros((6, 9), np.float32)
    img[:, 4:] = 1.0
    kx = np.array([[-0.5, 0.5], [-0.5, 0.5]], np.float32)
    sobel = np.array([[-1, 0, 1], [-2, 0, 2], [-1, 0, 1]], np.float32)
    for k in (kx, sobel, kx.T.copy()):
        got = _run(img, k)
        np.testing.assert_array_equal(got, oracle.fastconv_nd(img, k).astype(np.float32))
    E = scenes.normal_array((13, 29), seed=9)
    d = np.zeros((3, 4), np.float32)
    d[1, 2] = 1.0
    got = _run(E, d)
    np.testing.assert_array_equal(got[1:14, 2:31], E)


def test_fastconv_deterministic():
    E = scenes.uniform_array((300, 500), seed=11)
    k = scenes.normal_array((7, 7), seed=12)
    a = _run(E, k)
    b = _run(E, k)
    np.testing.assert_array_equal(a, b)


def test_fastconv_rejects_empty_and_bad_rank():
    dev = torch.device("cuda")
    with pytest.raises(ft.FtError):
        ft.fastconv_nd(torch.zeros((0, 4), device=dev), torch.ones((1, 1), device=dev))
    with pytest.raises(ValueError):
        ft.fastconv_nd(torch.zeros((4, 4), device=dev), torch.ones((1,), device=dev))


FULL_2D = [2, 3, 7, 15]


@pytest.mark.parametrize("kk", FULL_2D)
def test_fastconv_full_size_2d_every_element(kk):
    """1080x1920 U[0,1] conv normalised Gaussian k x k (sigma = k/6): every output
    element against the FP64 oracle, and the sum identity."""
    E = scenes.uniform_array((1080, 1920), seed=2024)
    k = scenes.gaussian_kernel(kk)
    got = _run(E, k)
    ref, rabs = oracle.fastconv_nd(E, k, with_abs=True)
    assert got.shape == ref.shape
    err = np.abs(got.astype(np.float64) - ref)
    assert np.all(err <= REL * rabs + 1e-30), float(np.max(err / np.maximum(rabs, 1e-30)))
    # sum identity over the whole output: sum(out) = sum(E) * sum(k)
    tot = got.astype(np.float64).sum()
    expect = E.astype(np.float64).sum() * k.astype(np.float64).sum()
    assert abs(tot - expect) <= REL * abs(expect)


@pytest.mark.parametrize("kk", [2, 5])
def test_fastconv_full_size_3d_every_element(kk):
    """64x256x256 U[0,1] conv k^3 N(0,1): every output element against the FP64
    oracle, and the sum identity."""
    E = scenes.uniform_array((64, 256, 256), seed=77)
    k = scenes.normal_array((kk, kk, kk), seed=78)
    got = _run(E, k)
    ref, rabs = oracle.fastconv_nd(E, k, with_abs=True)
    assert got.shape == ref.shape
    err = np.abs(got.astype(np.float64) - ref)
    assert np.all(err <= REL * rabs + 1e-30), float(np.max(err / np.maximum(rabs, 1e-30)))
    tot = got.astype(np.float64).sum()
    expect = E.astype(np.float64).sum() * k.astype(np.float64).sum()
    scale = np.abs(E).astype(np.float64).sum() * np.abs(k).astype(np.float64).sum()
    assert abs(tot - expect) <= REL * scale


@pytest.mark.parametrize("kc", list(range(1, 18)))
def test_fastconv_tma_and_load_paths_bitwise(kc):
    """The copy-engine kernel and the load-path kernel (taken for an input at a 4-byte
    offset) apply the taps of every output in the same order, so their outputs are the
    same bits; kernels of 4 and more rows, several 128-column tiles with a ragged tail,
    two planes."""
    for kr in (4, 9):
        k = scenes.normal_array((kr, kc), seed=300 + kc + kr)
        E = scenes.uniform_array((45, 600), seed=kc + 7)
        assert np.array_equal(_run(E, k), _run(E, k, offset=1))
    E3 = scenes.uniform_array((2, 29, 272), seed=kc + 9)
    k3 = scenes.normal_array((2, 5, kc), seed=kc + 11)
    assert np.array_equal(_run(E3, k3), _run(E3, k3, offset=1))


@pytest.mark.parametrize("kc", list(range(2, 18)))
def test_fastconv_fma_kernel_every_width(kc):
    """The FMA-bound kernels for every kernel width they serve (2..17 columns): rows equal to the tile's rows per thread (middle phase of length one) and
    longer; several 128-column tiles with a ragged tail; a width that is not a
    multiple of 4 and an offset base (scalar staging); two planes.  Kernels of 1-3 rows
    take the copy-engine kernel's small-row schedule (or the tile kernel when the rows
    are not addressable by the copy engine)."""
    for kr in (1, 2, 3, 4, 9):
        k = scenes.normal_array((kr, kc), seed=100 + kc + kr)
        _check_full(scenes.uniform_array((45, 600), seed=kc), k)
        _check_full(scenes.uniform_array((37, 531), seed=kc + 1), k)
        _check_full(scenes.uniform_array((30, 300), seed=kc + 2), k, offset=1)
    _check_full(scenes.uniform_array((2, 29, 270), seed=kc + 3), scenes.normal_array((2, 4, kc), seed=kc))


def test_fastconv_fma_kernel_large_grid():
    """Enough tiles for the 64-row variant (16 planes of 300 x 1100; 8 x 7 and 9 x 9
    kernels), the 32-row variant for wide and tall kernels, compared with the oracle
    on sampled outputs of every plane."""
    E = scenes.uniform_array((16, 300, 1100), seed=31)
    for ks in ((1, 8, 7), (1, 9, 9), (1, 15, 15), (1, 33, 5), (1, 4, 17)):
        k = scenes.normal_array(ks, seed=sum(ks))
        got = _run(E, k)
        rng = np.random.default_rng(ks[1])
        pts = rng.integers(0, got.size, 4000).astype(np.int64)
        ref, rabs = oracle.fastconv_points(E, k, pts)
        g = got.reshape(-1)[pts].astype(np.float64)
        assert np.all(np.abs(g - ref) <= REL * rabs + 1e-30), ks


@pytest.mark.parametrize("shape,kshape", [
    ((3, 40, 264), (2, 5, 5)), ((3, 40, 264), (3, 7, 9)), ((5, 33, 128), (5, 5, 5)),
    ((2, 2, 20, 68), (2, 2, 4, 5)), ((2, 3, 17, 36), (3, 1, 6, 7)),
])
def test_fastconv_tma_kernel_leading_dims(shape, kshape):
    """The persistent copy-engine-fed kernel over several leading kernel indices per
    output tile (planes outside the input skipped), rank 4 (general leading-index
    decomposition), row lengths that are multiples of 4 (copy engine path) with output
    rows that are (TMA store) or are not (plain stores) multiples of 4."""
    E = scenes.uniform_array(shape, seed=sum(shape))
    k = scenes.normal_array(kshape, seed=sum(kshape))
    _check_full(E, k)


@pytest.mark.parametrize("shape,klens", [
    ((37, 531), (7, 5)), ((300,), (9,)), ((5, 33, 128), (3, 5, 7)), ((2, 3, 17, 36), (2, 1, 6, 7)),
    ((64, 64), (1, 17)), ((40, 100), (33, 1)),
])
def test_fastconv_separable_matches_full_conv(shape, klens):
    """One 1-D pass per axis equals the full convolution with the outer-product kernel."""
    E = scenes.uniform_array(shape, seed=sum(shape))
    facs = [scenes.normal_array((k,), seed=10 + i) for i, k in enumerate(klens)]
    k = facs[0].astype(np.float64)
    for f in facs[1:]:
        k = np.multiply.outer(k, f.astype(np.float64))
    dev = torch.device("cuda")
    got = ft.fastconv_separable(torch.from_numpy(E).to(dev), [torch.from_numpy(f).to(dev) for f in facs])
    ft.fastconv_check()
    ref, rabs = oracle.fastconv_nd(E, k, with_abs=True)
    err = np.abs(got.cpu().numpy().astype(np.float64) - ref)
    assert np.all(err <= REL * rabs + 1e-30), float(np.max(err / np.maximum(rabs, 1e-30)))


def test_fastconv_separable_full_size_gaussian_sampled():
    """1080x1920 conv 15x15 normalised Gaussian through the factored path, sampled."""
    E = scenes.uniform_array((1080, 1920), seed=2024)
    k = scenes.gaussian_kernel(15)
    facs = ft.factor_kernel(k, rel_tol=1e-6)
    assert facs is not None
    dev = torch.device("cuda")
    got = ft.fastconv_separable(torch.from_numpy(E).to(dev), [torch.from_numpy(f).to(dev) for f in facs])
    got = got.cpu().numpy()
    pts = np.random.default_rng(5).integers(0, got.size, 3000).astype(np.int64)
    ref, rabs = oracle.fastconv_points(E, k, pts)
    g = got.reshape(-1)[pts].astype(np.float64)
    # the factors carry the rank-1 test's rounding (1e-6 of the largest tap)
    assert np.all(np.abs(g - ref) <= 2e-5 * rabs + 1e-30)


_TYPED = [torch.uint8, torch.int16, torch.float16, torch.bfloat16]


def _typed_input(shape, dtype, seed):
    rng = np.random.default_rng(seed)
    if dtype == torch.uint8:
        return torch.from_numpy(rng.integers(0, 256, shape).astype(np.uint8))
    if dtype == torch.int16:
        return torch.from_numpy(rng.integers(-32768, 32768, shape).astype(np.int16))
    return torch.from_numpy(rng.standard_normal(shape).astype(np.float32) * 3).to(dtype)


@pytest.mark.parametrize("dtype", _TYPED)
@pytest.mark.parametrize("shape,kshape", [
    ((45, 640), (7, 5)), ((40, 640), (1, 9)), ((33, 320), (3, 17)), ((37, 531), (5, 5)),
    ((3, 24, 96), (2, 4, 3)), ((700,), (9,)), ((30, 64), (3, 40)), ((20, 96), (2, 2)),
    ((3, 30, 256), (2, 5, 5)),               # copy-engine tiles, a 4-column last tile
])
def test_fastconv_typed_inputs_match_oracle(dtype, shape, kshape):
    """uint8 / int16 / float16 / bfloat16 inputs, widened to FP32 exactly: the copy
    engine path (aligned rows, up to 17 kernel columns) and the converted-copy path
    (odd widths, rank 1, wide kernels) against the oracle on the same values."""
    x = _typed_input(shape, dtype, sum(shape))
    k = scenes.normal_array(kshape, seed=sum(kshape))
    dev = torch.device("cuda")
    got = ft.fastconv_nd(x.to(dev), torch.from_numpy(k).to(dev))
    ft.fastconv_check()
    E = x.float().numpy().astype(np.float64)
    ref, rabs = oracle.fastconv_nd(E, k, with_abs=True)
    err = np.abs(got.cpu().numpy().astype(np.float64) - ref)
    assert np.all(err <= REL * rabs + 1e-30), float(np.max(err / np.maximum(rabs, 1e-30)))


def test_fastconv_typed_paths_and_errors():
    """An aligned request runs without scratch (fused staging); an unaligned one asks for
    it; a bad element type is rejected."""
    L = ft.load()
    dev = torch.device("cuda")
    k = torch.from_numpy(scenes.normal_array((5, 5), seed=1)).to(dev)
    import ctypes
    dims = (ctypes.c_int64 * 2)(32, 64)
    kd = (ctypes.c_int64 * 2)(5, 5)
    x = torch.zeros((32, 64), dtype=torch.uint8, device=dev)
    out = torch.empty((36, 68), device=dev)
    assert L.fastconv_nd_typed(x.data_ptr(), 0, dims, 2, k.data_ptr(), kd, out.data_ptr(), None, None) == 0
    dims2 = (ctypes.c_int64 * 2)(32, 63)
    assert L.fastconv_nd_typed(x.data_ptr(), 0, dims2, 2, k.data_ptr(), kd, out.data_ptr(), None, None) == 4
    assert L.fastconv_nd_typed(x.data_ptr(), 9, dims, 2, k.data_ptr(), kd, out.data_ptr(), None, None) == 1
    torch.cuda.synchronize()


@pytest.mark.parametrize("shape,kshape", [
    ((300,), (41,)), ((64, 80), (31, 33)), ((5, 33, 40), (3, 9, 9)), ((7, 9), (12, 30)), ((120, 200), (45, 45)),
])
def test_fastconv_fft_matches_oracle_normwise(shape, kshape):
    """The FFT path against the oracle within its normwise bound: FP32 rounding times
    log2 of the transform size times ||E||_2 ||k||_2 (a factor 8 of margin)."""
    E = scenes.uniform_array(shape, seed=sum(shape))
    k = scenes.normal_array(kshape, seed=sum(kshape))
    dev = torch.device("cuda")
    got = ft.fastconv_fft(torch.from_numpy(E).to(dev), torch.from_numpy(k).to(dev)).cpu().numpy()
    ref = oracle.fastconv_nd(E, k)
    R = np.prod([m + 8 for m in ref.shape])
    bound = 8 * 2.0 ** -24 * np.log2(R) * np.linalg.norm(E.ravel()) * np.linalg.norm(k.ravel())
    err = np.abs(got.astype(np.float64) - ref)
    assert err.max() <= bound, (err.max(), bound)


def test_fastconv_fft_errors_and_auto_switch():
    L = ft.load()
    import ctypes
    dims = (ctypes.c_int64 * 4)(2, 2, 8, 8)
    kd = (ctypes.c_int64 * 4)(1, 1, 3, 3)
    h = ctypes.c_void_p()
    b = ctypes.c_size_t()
    assert L.fastconv_fft_plan_create(dims, 4, kd, ctypes.byref(h), ctypes.byref(b)) == 3      # rank 4
    assert not h.value
    dev = torch.device("cuda")
    x = torch.rand((64, 64), device=dev)
    k = torch.rand((5, 5), device=dev)
    with pytest.raises(ft.FtError):
        _fft_small_workspace(L, x, k)                                    # workspace too small
    small = ft.fastconv(x, k)                                   # below the threshold: direct
    big = ft.fastconv(x, torch.rand((41, 41), device=dev))      # small image: direct as well
    assert small.shape == (68, 68) and big.shape == (104, 104)
    d2, d3 = (ctypes.c_int64 * 2), (ctypes.c_int64 * 3)
    assert L.fastconv_prefers_fft(d2(1080, 1920), 2, d2(29, 29)) == 0
    assert L.fastconv_prefers_fft(d2(1080, 1920), 2, d2(31, 31)) == 1
    assert L.fastconv_prefers_fft(d2(64, 64), 2, d2(31, 31)) == 0                # output area too small
    assert L.fastconv_prefers_fft(d3(64, 256, 256), 3, d3(10, 10, 10)) == 0      # 3-D: not measured


def test_fastconv_fft_two_streams_one_plan_bitwise():
    """One plan, two streams with their own workspaces, calls interleaved: each output
    bitwise equal to the same call made alone on the default stream."""
    dev = torch.device("cuda")
    E = [torch.from_numpy(scenes.uniform_array((300, 400), seed=s)).to(dev) for s in (1, 2)]
    k = torch.from_numpy(scenes.normal_array((33, 33), seed=3)).to(dev)
    plan = ft.FftPlan((300, 400), (33, 33), dev)
    ref = [plan(e, k).clone() for e in E]
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    ws = [plan.new_workspace(), plan.new_workspace()]
    outs = [torch.empty_like(ref[0]), torch.empty_like(ref[1])]
    for _ in range(5):
        for i in (0, 1):
            streams[i].wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(streams[i]):
                plan(E[i], k, out=outs[i], workspace=ws[i])
    torch.cuda.synchronize()
    for i in (0, 1):
        assert torch.equal(outs[i], ref[i])
    plan.close()


def _fft_small_workspace(L, x, k):
    plan = ft.FftPlan(tuple(x.shape), tuple(k.shape), x.device)
    out = torch.empty((68, 68), device=x.device)
    ws = torch.empty(256, dtype=torch.uint8, device=x.device)
    st = L.fastconv_fft(plan._h, x.data_ptr(), k.data_ptr(), out.data_ptr(), ws.data_ptr(), 256, None)
    plan.close()
    if st != 0:
        raise ft.FtError(st, "fastconv_fft")
