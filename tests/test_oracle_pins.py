"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Every check here compares the oracle with something it does not compute itself:
closed forms, library routines that implement the same mathematics (numpy.polymul,
scipy.signal.convolve/correlate2d, numpy.linalg.solve), exact rational arithmetic on
tiny integer inputs, invariances, and values worked by hand from the paper's text
(fixtures under tests/golden/, each with its citation).
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.signal

import oracle
import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# --------------------------------------------------------------------------- #
# Convolution (Eq. conv2, full extent)
# --------------------------------------------------------------------------- #

def test_conv_golden_polynomial_products():
    for case in _golden("conv_polynomial.json")["cases"]:
        out = oracle.fastconv_nd(np.array(case["E"], float), np.array(case["k"], float))
        np.testing.assert_array_equal(out, np.array(case["out"], float), err_msg=case["why"])


def test_conv_1d_equals_polymul():
    rng = np.random.default_rng(1)
    for n, k in [(1, 1), (5, 3), (17, 9), (4, 11)]:
        E = rng.integers(-9, 10, n).astype(float)
        k_ = rng.integers(-9, 10, k).astype(float)
        np.testing.assert_array_equal(oracle.fastconv_nd(E, k_), np.polymul(E, k_))


@pytest.mark.parametrize("shape,kshape", [
    ((7,), (3,)), ((6, 9), (3, 2)), ((5, 4, 6), (2, 3, 2)), ((3, 4, 2, 5), (2, 2, 3, 2)),
    ((2, 3), (5, 4)),                     # kernel larger than the input
    ((1, 1, 1), (1, 1, 1)),
])
def test_conv_matches_scipy_direct(shape, kshape):
    rng = np.random.default_rng(hash((shape, kshape)) % 2**32)
    E = rng.standard_normal(shape)
    k = rng.standard_normal(kshape)
    out, oabs = oracle.fastconv_nd(E, k, with_abs=True)
    ref = scipy.signal.convolve(E, k, mode="full", method="direct")
    assert out.shape == ref.shape
    assert np.all(np.abs(out - ref) <= 1e-13 * (oabs + 1e-300))
    ref_abs = scipy.signal.convolve(np.abs(E), np.abs(k), mode="full", method="direct")
    np.testing.assert_allclose(oabs, ref_abs, rtol=1e-13)


def test_conv_delta_and_shifted_delta():
    rng = np.random.default_rng(2)
    E = rng.standard_normal((5, 7))
    k = np.zeros((3, 4))
    k[0, 0] = 1.0
    out = oracle.fastconv_nd(E, k)
    np.testing.assert_array_equal(out[:5, :7], E)
    assert np.count_nonzero(out) == np.count_nonzero(E)
    for (a, b) in [(1, 0), (0, 3), (2, 2)]:
        k = np.zeros((3, 4))
        k[a, b] = 1.0
        out = oracle.fastconv_nd(E, k)
        np.testing.assert_array_equal(out[a:a + 5, b:b + 7], E)   # shift by +(a, b)
        assert np.count_nonzero(out) == np.count_nonzero(E)


def test_conv_sum_identity_commutativity_linearity_associativity():
    rng = np.random.default_rng(3)
    E = rng.standard_normal((6, 5, 4))
    k = rng.standard_normal((3, 2, 3))
    k2 = rng.standard_normal((3, 2, 3))
    out, oabs = oracle.fastconv_nd(E, k, with_abs=True)
    assert abs(out.sum() - E.sum() * k.sum()) <= 1e-12 * np.abs(E).sum() * np.abs(k).sum()
    np.testing.assert_allclose(oracle.fastconv_nd(k, E), out, rtol=0, atol=1e-12 * oabs.max())
    lin = oracle.fastconv_nd(E, 2.0 * k - 3.0 * k2)
    np.testing.assert_allclose(lin, 2.0 * out - 3.0 * oracle.fastconv_nd(E, k2), atol=1e-11)
    a = rng.standard_normal((2, 1, 3))
    b = rng.standard_normal((1, 3, 2))
    lhs = oracle.fastconv_nd(oracle.fastconv_nd(E, a), b)
    rhs = oracle.fastconv_nd(E, oracle.fastconv_nd(a, b))
    np.testing.assert_allclose(lhs, rhs, atol=1e-11)


def test_conv_points_match_full():
    rng = np.random.default_rng(4)
    E = rng.standard_normal((9, 8))
    k = rng.standard_normal((4, 3))
    full, fabs = oracle.fastconv_nd(E, k, with_abs=True)
    pts = rng.integers(0, full.size, 40)
    v, a = oracle.fastconv_points(E, k, pts)
    np.testing.assert_array_equal(v, full.reshape(-1)[pts])
    np.testing.assert_array_equal(a, fabs.reshape(-1)[pts])


def test_conv_out_dims():
    assert oracle.conv_out_dims((1080, 1920), (3, 3)) == (1082, 1922)
    assert oracle.conv_out_dims((64, 256, 256), (5, 5, 5)) == (68, 260, 260)


# --------------------------------------------------------------------------- #
# Down-sampling (Sec. V-B)
# --------------------------------------------------------------------------- #

def test_downsample_constant_sum_and_reshape_mean():
    img = np.full((7, 9), 3.25)
    np.testing.assert_array_equal(oracle.downsample(img), np.full((3, 4), 3.25))
    rng = np.random.default_rng(5)
    img = rng.integers(0, 256, (11, 14)).astype(float)
    d = oracle.downsample(img)
    assert d.shape == (5, 7)
    crop = img[:10, :14]
    assert d.sum() == crop.sum() / 4.0
    np.testing.assert_array_equal(d, crop.reshape(5, 2, 7, 2).mean(axis=(1, 3)))


# --------------------------------------------------------------------------- #
# Derivative stencils (Sec. II, Sec. V-A)
# --------------------------------------------------------------------------- #

def test_derivatives_golden_paper_mask():
    g = _golden("paper_mask_sec2.json")
    img = np.array(g["image"], float)
    Ex, Ey, Et = oracle.derivatives(img, img)
    np.testing.assert_array_equal(Ex, np.array(g["expected_Ex"], float))
    np.testing.assert_array_equal(Ey, np.array(g["expected_Ey"], float))
    assert not Et.any()
    # static pair == the paper's 2x2 masks applied as sliding windows
    rng = np.random.default_rng(6)
    E = rng.standard_normal((6, 8))
    Ex, Ey, _ = oracle.derivatives(E, E)
    np.testing.assert_allclose(Ex, scipy.signal.correlate2d(E, np.array(g["mask_x"]), "valid"), atol=1e-14)
    np.testing.assert_allclose(Ey, scipy.signal.correlate2d(E, np.array(g["mask_y"]), "valid"), atol=1e-14)


def test_gradient_golden_edges():
    for case in _golden("gradient_edges_sec2.json")["cases"]:
        mag, ang = oracle.gradient(np.array(case["image"], float))
        np.testing.assert_array_equal(mag, np.array(case["mag"], float), err_msg=case["name"])
        np.testing.assert_allclose(ang, np.pi * np.array(case["dir_over_pi"], float), atol=1e-15,
                                   err_msg=case["name"])


@pytest.mark.parametrize("a,b", [(1.5, 0.0), (0.0, 2.0), (-1.0, 0.5), (-0.75, -2.0), (3.0, -1.0)])
def test_gradient_closed_form_on_planes(a, b):
    """E = a x + b y (x: column, y: row) has Ex = a, Ey = b on every block: the magnitude
    is hypot(a, b) and the direction atan2(b, a), one value per quadrant."""
    yy, xx = np.mgrid[0:7, 0:9].astype(float)
    mag, ang = oracle.gradient(a * xx + b * yy + 5.0)
    np.testing.assert_allclose(mag, np.hypot(a, b), rtol=1e-14)
    np.testing.assert_allclose(ang, np.arctan2(b, a), atol=1e-14)


def test_gradient_transpose_and_range():
    """Transposing the image swaps Ex and Ey: the magnitude is transposed and the
    direction reflects about pi/4; every direction lies in [-pi, pi]."""
    E = np.random.default_rng(17).standard_normal((9, 12))
    mag, ang = oracle.gradient(E)
    magT, angT = oracle.gradient(E.T)
    np.testing.assert_allclose(magT, mag.T, rtol=1e-14)
    np.testing.assert_allclose(np.cos(angT), np.sin(ang).T, atol=1e-12)
    np.testing.assert_allclose(np.sin(angT), np.cos(ang).T, atol=1e-12)
    assert np.all(np.abs(ang) <= np.pi)


def test_derivatives_equal_interior_of_3d_full_conv():
    rng = np.random.default_rng(7)
    E0 = rng.standard_normal((5, 6))
    E1 = rng.standard_normal((5, 6))
    stack = np.stack([E0, E1])
    kx = np.zeros((2, 2, 2)); kx[:, :, 0] = 0.25; kx[:, :, 1] = -0.25
    ky = np.zeros((2, 2, 2)); ky[:, 0, :] = 0.25; ky[:, 1, :] = -0.25
    kt = np.zeros((2, 2, 2)); kt[0] = 0.25; kt[1] = -0.25
    Ex, Ey, Et = oracle.derivatives(E0, E1)
    for got, kk in [(Ex, kx), (Ey, ky), (Et, kt)]:
        ref = scipy.signal.convolve(stack, kk, mode="full", method="direct")[1, 1:5, 1:6]
        np.testing.assert_allclose(got, ref, atol=1e-14)


def test_derivatives_exact_on_trilinear():
    c = np.array([0.3, -1.2, 0.7, 2.1, 0.05, -0.4, 0.9, -0.15])
    H, W = 5, 7

    def E(x, y, t):
        return (c[0] + c[1] * x + c[2] * y + c[3] * t + c[4] * x * y + c[5] * x * t
                + c[6] * y * t + c[7] * x * y * t)

    yy, xx = np.meshgrid(np.arange(H, dtype=float), np.arange(W, dtype=float), indexing="ij")
    Ex, Ey, Et = oracle.derivatives(E(xx, yy, 0.0), E(xx, yy, 1.0))
    xc, yc, tc = xx[:-1, :-1] + 0.5, yy[:-1, :-1] + 0.5, 0.5
    np.testing.assert_allclose(Ex, c[1] + c[4] * yc + c[5] * tc + c[7] * yc * tc, atol=1e-12)
    np.testing.assert_allclose(Ey, c[2] + c[4] * xc + c[6] * tc + c[7] * xc * tc, atol=1e-12)
    np.testing.assert_allclose(Et, c[3] + c[5] * xc + c[6] * yc + c[7] * xc * yc, atol=1e-12)


# --------------------------------------------------------------------------- #
# Sums and solve (Sec. V-A)
# --------------------------------------------------------------------------- #

def test_sums_exact_rational_uint8():
    """Exact rational sums (Fractions) on tiny uint8 frames vs the oracle's FP64 sums."""
    rng = np.random.default_rng(8)
    H, W = 5, 6
    E0 = rng.integers(0, 256, (H, W))
    E1 = rng.integers(0, 256, (H, W))
    cx, cy = Fraction(W - 1, 2), Fraction(H - 1, 2)
    exact = [Fraction(0)] * 10
    for i in range(H - 1):
        for j in range(W - 1):
            # differences written per corner pair, in integers
            ex = sum(int(F[i + a, j + 1]) - int(F[i + a, j]) for F in (E0, E1) for a in (0, 1))
            ey = sum(int(F[i + 1, j + b]) - int(F[i, j + b]) for F in (E0, E1) for b in (0, 1))
            et = sum(int(E1[i + a, j + b]) - int(E0[i + a, j + b]) for a in (0, 1) for b in (0, 1))
            ex, ey, et = Fraction(ex, 4), Fraction(ey, 4), Fraction(et, 4)
            x = j + Fraction(1, 2) - cx
            y = i + Fraction(1, 2) - cy
            G = x * ex + y * ey
            for s, v in enumerate([ex * ex, ex * ey, ey * ey, G * ex, G * ey, G * G,
                                   ex * et, ey * et, G * et, et * et]):
                exact[s] += v
    Ex, Ey, Et = oracle.derivatives(E0, E1)
    s, a = oracle.sums(Ex, Ey, Et, float(cx), float(cy))
    for k in range(10):
        assert abs(s[k] - float(exact[k])) <= 1e-15 * a[k] + 1e-300


def test_sums_error_scale():
    """abssums: the sum of |term| for the six plain products; for the four G terms the
    rounding scale |x Ex| + |y Ey| replaces |G|, so it bounds |G| terms from above and
    equals them when x Ex and y Ey never have opposite signs."""
    rng = np.random.default_rng(5)
    h, w = 9, 12
    Ex, Ey, Et = (rng.standard_normal((h, w)) for _ in range(3))
    cx, cy = 5.5, 4.0
    s, a = oracle.sums(Ex, Ey, Et, cx, cy)
    x = np.arange(w)[None, :] + 0.5 - cx
    y = np.arange(h)[:, None] + 0.5 - cy
    G = x * Ex + y * Ey
    Gm = np.abs(x * Ex) + np.abs(y * Ey)
    for k, t in ((0, Ex * Ex), (1, Ex * Ey), (2, Ey * Ey), (6, Ex * Et), (7, Ey * Et), (9, Et * Et)):
        assert a[k] == pytest.approx(np.abs(t).sum(), rel=1e-13)
    for k, g, e in ((3, G, Ex), (4, G, Ey), (5, G, G), (8, G, Et)):
        assert a[k] >= np.abs(g * e).sum() * (1 - 1e-13)
    assert a[5] == pytest.approx((Gm * Gm).sum(), rel=1e-13)
    assert np.all(np.abs(s) <= a * (1 + 1e-13))
    # Ey = 0: G = x Ex, so the scale is |G| itself
    z = np.zeros_like(Ey)
    s0, a0 = oracle.sums(Ex, z, Et, cx, cy)
    assert a0[5] == pytest.approx(s0[5], rel=1e-13)
    assert a0[3] == pytest.approx(np.abs(x * Ex * Ex).sum(), rel=1e-13)


def test_solve_manufactured_Et_recovers_ABC():
    rng = np.random.default_rng(9)
    h, w = 40, 50
    Ex = rng.standard_normal((h, w))
    Ey = rng.standard_normal((h, w))
    cx, cy = (w - 1) / 2.0 + 0.5, (h - 1) / 2.0 + 0.5
    yy, xx = np.meshgrid(np.arange(h) + 0.5 - cy, np.arange(w) + 0.5 - cx, indexing="ij")
    G = xx * Ex + yy * Ey
    A, B, C = 0.37, -1.25, 0.0125
    Et = -(A * Ex + B * Ey + C * G)
    s, _ = oracle.sums(Ex, Ey, Et, cx, cy)
    r = oracle.solve(s, mode=1, level=0)
    assert r["flags"] == 0
    np.testing.assert_allclose([r["A"], r["B"], r["C"]], [A, B, C], rtol=1e-10)
    assert abs(r["ttc"] - 1 / C) < 1e-8 * (1 / C)
    assert abs(r["x0"] + A / C) < 1e-8 and abs(r["y0"] + B / C) < 1e-8
    assert abs(r["resid"]) < 1e-10
    r2 = oracle.solve(s, mode=1, level=3)
    assert abs(r2["x0"] - 8 * r["x0"]) < 1e-9 and abs(r2["y0"] - 8 * r["y0"]) < 1e-9


def test_solve_matches_numpy_and_spd():
    rng = np.random.default_rng(10)
    for _ in range(20):
        V = rng.standard_normal((4, 200)) * np.array([[1.0], [2.0], [30.0], [0.5]])
        M4 = V @ V.T
        s = np.array([M4[0, 0], M4[0, 1], M4[1, 1], M4[0, 2], M4[1, 2], M4[2, 2],
                      M4[0, 3], M4[1, 3], M4[2, 3], M4[3, 3]])
        r = oracle.solve(s, mode=1)
        M = np.array([[s[0], s[1], s[3]], [s[1], s[2], s[4]], [s[3], s[4], s[5]]])
        np.linalg.cholesky(M)  # SPD
        th = np.linalg.solve(M, -s[[6, 7, 8]])
        np.testing.assert_allclose([r["A"], r["B"], r["C"]], th, rtol=1e-10, atol=1e-13)
        # residual identity: sum (A Ex + B Ey + C G + Et)^2 / sum Et^2
        res = np.sum((th @ V[:3] + V[3]) ** 2) / s[9]
        assert abs(r["resid"] - res) < 1e-9
        r0 = oracle.solve(s, mode=0)
        assert abs(r0["C"] + s[8] / s[5]) <= 1e-15 * abs(s[8] / s[5])
        assert r0["A"] == 0.0 and r0["B"] == 0.0


def test_solve_flags():
    s = np.zeros(10)
    assert oracle.solve(s, mode=1)["flags"] & oracle.FLAG_SINGULAR
    assert oracle.solve(s, mode=0)["flags"] & oracle.FLAG_SINGULAR
    s = np.array([1.0, 0, 1.0, 0, 0, 4.0, 0, 0, 0.0, 1.0])       # C = 0
    r = oracle.solve(s, mode=1)
    assert r["flags"] & oracle.FLAG_C_ZERO and math.isinf(r["ttc"]) and math.isnan(r["x0"])
    s = np.array([1.0, 0, 1.0, 0, 0, 4.0, 0, 0, 2.0, 1.0])       # C = -1/2: receding
    r = oracle.solve(s, mode=1)
    assert r["flags"] == oracle.FLAG_RECEDING and r["ttc"] == -2.0


# --------------------------------------------------------------------------- #
# Whole chain on scenes with closed-form answers (Sec. V-A model)
# --------------------------------------------------------------------------- #

@pytest.mark.parametrize("H,W,levels", [(64, 96, 4), (67, 101, 3), (33, 48, 5)])
def test_ramp_scene_exact_ttc_every_level(H, W, levels):
    Z0, speed, f = 10.0, 0.1, float(W)
    fr = scenes.ramp_sequence(H, W, Z0, speed, a=0.8, b=-0.35, c=0.5, f=f, T=2)
    res = oracle.ttc_pair(fr[0], fr[1], levels=levels, mode=0)
    expect = speed / (Z0 - 0.5 * speed)            # W / Z at t + 1/2
    for l in range(levels):
        assert res[l]["flags"] == 0
        assert abs(res[l]["C"] - expect) <= 1e-12 * expect, (l, res[l]["C"], expect)
    # FOE is not identifiable on a ramp: Ex, Ey constant -> singular 3x3
    resf = oracle.ttc_pair(fr[0], fr[1], levels=levels, mode=1)
    assert all(r["flags"] & oracle.FLAG_SINGULAR for r in resf)


def test_ramp_half_pixel_centre_error_would_fail():
    """A half-pixel error in the cube centre breaks the ramp's exact TTC.

    (The ramp cannot tell the level-l centre (W - 2^l)/2^(l+1) from (W_l - 1)/2:
    the cube grid is symmetric about the latter, which makes both exact; the FOE
    test below pins that choice.)
    """
    H, W = 67, 101
    fr = scenes.ramp_sequence(H, W, 10.0, 0.1, 0.8, -0.35, 0.5, float(W))
    a, b = oracle.downsample(fr[0]), oracle.downsample(fr[1])
    Ex, Ey, Et = oracle.derivatives(a, b)
    good_cx, good_cy = (W - 2) / 4.0, (H - 2) / 4.0
    sg, _ = oracle.sums(Ex, Ey, Et, good_cx, good_cy)
    sb, _ = oracle.sums(Ex, Ey, Et, good_cx + 0.5, good_cy + 0.5)
    expect = 0.1 / (10.0 - 0.05)
    assert abs(-sg[8] / sg[5] - expect) < 1e-12 * expect
    assert abs(-sb[8] / sb[5] - expect) > 1e-6 * expect


def test_level_centre_convention_via_foe():
    """Odd sizes (W = 16*24 + 15): FOE per level stays on the ground truth.

    Level l drops r = W mod 2^l columns; centring level l at (W_l - 1)/2 instead
    of (W - 2^l)/2^(l+1) would move the FOE by r/2 level-0 pixels (1.5 px at l=2,
    3.5 px at l=3), well outside the tolerances below.
    """
    tol = [0.3, 0.3, 0.6, 1.5]
    for seed in (0, 1):
        sc = scenes.fronto_parallel_scene(H=16 * 16 + 15, W=16 * 24 + 15, seed=seed, Z0=10.0,
                                          speed=0.05, pmin=64, pmax=160, m=12)
        sc.T = np.array([0.012, -0.008, 0.05])
        E0 = scenes.render(sc, 0.0).double().numpy()
        E1 = scenes.render(sc, 1.0).double().numpy()
        gt, fx, fy = scenes.ground_truth(sc, 0.5)
        r = oracle.ttc_pair(E0, E1, levels=4, mode=1)
        for l in range(4):
            assert r[l]["flags"] == 0
            assert abs(r[l]["x0"] - fx) < tol[l], (seed, l, r[l]["x0"], fx)
            assert abs(r[l]["y0"] - fy) < tol[l], (seed, l, r[l]["y0"], fy)
        for l in (2, 3):
            assert ((16 * 24 + 15) % 2 ** l) / 2.0 > 2 * tol[l]


def test_invariances_on_textured_plane():
    sc = scenes.tilted_plane_scene(H=48, W=64, seed=3, quantize=False, m=16, pmin=6, pmax=24)
    E0 = scenes.render(sc, 0.0).double().numpy()
    E1 = scenes.render(sc, 1.0).double().numpy()
    base = oracle.ttc_pair(E0, E1, levels=2, mode=1)
    # brightness: E -> 2E + 0.3 leaves A, B, C unchanged
    br = oracle.ttc_pair(2 * E0 + 0.3, 2 * E1 + 0.3, levels=2, mode=1)
    for k in ("A", "B", "C"):
        np.testing.assert_allclose(br[k], base[k], rtol=1e-9)
    # time reversal negates A, B, C; FOE unchanged
    tr = oracle.ttc_pair(E1, E0, levels=2, mode=1)
    for k in ("A", "B", "C"):
        np.testing.assert_allclose(tr[k], -base[k], rtol=1e-9)
    np.testing.assert_allclose(tr["x0"], base["x0"], rtol=1e-9)
    # mirror in x: x0 -> -x0
    mi = oracle.ttc_pair(E0[:, ::-1], E1[:, ::-1], levels=2, mode=1)
    np.testing.assert_allclose(mi["x0"], -base["x0"], rtol=1e-9)
    np.testing.assert_allclose(mi["y0"], base["y0"], rtol=1e-9)
    np.testing.assert_allclose(mi["C"], base["C"], rtol=1e-9)
    # transpose: x0 <-> y0
    tp = oracle.ttc_pair(E0.T.copy(), E1.T.copy(), levels=2, mode=1)
    np.testing.assert_allclose(tp["x0"], base["y0"], rtol=1e-9)
    np.testing.assert_allclose(tp["y0"], base["x0"], rtol=1e-9)


def test_fronto_parallel_ttc_close_to_ground_truth():
    """Smooth texture, small motion: the estimate is within a few percent of Z/W."""
    sc = scenes.fronto_parallel_scene(H=96, W=96, seed=11, Z0=10.0, speed=0.05, pmin=24, pmax=48)
    E0 = scenes.render(sc, 4.0).double().numpy()
    E1 = scenes.render(sc, 5.0).double().numpy()
    gt, fx, fy = scenes.ground_truth(sc, 4.5)
    r0 = oracle.ttc_pair(E0, E1, levels=1, mode=0)[0]
    assert abs(r0["ttc"] - gt) < 0.03 * gt
    r1 = oracle.ttc_pair(E0, E1, levels=1, mode=1)[0]
    assert abs(r1["ttc"] - gt) < 0.05 * gt
    assert abs(r1["x0"] - fx) < 3.0 and abs(r1["y0"] - fy) < 3.0


def test_ttc_bias_converges_quadratically_in_speed():
    """Sec. V-A estimates from two frames with the stencils centred at t + 1/2: the error
    against the closed-form Z/W has a spatial floor (texture sampling) plus a part that
    shrinks with the squared per-frame motion, so successive differences of the
    relative bias between speeds W, W/2, W/4, ... fall by about 4 (a stamp at t instead
    of t + 1/2 leaves a first-order term: the ratios fall towards 2)."""
    for pmin, pmax in ((24, 48), (16, 32)):
        bias = []
        for W in (0.4, 0.2, 0.1, 0.05, 0.025):
            sc = scenes.fronto_parallel_scene(H=96, W=96, seed=11, Z0=10.0, speed=W, pmin=pmin, pmax=pmax)
            E0 = scenes.render(sc, 4.0).double().numpy()
            E1 = scenes.render(sc, 5.0).double().numpy()
            gt, _, _ = scenes.ground_truth(sc, 4.5)
            bias.append((oracle.ttc_pair(E0, E1, levels=1, mode=0)[0]["ttc"] - gt) / gt)
        d = np.diff(bias)
        assert np.all(d > 0), bias
        ratios = d[:-1] / d[1:]
        assert np.all((ratios > 2.8) & (ratios < 4.6)), ratios


def test_multiscale_rule_golden():
    for case in _golden("multiscale_rule.json")["cases"]:
        L = len(case["ttc"])
        r = np.zeros(L, dtype=oracle.RESULT_DTYPE)
        r["ttc"] = case["ttc"]
        r["resid"] = case["resid"]
        r["flags"] = case["flags"]
        r["level"] = np.arange(L)
        assert oracle.select_level(r, 0) == case["rule0"], case
        assert oracle.select_level(r, 1) == case["rule1"], case


def test_ttc_pair_rejects_too_deep():
    E = np.zeros((8, 8))
    with pytest.raises(ValueError):
        oracle.ttc_pair(E, E, levels=4)
    oracle.ttc_pair(E, E, levels=3)
