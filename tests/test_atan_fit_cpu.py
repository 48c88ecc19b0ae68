"""The gradient kernel's arctangent (Sec. II, Eq. Eangle): its polynomial coefficients in
csrc/ttc.cu come from csrc/fit_atan.py, their FP32 evaluation stays within 1e-7 of atan
on [0, 1], and the octant reduction, emulated in FP32 step by step, stays within the
5e-7 rad the GPU test uses against FP64 atan2 on exact (Ex, Ey) pairs."""
import importlib.util
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1612_08825_gb300", "csrc")


def _fit_module():
    pytest.importorskip("scipy")
    spec = importlib.util.spec_from_file_location("fit_atan", os.path.join(CSRC, "fit_atan.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _kernel_coefficients():
    src = open(os.path.join(CSRC, "ttc.cu")).read()
    body = src[src.index("float atan2_poly(float y, float x)"):]
    body = body[body.index("float p = "):body.index("float r = p * t;")]
    vals = [float(v) for v in re.findall(r"([-+]?\d\.\d+e[-+]\d+)f", body)]
    # Horner order: c8 first, c0 last
    return np.array(vals[::-1], dtype=np.float32)


def test_kernel_coefficients_are_the_fit():
    fa = _fit_module()
    c = _kernel_coefficients()
    assert len(c) == fa.DEGREE + 1
    fresh, e = fa.fit()
    assert e < 1e-8
    np.testing.assert_allclose(c.astype(np.float64), fresh, rtol=0, atol=1e-6)
    t = np.linspace(0.0, 1.0, 200001)
    err = np.abs(fa.eval_fp32(c, t).astype(np.float64) - np.arctan(t.astype(np.float32).astype(np.float64)))
    assert err.max() < 1e-7


def _atan2_fp32(y, x, c):
    """The kernel's steps in FP32 (one rounding per operation, fused multiply-adds); t is
    taken correctly rounded here, the kernel's corrected quotient is within about half
    an ulp of it."""
    f32 = np.float32
    ax, ay = np.abs(x), np.abs(y)
    mx, mn = np.maximum(ax, ay), np.minimum(ax, ay)
    with np.errstate(invalid="ignore", divide="ignore"):
        t = np.where(mx > 0, (mn.astype(np.float64) / mx).astype(f32), f32(0))
    s = (t.astype(np.float64) * t).astype(f32)
    p = np.full_like(t, c[-1])
    for k in range(len(c) - 2, -1, -1):
        p = (p.astype(np.float64) * s + np.float64(c[k])).astype(f32)
    r = (p.astype(np.float64) * t).astype(f32)
    r = np.where(ay > ax, (np.float64(f32(1.57079632679489662)) - r).astype(f32), r)
    r = np.where(np.signbit(x), (np.float64(f32(3.14159265358979324)) - r).astype(f32), r)
    return np.copysign(r, y)


def test_octant_reduction_within_bound_on_exact_pairs():
    c = _kernel_coefficients()
    # every (Ex, Ey) a uint8 image can give: half-integers in [-255, 255] (subsampled grid)
    v = np.arange(-510, 511, 3, dtype=np.float64) / 2.0
    Y, X = np.meshgrid(v, v, indexing="ij")
    y, x = Y.astype(np.float32).ravel(), X.astype(np.float32).ravel()
    got = _atan2_fp32(y, x, c).astype(np.float64)
    ref = np.arctan2(y.astype(np.float64), x.astype(np.float64))
    d = np.abs(np.angle(np.exp(1j * (got - ref))))
    ok = (x != 0) | (y != 0)
    assert d[ok].max() < 5e-7, d[ok].max()
    # axes, diagonals and the signed zeros
    specials = [(0.0, 1.0, 0.0), (1.0, 0.0, np.pi / 2), (0.0, -1.0, np.pi), (-0.0, -1.0, -np.pi),
                (-1.0, 0.0, -np.pi / 2), (1.0, 1.0, np.pi / 4), (1.0, -1.0, 3 * np.pi / 4),
                (-1.0, -1.0, -3 * np.pi / 4), (0.0, 0.0, 0.0), (0.0, -0.0, np.pi)]
    for yy, xx, want in specials:
        g = float(_atan2_fp32(np.float32([yy]), np.float32([xx]), c)[0])
        assert abs(g - want) < 5e-7, (yy, xx, g, want)
