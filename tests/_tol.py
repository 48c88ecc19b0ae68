"""Tolerances for the TTC parity tests, derived from the arithmetic.

Sums, uint8 frames.  Ex, Ey, Et are exact integers in FP32 (the pyramid levels are
exact integer block sums), and so are the cube coordinates x, y (half-integers).
The rounding errors are:
  - G = x Ex + y Ey: one rounding of y Ey and one of the fused multiply-add, so
    |g - G| <= 2u (|x Ex| + |y Ey|); a G^2 term carries twice that;
  - the products enter fused multiply-adds, so each term is rounded only as part of
    its sum: per-thread runs of at most 32 terms, the fold of the two packed lanes
    (1), a 16-way strided sum (16) and a 16-lane tree (4) before the FP64 merge, at
    most 53 roundings on any term's path.
With u = 2^-24 the error of sum k is at most (53 + 4) u * abssum_k, where abssum_k is
the oracle's error scale: the sum of |term|, with |G| replaced by |x Ex| + |y Ey| in
the four G terms.  57 u = 3.40e-6; SUM_REL = 3.5e-6.

Sums, float32 frames.  The stencil values themselves carry the rounding of pixel
sums and differences (three roundings, relative to the pixel magnitudes rather than
to the derivatives), and the pyramid levels are rounded block sums, so no bound of
the form above holds; SUM_REL_F32 = 1e-5 is the tolerance stated for them.

Solve: the first-order perturbation of M theta = b is
    d theta = M^-1 (d b - d M theta),
so |d theta| <= |M^-1| (|d b| + |d M| |theta|) componentwise, with |d s_k| bounded
by rel * abssum_k.  TTC = 1/C and x0 = -2^l A / C follow by the chain rule.
A factor of 2 covers second-order terms.
"""
import numpy as np

SUM_REL = 3.5e-6
SUM_REL_F32 = 1e-5


def sums_close(got, ref, rel=SUM_REL):
    """Per-sum check |got - ref| <= rel * abssum (+ tiny absolute floor)."""
    g = np.asarray(got["sums"], dtype=np.float64)
    r = np.asarray(ref["sums"], dtype=np.float64)
    a = np.asarray(ref["abssums"], dtype=np.float64)
    err = np.abs(g - r)
    bound = rel * a + 1e-300
    return bool(np.all(err <= bound)), float(np.max(err / np.maximum(a, 1e-300)))


def solve_bounds(ref, mode, level, rel=SUM_REL):
    """Componentwise bounds on (A, B, C, ttc, x0, y0) from the sum bounds."""
    s = np.asarray(ref["sums"], dtype=np.float64)
    ds = rel * np.asarray(ref["abssums"], dtype=np.float64)
    A, B, C = float(ref["A"]), float(ref["B"]), float(ref["C"])
    if mode == 0:
        dC = (ds[8] + abs(C) * ds[5]) / s[5]
        dA = dB = 0.0
    else:
        M = np.array([[s[0], s[1], s[3]], [s[1], s[2], s[4]], [s[3], s[4], s[5]]])
        dM = np.array([[ds[0], ds[1], ds[3]], [ds[1], ds[2], ds[4]], [ds[3], ds[4], ds[5]]])
        db = np.array([ds[6], ds[7], ds[8]])
        th = np.array([A, B, C])
        Mi = np.abs(np.linalg.inv(M))
        d = Mi @ (db + dM @ np.abs(th))
        dA, dB, dC = (float(v) for v in d)
    dA, dB, dC = 2 * dA, 2 * dB, 2 * dC
    sc = 2.0 ** level
    dttc = dC / (C * C)
    dx0 = sc * (dA / abs(C) + abs(A) * dC / (C * C))
    dy0 = sc * (dB / abs(C) + abs(B) * dC / (C * C))
    return {"A": dA, "B": dB, "C": dC, "ttc": dttc, "x0": dx0, "y0": dy0}


def check_record(got, ref, mode, level, rel=SUM_REL):
    """Assert one GPU record agrees with the oracle record; returns max sum error."""
    ok, worst = sums_close(got, ref, rel)
    assert ok, f"level {level}: sums differ (worst {worst:.3e} of abssum)"
    assert int(got["flags"]) == int(ref["flags"]), (level, int(got["flags"]), int(ref["flags"]))
    assert int(got["n"]) == int(ref["n"]) and int(got["level"]) == level
    if int(ref["flags"]) & 1:
        for k in ("A", "B", "C", "ttc", "x0", "y0"):
            assert np.isnan(got[k])
        return worst
    b = solve_bounds(ref, mode, level, rel)
    for k in ("A", "B", "C", "ttc", "x0", "y0"):
        g, r = float(got[k]), float(ref[k])
        if np.isnan(r) or np.isinf(r):
            assert (np.isnan(g) and np.isnan(r)) or g == r, (k, g, r)
            continue
        assert abs(g - r) <= b[k] + 1e-12 * abs(r), f"level {level} {k}: {g} vs {r} (bound {b[k]:.3e})"
    return worst
