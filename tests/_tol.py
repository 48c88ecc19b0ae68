"""Tolerances for the TTC parity tests, derived from the arithmetic.

Sums: the CUDA path forms products in FP32 and sums them pairwise in FP32 (per-
thread runs of at most 32 terms, a 16-way strided sum, a 16-lane tree) before an
FP64 merge.  The textbook bound for such a sum is about (32 + 16 + 4) u |terms|
with u = 2^-24 (~3.1e-6 of the absolute sum), plus the FP32 rounding of the
derivative values for float frames and of G (a few u per term).  SUM_REL = 1e-5 of
the oracle's sum of |terms| covers the bound with a margin of about 3.

Solve: the first-order perturbation of M theta = b is
    d theta = M^-1 (d b - d M theta),
so |d theta| <= |M^-1| (|d b| + |d M| |theta|) componentwise, with |d s_k| bounded
by SUM_REL * abssum_k.  TTC = 1/C and x0 = -2^l A / C follow by the chain rule.
A factor of 2 covers second-order terms.
"""
import numpy as np

SUM_REL = 1e-5


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
