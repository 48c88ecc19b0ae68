"""Coefficients of the arctangent polynomial in ttc.cu (gradient direction, Sec. II).

atan(t) on [0, 1] is approximated as t * P(t^2) with P of degree 8; the coefficients are
the discrete minimax (Chebyshev) fit over 4000 Chebyshev points, solved as a linear
programme (minimise e subject to |atan(t_i) - t_i P(t_i^2)| <= e), then rounded to FP32.
The script prints the coefficients and the error of the FP32 evaluation (Horner with
fused multiply-adds, emulated in float64 with one rounding per step) over 10^6 points.

    python paper_1612_08825_gb300/csrc/fit_atan.py
"""
import numpy as np
from scipy.optimize import linprog

DEGREE = 8
SCALE = 1e6          # the LP solver's tolerances are absolute: fit the error in micro-units


def fit(deg=DEGREE, n=4000):
    t = np.cos(np.linspace(0.0, np.pi, n)) * 0.5 + 0.5
    s = t * t
    A = np.stack([t * s ** k for k in range(deg + 1)], axis=1) * SCALE
    f = np.arctan(t) * SCALE
    m = deg + 1
    obj = np.zeros(m + 1)
    obj[-1] = 1.0
    A_ub = np.vstack([np.hstack([A, -np.ones((n, 1))]), np.hstack([-A, -np.ones((n, 1))])])
    b_ub = np.concatenate([f, -f])
    r = linprog(obj, A_ub=A_ub, b_ub=b_ub, bounds=[(None, None)] * m + [(0, None)], method="highs")
    if not r.success:
        raise RuntimeError(r.message)
    return r.x[:m], r.x[-1] / SCALE


def eval_fp32(c32, t):
    """t * P(t^2) as the kernel evaluates it: s = t*t rounded, Horner by fused
    multiply-adds (one rounding each), final product rounded."""
    t = t.astype(np.float32)
    s = (t.astype(np.float64) * t).astype(np.float32)
    p = np.full_like(t, c32[-1])
    for k in range(len(c32) - 2, -1, -1):
        p = (p.astype(np.float64) * s + np.float64(c32[k])).astype(np.float32)
    return (p.astype(np.float64) * t).astype(np.float32)


def main():
    c, e = fit()
    c32 = c.astype(np.float32)
    t = np.linspace(0.0, 1.0, 1000001)
    err = np.max(np.abs(eval_fp32(c32, t).astype(np.float64) - np.arctan(t.astype(np.float32).astype(np.float64))))
    print(f"degree {DEGREE}: minimax error {e:.3e}, FP32 evaluation error {err:.3e}")
    for k, v in enumerate(c32):
        print(f"c{k} = {float(v):.9e}f")


if __name__ == "__main__":
    main()
