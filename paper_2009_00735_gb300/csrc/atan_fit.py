"""Coefficients of the odd polynomial atan(t) ~ t * P(t^2) on [0, 1] used by
the refinement kernels (indexing.cu, atan01).

P has degree 7 in s = t^2.  The coefficients minimise the maximum absolute
error on [0, 1] by Lawson's algorithm (iteratively reweighted least squares,
whose weights converge to the minimax solution).  Run this file to print the
coefficients and the error bounds (exact arithmetic and FP32 Horner
evaluation); tests/test_atan_poly_cpu.py checks the constants in indexing.cu
against np.arctan.
"""
import numpy as np


def fit(deg: int = 7, iters: int = 3000):
    x = np.linspace(0.0, 1.0, 20001)[1:]
    y = np.arctan(x)
    A = np.stack([x * x ** (2 * j) for j in range(deg + 1)], 1)
    w = np.full_like(x, 1.0 / x.size)
    best = None
    for _ in range(iters):
        sw = np.sqrt(w)
        c, *_ = np.linalg.lstsq(A * sw[:, None], y * sw, rcond=None)
        e = np.abs(A @ c - y)
        if best is None or e.max() < best[1]:
            best = (c, e.max())
        w = w * e
        w /= w.sum()
    return best[0]


if __name__ == "__main__":
    c = fit()
    xx = np.linspace(0.0, 1.0, 2000001)
    print("max |error| exact:", np.abs(xx * np.polyval(c[::-1], xx * xx) - np.arctan(xx)).max())
    for v in c:
        print(f"{v:.9e}f")
