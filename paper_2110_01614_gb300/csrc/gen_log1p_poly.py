"""Derives the polynomial the tensor-core epilogue uses for log1p.

softplus_beta(z) = max(z, 0) + log1p(u) / beta with u = exp(-beta |z|) in (0, 1].
The kernel evaluates log1p(u) = u * P(u), where P approximates log1p(u) / u on
[0, 1] (so the error is relative to log1p(u), also for tiny u).  P is the
Chebyshev interpolant of log1p(u)/u at the Chebyshev points of [0, 1]
(near-minimax), expanded to monomial coefficients for Horner evaluation in
FP32.  Run this script to print the coefficients and the worst relative error
over a dense grid; the kernel's constants are its output.
"""

import numpy as np


def fit(degree):
    k = np.arange(degree + 1)
    x = 0.5 + 0.5 * np.cos(np.pi * (k + 0.5) / (degree + 1))   # Chebyshev points on [0, 1]
    y = np.log1p(x) / x
    cheb = np.polynomial.chebyshev.Chebyshev.fit(x, y, degree, domain=[0.0, 1.0])
    return cheb.convert(kind=np.polynomial.Polynomial, domain=[0.0, 1.0], window=[0.0, 1.0]).coef


def max_rel_error(coef, n=200001):
    u = np.linspace(1e-12, 1.0, n)
    p = np.zeros_like(u, dtype=np.float32)
    for c in coef[::-1]:
        p = (p * u.astype(np.float32) + np.float32(c)).astype(np.float32)
    approx = u * p.astype(np.float64)
    return float(np.max(np.abs(approx - np.log1p(u)) / np.log1p(u)))


if __name__ == "__main__":
    for d in (5, 6, 7):
        c = fit(d)
        print(d, max_rel_error(c), ", ".join(f"{v:.9e}f" for v in c))
