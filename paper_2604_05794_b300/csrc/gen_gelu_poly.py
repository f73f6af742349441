"""Coefficients of the inference GELU's polynomial (hf_gemm.cu, gelu_poly2).

GELU(x) = x Phi(x), Phi the standard normal CDF.  The kernel clamps x to [-c, c] through
t = sat(x / (2c) + 1/2), forms w8 = 8 t - 4 (= 4 x / c on the clamped range) and q = w8^2 - 8, and
takes Phi = 1/2 + w8 R(q) with R a polynomial of degree M - 1 in q.  This script fits R by
iteratively reweighted least squares (Lawson's method, which converges towards the minimax fit) on
Chebyshev-spaced nodes, rounds the coefficients to FP32, and checks the FP32 evaluation of the
whole sequence (every fused multiply-add rounded once) against x Phi(x) in FP64 over a dense sweep.

    python gen_gelu_poly.py        # prints the C initialiser and the measured bound
"""
import numpy as np
from scipy.special import erf

C = 5.0     # clamp: 1 - Phi(5) = 2.9e-7
M = 13      # coefficients of R


def fit(c=C, m=M, iters=400):
    w8 = 4.0 * np.cos(np.linspace(0.0, np.pi / 2, 60001))
    w8 = w8[w8 > 1e-6]
    y = 0.5 * erf((c * w8 / 4.0) / np.sqrt(2.0))          # Phi - 1/2, odd in w8
    q = w8 * w8 - 8.0
    A = np.vander(q, m, increasing=True) * w8[:, None]
    wt = np.ones_like(y)
    for _ in range(iters):
        coef, *_ = np.linalg.lstsq(A * wt[:, None], y * wt, rcond=None)
        e = A @ coef - y
        wt = wt * (1.0 + np.abs(e) / np.abs(e).max())
        wt /= wt.mean()
    return coef.astype(np.float32)


def _fma(a, b, c):
    # one rounding to FP32 (the product of two FP32 values is exact in FP64)
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(np.float32)


def gelu_fp32(x, coef, c=C):
    """The kernel's operation sequence in FP32."""
    x = np.asarray(x, np.float32)
    t = np.clip(_fma(x, np.float32(1.0 / (2.0 * c)), np.float32(0.5)), 0.0, 1.0).astype(np.float32)
    w8 = _fma(t, np.float32(8.0), np.float32(-4.0))
    q = _fma(w8, w8, np.float32(-8.0))
    r = np.full_like(q, coef[-1])
    for j in range(len(coef) - 2, -1, -1):
        r = _fma(r, q, coef[j])
    phi = _fma(w8, r, np.float32(0.5))
    return (x.astype(np.float64) * phi.astype(np.float64)).astype(np.float32)


def bound(coef, c=C):
    """max |gelu_fp32(x) - x Phi(x)| / |x| over a dense sweep of [-40, 40] and the FP32 values
    around the clamp points."""
    x = np.concatenate([np.linspace(-40.0, 40.0, 8000001), np.linspace(-6.0, 6.0, 4000001)]).astype(np.float32)
    x = x[x != 0]
    xd = x.astype(np.float64)
    ref = 0.5 * xd * (1.0 + erf(xd / np.sqrt(2.0)))
    return float(np.max(np.abs(gelu_fp32(x, coef, c).astype(np.float64) - ref) / np.abs(xd)))


if __name__ == "__main__":
    coef = fit()
    print("constexpr float kGeluC[%d] = {%s};" % (M, ", ".join("%.9ef" % v for v in coef)))
    print("max |error| / |x| = %.3e" % bound(coef))
