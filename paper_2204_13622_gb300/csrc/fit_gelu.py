"""Coefficients of the inference kernel's GELU (csrc/fcc_mlp.cu, gelu_fast).

GELU(x) = x Phi(x) = max(x, 0) - t Phi(-t) with t = |x|, and
Phi(-t) = exp(-t^2 / 2) S(t), where S(t) = Phi(-t) exp(t^2 / 2) is smooth and
slowly varying (S(0) = 1/2, S(t) ~ 1 / (t sqrt(2 pi)) for large t).  S is fitted
as a polynomial of degree 7 in u = 1 / (1 + A t) by least squares on Chebyshev
points of u over t in [0, T_MAX]; beyond T_MAX the kernel clamps t (the term
t Phi(-t) is below 1e-11 there).  Run: python fit_gelu.py  (prints the monomial
coefficients c0..c7 of S in u and the error of GELU evaluated in FP32).
"""
import numpy as np
from scipy.special import erfc

A, T_MAX, DEG = 0.3, 7.0, 7


def fit():
    u_lo = 1.0 / (1.0 + A * T_MAX)
    k = np.arange(4096)
    # Chebyshev points of the u interval [u_lo, 1]
    u = u_lo + (1.0 - u_lo) * 0.5 * (1.0 - np.cos(np.pi * (k + 0.5) / k.size))
    t = (1.0 / u - 1.0) / A
    S = 0.5 * erfc(t / np.sqrt(2.0)) * np.exp(0.5 * t * t)
    V = np.vander(u, DEG + 1, increasing=True)
    c, *_ = np.linalg.lstsq(V, S, rcond=None)
    return c


def gelu_fp32(x, c):
    """The kernel's evaluation order, in FP32."""
    f = np.float32
    x = x.astype(f)
    t = np.minimum(np.abs(x), f(T_MAX))
    u = (f(1.0) / (f(A) * t + f(1.0))).astype(f)
    s = np.full_like(x, f(c[DEG]))
    for j in range(DEG - 1, -1, -1):
        s = (s * u + f(c[j])).astype(f)
    e = np.exp2((t * f(-0.5 / np.log(2.0))) * t).astype(f)
    return (np.maximum(x, f(0.0)) - (t * e) * s).astype(f)


if __name__ == "__main__":
    c = fit()
    for j, v in enumerate(c):
        print(f"c{j} = {v:.9e}f")
    x = np.linspace(-12.0, 12.0, 2_000_001)
    exact = 0.5 * x * erfc(-x / np.sqrt(2.0))
    err = np.abs(gelu_fp32(x, c).astype(np.float64) - exact)
    print(f"max |GELU error| on [-12, 12]: {err.max():.3e}; "
          f"relative to max(1, |x|): {(err / np.maximum(1.0, np.abs(x))).max():.3e}")
