"""Coefficients of the branch-free atan2 used by the inverse-product epilogue.

atan(a) for a in [0, 1] is written a * P(a^2), P of degree DEG.  P is the
least-squares fit of atan(sqrt(t)) / sqrt(t) on Chebyshev nodes of [0, 1]
(numpy, float64).  Run to print the coefficients (highest degree first, for
Horner's rule) and the float32 maximum absolute error of a * P(a^2) over a
dense grid of [0, 1].
"""
import numpy as np

DEG = 8


def fit(deg=DEG, nodes=4000):
    k = np.arange(nodes)
    t = 0.5 * (1 - np.cos(np.pi * (k + 0.5) / nodes))          # Chebyshev nodes on [0, 1]
    f = np.where(t > 0, np.arctan(np.sqrt(t)) / np.sqrt(np.maximum(t, 1e-300)), 1.0)
    coef = np.polynomial.polynomial.polyfit(t, f, deg)        # monomial basis in t
    return coef[::-1]


def eval_f32(c, a):
    a = a.astype(np.float32)
    t = a * a
    p = np.float32(c[0])
    for ci in c[1:]:
        p = (p * t + np.float32(ci)).astype(np.float32)
    return (a * p).astype(np.float32)


if __name__ == "__main__":
    c = fit()
    a = np.linspace(0, 1, 2_000_001)
    err = np.max(np.abs(eval_f32(c, a).astype(np.float64) - np.arctan(a)))
    print("coefficients (Horner order):")
    for ci in c:
        print(f"  {np.float32(ci)!r}")
    print(f"max |error| in float32 on [0,1]: {err:.3e}")
