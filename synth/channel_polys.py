"""Derivation of the polynomial coefficients in the channel generator's definition.

The BPSK/AWGN channel draws its noise by Box-Muller from Philox4x32-10 words.  So that
the device and the CPU oracle produce the same binary32 LLRs bit for bit, the generator
is defined down to its binary32 operations.  ln and sin/cos of 2*pi*u are range
reductions plus polynomials whose coefficients are fixed by this script.  Each side
implements the definition independently, with its own copy of the constants.  This
script is neither imported nor run by either side.

Method: minimax fits by Lawson's iteratively reweighted least squares on a dense grid
(C. L. Lawson, "Contributions to the theory of linear least maximum approximation",
PhD thesis, UCLA, 1961), in float64.  The coefficients are then rounded to binary32
one at a time, constant term first, and the higher-degree ones are refitted after
each rounding.

  ln(1 + f) = f + f^2 (-1/2 + f R(f)),   f in [sqrt(1/2) - 1, sqrt(2) - 1],  R of degree 7
  sin(2 pi r) = r S(r^2),                r in [-1/8, 1/8],                    S of degree 4
  cos(2 pi r) = 1 + r^2 C(r^2),          r in [-1/8, 1/8],                    C of degree 4

R minimizes the relative error of ln(1 + f), S that of sin, and C the absolute error of cos.

Run:  python -m synth.channel_polys   (prints the constants as hexadecimal float literals)
"""
from __future__ import annotations

import numpy as np


def _lawson(basis: np.ndarray, target: np.ndarray, weight: np.ndarray, iters: int = 400) -> np.ndarray:
    """Coefficients c minimizing max_i weight_i |basis_i . c - target_i| (Lawson's algorithm)."""
    u = np.full(len(target), 1.0 / len(target))
    c = None
    for _ in range(iters):
        sw = np.sqrt(u) * weight
        c, *_ = np.linalg.lstsq(basis * sw[:, None], target * sw, rcond=None)
        e = np.abs(basis @ c - target) * weight
        u = u * e
        u /= u.sum()
    return c


def _fit_rounded(x: np.ndarray, target_of, basis_of, weight: np.ndarray, deg: int):
    """Fit, round the leading coefficient to binary32, refit the rest with it fixed, and so on."""
    fixed: list[float] = []
    for k in range(deg + 1):
        B = basis_of(x, deg)
        t = target_of(x) - (B[:, :k] @ np.array(fixed) if k else 0.0)
        c = _lawson(B[:, k:], t, weight)
        fixed.append(float(np.float32(c[0])))
    return np.array(fixed)


def fit_ln(deg: int = 7):
    lo, hi = np.sqrt(0.5) - 1.0, np.sqrt(2.0) - 1.0
    f = np.cos(np.linspace(np.pi, 0.0, 40001)) * (hi - lo) / 2 + (hi + lo) / 2
    f = f[f != 0.0]
    # R(f) = (ln(1+f) - f + f^2/2) / f^3; the result's error is f^3 dR, relative to ln(1+f)
    target = lambda x: (np.log1p(x) - x + 0.5 * x * x) / x**3
    basis = lambda x, d: np.stack([x**i for i in range(d + 1)], axis=1)
    weight = np.abs(f**3 / np.log1p(f))
    return _fit_rounded(f, target, basis, weight, deg)


def fit_sin(deg: int = 4):
    r = np.linspace(1e-6, 0.125, 20001)
    z = r * r
    target = lambda x: np.sin(2 * np.pi * np.sqrt(x)) / np.sqrt(x)
    basis = lambda x, d: np.stack([x**i for i in range(d + 1)], axis=1)
    return _fit_rounded(z, target, basis, np.ones_like(z), deg)


def fit_cos(deg: int = 4):
    r = np.linspace(1e-6, 0.125, 20001)
    z = r * r
    target = lambda x: (np.cos(2 * np.pi * np.sqrt(x)) - 1.0) / x
    basis = lambda x, d: np.stack([x**i for i in range(d + 1)], axis=1)
    return _fit_rounded(z, target, basis, z, deg)


def main():
    for name, c in (("ln R", fit_ln()), ("sin S", fit_sin()), ("cos C", fit_cos())):
        print(name, ", ".join(float(np.float32(v)).hex() for v in c[::-1]), "(highest degree first)")


if __name__ == "__main__":
    main()
