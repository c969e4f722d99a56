"""Kaiser-Bessel interpolation kernel and grid correction, FP64 (oracle).

The paper's NUFFT follows Fessler & Sutton (2003) without fixing the kernel
(Section 2, Eq. 3; Section 3.2, Eq. 6).  The reading used here: a Kaiser-Bessel
kernel of J taps, shape parameter beta = 2.34 J (the Fessler-Sutton choice for
oversampling 2), and a grid correction equal to the reciprocal of the kernel's
continuous Fourier transform at each image pixel.
"""
from __future__ import annotations

import math

import numpy as np


def i0(x):
    """Modified Bessel function I0 by its power series sum_k (x^2/4)^k / (k!)^2."""
    x = np.asarray(x, dtype=np.float64)
    q = 0.25 * x * x
    term = np.ones_like(q)
    total = np.ones_like(q)
    for k in range(1, 200):
        term = term * q / (k * k)
        total = total + term
        if np.all(term <= 1e-18 * total):
            break
    return total


def default_beta(J: int) -> float:
    return 2.34 * J


def kb(t, J: int, beta: float):
    """KB(t) = I0(beta sqrt(1 - (2t/J)^2)) / I0(beta) for |t| <= J/2, else 0."""
    t = np.asarray(t, dtype=np.float64)
    r = 1.0 - (2.0 * t / J) ** 2
    inside = r >= 0.0
    val = i0(beta * np.sqrt(np.where(inside, r, 0.0))) / i0(beta)
    return np.where(inside, val, 0.0)


def kb_hat(nu, J: int, beta: float):
    """Continuous Fourier transform of KB at frequency nu (cycles per grid cell).

    int KB(t) e^{-2 pi i nu t} dt = J sinh(sqrt(beta^2 - (pi J nu)^2))
                                     / (I0(beta) sqrt(beta^2 - (pi J nu)^2)),
    continued analytically (sinh -> sin) where (pi J nu)^2 > beta^2.
    """
    nu = np.asarray(nu, dtype=np.float64)
    a2 = beta * beta - (math.pi * J * nu) ** 2
    out = np.empty_like(a2)
    pos = a2 > 1e-12
    neg = a2 < -1e-12
    mid = ~(pos | neg)
    s = np.sqrt(np.abs(a2))
    out[pos] = np.sinh(s[pos]) / s[pos]
    out[neg] = np.sin(s[neg]) / s[neg]
    out[mid] = 1.0
    return J * out / i0(beta)


def grid_correction_1d(n: int, J: int, beta: float) -> np.ndarray:
    """1 / KB_hat(j_c / (2n)) for pixel j in [0, n), j_c = j - n/2 (oversampling 2)."""
    jc = np.arange(n) - n // 2
    return 1.0 / kb_hat(jc / (2.0 * n), J, beta)


def kb_taps(phi, J: int, beta: float) -> np.ndarray:
    """The J interpolation weights of a sample at fractional offset phi in [0, 1).

    Weight i multiplies grid cell floor(u~ - J/2) + 1 + i, whose distance to the
    sample is u~ - cell = phi + J/2 - 1 - i.
    """
    phi = np.asarray(phi, dtype=np.float64)
    i = np.arange(J)
    return kb(phi[..., None] + J / 2.0 - 1.0 - i, J, beta)
