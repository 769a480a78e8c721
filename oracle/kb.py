"""Kaiser-Bessel interpolation kernel (test infrastructure, FP64).

The paper names a "potentially non-uniform" Fourier operator (Sec. 2.1, Eq. (1))
and gives no interpolation kernel; the kernel family, width W and oversampling
sigma are the configuration's.  The shape parameter follows Beatty et al. 2005:
beta = pi * sqrt((W/sigma)^2 (sigma - 1/2)^2 - 0.8).
"""
from __future__ import annotations

import math

import numpy as np


def i0(z):
    """Modified Bessel function I0 by its power series sum_m (z/2)^(2m) / (m!)^2.

    All terms are positive, so the partial sums carry no cancellation; terms are
    added until they fall below 1e-18 of the running sum.
    """
    z = np.asarray(z, dtype=np.float64)
    q = (z * 0.5) ** 2
    term = np.ones_like(z)
    total = np.ones_like(z)
    m = 0
    while True:
        m += 1
        term = term * q / (m * m)
        total = total + term
        if np.all(term <= 1e-18 * total):
            break
    return total


def beta(W: int, sigma: float) -> float:
    return math.pi * math.sqrt((W / sigma) ** 2 * (sigma - 0.5) ** 2 - 0.8)


def phi(t, W: int, b: float):
    """phi(t) = I0(b*sqrt(1 - (2t/W)^2)) for |t| <= W/2, else 0."""
    t = np.asarray(t, dtype=np.float64)
    s = 1.0 - (2.0 * t / W) ** 2
    inside = s >= 0.0
    out = np.zeros_like(t)
    out[inside] = i0(b * np.sqrt(s[inside]))
    return out


def phihat(nu, W: int, b: float):
    """Continuous Fourier transform of phi at frequency nu (cycles per grid step):
    int phi(t) exp(2 pi i nu t) dt = W sinh(r)/r, r = sqrt(b^2 - (pi W nu)^2),
    with the sin form when the radicand is negative."""
    nu = np.asarray(nu, dtype=np.float64)
    r2 = b * b - (math.pi * W * nu) ** 2
    out = np.empty_like(nu)
    pos = r2 > 1e-300
    neg = r2 < -1e-300
    zero = ~(pos | neg)
    r = np.sqrt(r2[pos])
    out[pos] = W * np.sinh(r) / r
    rn = np.sqrt(-r2[neg])
    out[neg] = W * np.sin(rn) / rn
    out[zero] = W
    return out
