"""Plug-and-play outer loops (test infrastructure, FP64).

PnP-HQS (Sec. 3.3):   u_k = prox^P_{gamma_k f}(x_k);  x_{k+1} = D_{sigma_k}(u_k)
PnP-PGD (Sec. 3.3):   u_k = x_k - gamma P grad f(x_k);  x_{k+1} = D_sigma(u_k)

with f(x) = 1/2 sum_l ||F S_l x - y_l||^2 (Sec. 2.2, Eq. (2)), so grad f(x) =
A^H A x - A^H y.  The P-metric prox of Sec. 3.4 solves
    (gamma A^H A + P) u = gamma A^H y + P x,   P = c0 I + c1 A^H A,
P = Id: (c0, c1) = (1, 0); "F-1": (2, -alpha); Chebyshev: (4, -10 alpha / 3).
Dividing by gamma = 1/mu gives the data-consistency system used here,
    ((1 + c1 mu) A^H A + c0 mu I) u = A^H y + mu (c0 x + c1 A^H A x),
which for P = Id is (A^H A + mu I) u = A^H y + mu x.  It is solved by PCG with
a fixed number of iterations, warm-started at x_k.

The default denoiser is separable complex Gaussian smoothing with periodic
boundaries (a stand-in for the trained prior of Sec. 4.2), on images or volumes.
"""
from __future__ import annotations

import math

import numpy as np

from . import solvers, toeplitz


def prox_coefficients(mu: float, c0: float, c1: float):
    """(a, b) of the data-consistency system a A^H A + b I for step mu = 1/gamma."""
    return 1.0 + c1 * mu, c0 * mu


def gaussian_taps(s: float) -> np.ndarray:
    r = int(math.ceil(3.0 * s))
    i = np.arange(-r, r + 1, dtype=np.float64)
    g = np.exp(-(i * i) / (2.0 * s * s))
    return g / g.sum()


def gaussian_denoise(v, s: float) -> np.ndarray:
    """Separable Gaussian blur (std s pixels, radius ceil(3 s), periodic) of the
    real and imaginary parts of an image or a volume, one axis at a time from
    the last (x) to the first; identity when s < 0.1."""
    v = np.asarray(v, dtype=np.complex128)
    if s < 0.1:
        return v.copy()
    g = gaussian_taps(s)
    r = (len(g) - 1) // 2
    out = v
    for axis in reversed(range(v.ndim)):
        acc = np.zeros_like(v)
        for i, gi in enumerate(g):
            acc += gi * np.roll(out, -(i - r), axis=axis)   # acc[.., n, ..] += g * out[.., n + (i - r), ..]
        out = acc
    return out


def denoiser_std(sigma_k: float, sigma_0: float, kappa: float = 1.5) -> float:
    """Blur width tied to the noise level: s_k = kappa * sigma_k / sigma_0 pixels."""
    return kappa * sigma_k / sigma_0


def hqs(apply_AHA, b0, x0, mu, sigma, K, k0=0, cg_iters=5, c0=1.0, c1=0.0,
        denoiser=None, lam=None, precond_apply=None):
    """Annealed PnP-HQS from iteration k0 to K; returns (x_K, u_{K-1}, history).

    denoiser(u, sigma_k) defaults to gaussian_denoise(u, 1.5*sigma_k/sigma_0)
    with sigma_0 = sigma[0]; lam is the circulant preconditioner symbol (None
    for unpreconditioned CG), applied by precond_apply(v, lam, a, b) (default:
    the 2D one of toeplitz; volumes pass nufft3d.precond_apply)."""
    if precond_apply is None:
        precond_apply = toeplitz.precond_apply
    if denoiser is None:
        s0 = float(sigma[0])
        denoiser = lambda u, sk: gaussian_denoise(u, denoiser_std(sk, s0))
    x = np.array(x0, dtype=np.complex128, copy=True)
    u = x
    hist = []
    for k in range(k0, K):
        a, b = prox_coefficients(float(mu[k]), c0, c1)
        rhs = b0 + mu[k] * c0 * x
        if c1 != 0.0:
            rhs = rhs + mu[k] * c1 * apply_AHA(x)
        H = lambda v, a=a, b=b: a * apply_AHA(v) + b * v
        Minv = None
        if lam is not None:
            Minv = lambda v, a=a, b=b: precond_apply(v, lam, a, b)
        u, _ = solvers.pcg(H, rhs, x, Minv, max_iter=cg_iters, tol=0.0)
        x = denoiser(u, float(sigma[k]))
        hist.append(x.copy())
    return x, u, hist


def pgd(apply_AHA, b0, x0, gamma, sigma, K, c0=1.0, c1=0.0, denoiser=None):
    """PnP-PGD with P = c0 I + c1 A^H A: u = x - gamma P (A^H A x - A^H y); x = D(u)."""
    if denoiser is None:
        s0 = float(sigma[0])
        denoiser = lambda u, sk: gaussian_denoise(u, denoiser_std(sk, s0))
    x = np.array(x0, dtype=np.complex128, copy=True)
    for k in range(K):
        g = apply_AHA(x) - b0
        Pg = c0 * g + (c1 * apply_AHA(g) if c1 != 0.0 else 0.0)
        x = denoiser(x - gamma[k] * Pg, float(sigma[k]))
    return x
