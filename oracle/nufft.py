"""Gridding NUFFT with a Kaiser-Bessel kernel (test infrastructure, FP64).

Approximates the multicoil operator of Eq. (1) (Sec. 2.1) with the same kernel
parameters as the GPU path, so that the two can be compared at equal
parameters.  The paper does not describe a NUFFT; the steps below are the
classical gridding construction:

forward (type 2): g = S_l x / (phihat_x phihat_y), placed on the
    sigma-oversampled grid at n mod G; Ghat = FFT_G(g) (unnormalised,
    exp(-2 pi i m n / G)); y[j] = Npix^(-1/2) sum_taps phi(u_j - m) Ghat[m mod G]
    with u_j = k_j G / (2 pi).
adjoint (type 1): H[m mod G] = sum_j y[j] phi(u_j - m);
    V = sum_m H[m] exp(+2 pi i m n / G); x = Npix^(-1/2) sum_l conj(S_l) V / phihat.

Taps: for each point and axis, u is wrapped into [0, G) (u < 0 -> u + G), the
first tap is i0 = ceil(u - W/2), and the W taps are i0 .. i0+W-1 with weights
phi(u - i); grid indices are taken mod G.
"""
from __future__ import annotations

import math

import numpy as np

from . import kb
from .nudft import centred


def grid_size(n: int, sigma: float) -> int:
    G = int(round(sigma * n))
    if abs(G - sigma * n) > 1e-9:
        raise ValueError("sigma * n must be an integer")
    return G


def point_taps(k, G: int, W: int):
    """Per-axis tap origin and offset: u = k*G/(2 pi) wrapped to [0, G),
    i0 = ceil(u - W/2), d = u - i0 (so tap w has weight phi(d - w))."""
    u = (np.asarray(k, dtype=np.float64) * G) / (2.0 * math.pi)
    u = np.where(u < 0.0, u + G, u)
    i0 = np.ceil(u - W / 2.0)
    d = u - i0
    return i0.astype(np.int64), d


def apodisation(n: int, G: int, W: int, b: float):
    """1 / phihat(n_c / G) for the centred pixel coordinates n_c of one axis."""
    return 1.0 / kb.phihat(centred(n) / G, W, b)


def _tap_tables(traj, Gy, Gx, W, b):
    i0x, dx = point_taps(traj[:, 0], Gx, W)
    i0y, dy = point_taps(traj[:, 1], Gy, W)
    w = np.arange(W)
    wx = kb.phi(dx[:, None] - w[None, :], W, b)       # (M, W)
    wy = kb.phi(dy[:, None] - w[None, :], W, b)
    ix = np.mod(i0x[:, None] + w[None, :], Gx)         # (M, W)
    iy = np.mod(i0y[:, None] + w[None, :], Gy)
    return ix, iy, wx, wy


def forward(x, smaps, traj, W: int, sigma: float):
    """A x by gridding; returns (L, M) complex128."""
    x = np.asarray(x, dtype=np.complex128)
    smaps = np.asarray(smaps, dtype=np.complex128)
    traj = np.asarray(traj, dtype=np.float64)
    L, ny, nx = smaps.shape
    Gy, Gx = grid_size(ny, sigma), grid_size(nx, sigma)
    b = kb.beta(W, sigma)
    apx = apodisation(nx, Gx, W, b)
    apy = apodisation(ny, Gy, W, b)
    py = np.mod(centred(ny).astype(np.int64), Gy)
    px = np.mod(centred(nx).astype(np.int64), Gx)
    ix, iy, wx, wy = _tap_tables(traj, Gy, Gx, W, b)
    M = traj.shape[0]
    y = np.zeros((L, M), dtype=np.complex128)
    for l in range(L):
        grid = np.zeros((Gy, Gx), dtype=np.complex128)
        grid[np.ix_(py, px)] = smaps[l] * x * apy[:, None] * apx[None, :]
        Ghat = np.fft.fft2(grid)
        acc = np.zeros(M, dtype=np.complex128)
        for a in range(W):
            for c in range(W):
                acc += wy[:, a] * wx[:, c] * Ghat[iy[:, a], ix[:, c]]
        y[l] = acc
    return y / math.sqrt(ny * nx)


def spread(y_l, traj, Gy, Gx, W, b):
    """Type-1 gridding of one coil's samples onto the (Gy, Gx) grid."""
    ix, iy, wx, wy = _tap_tables(np.asarray(traj, dtype=np.float64), Gy, Gx, W, b)
    H = np.zeros(Gy * Gx, dtype=np.complex128)
    for a in range(W):
        for c in range(W):
            flat = iy[:, a] * Gx + ix[:, c]
            v = y_l * wy[:, a] * wx[:, c]
            H += np.bincount(flat, weights=v.real, minlength=Gy * Gx)
            H += 1j * np.bincount(flat, weights=v.imag, minlength=Gy * Gx)
    return H.reshape(Gy, Gx)


def adjoint(y, smaps, traj, W: int, sigma: float):
    """A^H y by gridding; y (L, M) -> (ny, nx) complex128."""
    y = np.asarray(y, dtype=np.complex128)
    smaps = np.asarray(smaps, dtype=np.complex128)
    L, ny, nx = smaps.shape
    Gy, Gx = grid_size(ny, sigma), grid_size(nx, sigma)
    b = kb.beta(W, sigma)
    apx = apodisation(nx, Gx, W, b)
    apy = apodisation(ny, Gy, W, b)
    py = np.mod(centred(ny).astype(np.int64), Gy)
    px = np.mod(centred(nx).astype(np.int64), Gx)
    x = np.zeros((ny, nx), dtype=np.complex128)
    for l in range(L):
        H = spread(y[l], traj, Gy, Gx, W, b)
        V = np.fft.ifft2(H) * (Gy * Gx)      # unnormalised exp(+2 pi i m n / G)
        x += np.conj(smaps[l]) * V[np.ix_(py, px)] * apy[:, None] * apx[None, :]
    return x / math.sqrt(ny * nx)
