"""Exact multicoil non-uniform DFT (test infrastructure, FP64).

Eq. (1) of Sec. 2.1: y_l = F_Omega S_l x + e_l.  The Fourier operator is
written out as its definition,

    y_l[j] = Npix^(-1/2) * sum_n S_l[n] x[n] exp(-i (kx_j n_x + ky_j n_y)),

with pixel (iy, ix) at the centred coordinate n = (ix - nx/2, iy - ny/2).
The sum factorises over the two axes, so it is evaluated as two matrix
products per coil (cost O(Npix * M) per coil); the adjoint is the conjugate
transpose of the same matrices.
"""
from __future__ import annotations

import numpy as np


def centred(n: int) -> np.ndarray:
    return np.arange(n, dtype=np.float64) - n // 2


def _axis_matrices(traj, ny, nx, sign):
    k = np.asarray(traj, dtype=np.float64)
    Ex = np.exp(sign * 1j * np.outer(k[:, 0], centred(nx)))  # (M, nx)
    Ey = np.exp(sign * 1j * np.outer(k[:, 1], centred(ny)))  # (M, ny)
    return Ex, Ey


def forward(x, smaps, traj):
    """A x for the exact NUDFT; x (ny, nx), smaps (L, ny, nx), traj (M, 2)
    -> y (L, M) complex128."""
    x = np.asarray(x, dtype=np.complex128)
    smaps = np.asarray(smaps, dtype=np.complex128)
    ny, nx = x.shape
    Ex, Ey = _axis_matrices(traj, ny, nx, -1.0)
    y = np.empty((smaps.shape[0], Ex.shape[0]), dtype=np.complex128)
    for l in range(smaps.shape[0]):
        v = smaps[l] * x                      # (ny, nx)
        inner = v @ Ex.T                      # (ny, M): sum over n_x
        y[l] = np.einsum("jy,yj->j", Ey, inner)  # sum over n_y
    return y / np.sqrt(ny * nx)


def adjoint(y, smaps, traj):
    """A^H y for the exact NUDFT; y (L, M) -> x (ny, nx) complex128."""
    y = np.asarray(y, dtype=np.complex128)
    smaps = np.asarray(smaps, dtype=np.complex128)
    L, ny, nx = smaps.shape
    Ex, Ey = _axis_matrices(traj, ny, nx, +1.0)
    x = np.zeros((ny, nx), dtype=np.complex128)
    for l in range(L):
        img = (Ey * y[l][:, None]).T @ Ex     # (ny, nx)
        x += np.conj(smaps[l]) * img
    return x / np.sqrt(ny * nx)


def normal(x, smaps, traj):
    """A^H A x with the exact NUDFT."""
    return adjoint(forward(x, smaps, traj), smaps, traj)
