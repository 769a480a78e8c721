"""Toeplitz form of the normal operator A^H A and the circulant (Strang)
data-consistency preconditioner (test infrastructure, FP64).

Sec. 3.4 builds its preconditioners from A^H A, with A = F_Omega (x) S_l.  For
the exact NUDFT, F^H F is a convolution:

    (F^H F v)[n] = sum_m t(n - m) v[m],   t(d) = Npix^(-1) sum_j exp(+i k_j . d),

for d in (-N, N) per axis.  Embedding t in a circulant of size 2N (c[d mod 2N]
= t(d), the d = -N row/column set to zero) gives the exact identity
A^H A x = sum_l conj(S_l) crop(IFFT_2N(Khat * FFT_2N(pad(S_l x)))), Khat = FFT_2N(c),
with x padded into [0, N) and the result read back from [0, N).

Density-compensation preconditioner for the CG solve.  Its symbol is the
gridded sampling density: the eigenvalues lam of T. Chan's optimal circulant
approximation of the N-grid Toeplitz part of F^H F (the circulant nearest in
Frobenius norm, whose first column averages the wrapped diagonals:
c_N[q] = sum over the per-axis choices d in {q, q - N} of
prod_axis w(d) t(d), with w(q) = (N - q)/N and w(q - N) = q/N).  For
H = a A^H A + b I it applies
    M^-1 v = IFFT_N(FFT_N(v) * s^(-1/2)),  s = max(a*max(lam, 0) + b, b/4),
i.e. the square root of the density-compensated symbol.  (The Strang
circulant with the full inverse symbol, the first reading tried, slows CG
down on variable-density spirals; the square-root Chan form speeds it up.)
"""
from __future__ import annotations

import numpy as np


def _circ_offsets(n2: int, n: int) -> np.ndarray:
    """Offset d represented by circulant position p in [0, 2n): p for p < n, p - 2n otherwise."""
    p = np.arange(n2, dtype=np.int64)
    return np.where(p < n, p, p - n2)


def kernel(traj, ny: int, nx: int) -> np.ndarray:
    """Circulant first column c (2ny, 2nx) complex128: c[p] = t(d(p)), zero at d = -N."""
    k = np.asarray(traj, dtype=np.float64)
    dy = _circ_offsets(2 * ny, ny).astype(np.float64)
    dx = _circ_offsets(2 * nx, nx).astype(np.float64)
    Ey = np.exp(1j * np.outer(k[:, 1], dy))  # (M, 2ny)
    Ex = np.exp(1j * np.outer(k[:, 0], dx))  # (M, 2nx)
    c = (Ey.T @ Ex) / (ny * nx)
    c[ny, :] = 0.0
    c[:, nx] = 0.0
    return c


def khat(c: np.ndarray) -> np.ndarray:
    """Khat = FFT_2N(c); real because c is Hermitian (c[-d] = conj c[d])."""
    K = np.fft.fft2(c)
    return K.real


def normal(x, smaps, Kh) -> np.ndarray:
    """A^H A x via the 2N circulant embedding; Kh (2ny, 2nx) real."""
    x = np.asarray(x, dtype=np.complex128)
    smaps = np.asarray(smaps, dtype=np.complex128)
    L, ny, nx = smaps.shape
    out = np.zeros((ny, nx), dtype=np.complex128)
    for l in range(L):
        pad = np.zeros((2 * ny, 2 * nx), dtype=np.complex128)
        pad[:ny, :nx] = smaps[l] * x
        w = np.fft.ifft2(Kh * np.fft.fft2(pad))[:ny, :nx]
        out += np.conj(smaps[l]) * w
    return out


def strang_symbol(c: np.ndarray, ny: int, nx: int) -> np.ndarray:
    """Strang circulant symbol: Re FFT_N of t(d) for d in [-N/2, N/2) wrapped to N."""
    dy = np.arange(ny) - ny // 2
    dx = np.arange(nx) - nx // 2
    cn = np.zeros((ny, nx), dtype=np.complex128)
    cn[np.ix_(np.mod(dy, ny), np.mod(dx, nx))] = c[np.ix_(np.mod(dy, 2 * ny), np.mod(dx, 2 * nx))]
    return np.fft.fft2(cn).real


def chan_column(c: np.ndarray, ny: int, nx: int) -> np.ndarray:
    """First column (ny, nx) of T. Chan's optimal circulant for the N-grid
    Toeplitz operator with kernel t (given as the 2N circulant column c)."""
    qy = np.arange(ny)
    qx = np.arange(nx)
    out = np.zeros((ny, nx), dtype=np.complex128)
    for dy, wy in ((qy, (ny - qy) / ny), (qy - ny, qy / ny)):
        for dx, wx in ((qx, (nx - qx) / nx), (qx - nx, qx / nx)):
            t = c[np.ix_(np.mod(dy, 2 * ny), np.mod(dx, 2 * nx))]
            out += wy[:, None] * wx[None, :] * t
    return out


def chan_symbol(c: np.ndarray, ny: int, nx: int) -> np.ndarray:
    """Eigenvalues of the Chan circulant: Re FFT_N(chan_column)."""
    return np.fft.fft2(chan_column(c, ny, nx)).real


def precond_scale(lam, a: float, b: float) -> np.ndarray:
    """Per-frequency multiplier s^(-1/2) of the density-compensation preconditioner."""
    s = a * np.maximum(lam, 0.0) + b
    return 1.0 / np.sqrt(np.maximum(s, 0.25 * b))


def precond_apply(v, lam, a: float, b: float) -> np.ndarray:
    """M^-1 v for H = a A^H A + b I."""
    return np.fft.ifft2(np.fft.fft2(v) * precond_scale(lam, a, b))
