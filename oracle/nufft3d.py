"""Volumetric (3D) multicoil operator of Eq. (1) (test infrastructure, FP64).

The paper's conclusion (Sec. 5) names 3D and 2D+time data as the next step;
nothing in it changes for a volume except the number of axes.  With voxel
(iz, iy, ix) at the centred coordinate n = (ix - nx//2, iy - ny//2,
iz - nz//2) and trajectory rows k_j = (kx, ky, kz) in radians per voxel:

  exact NUDFT      y_l[j] = Nvox^(-1/2) sum_n S_l[n] x[n] exp(-i k_j . n)
  gridding NUFFT   the same three steps as the 2D oracle (apodise by
                   1/phihat per axis, zero-pad into the sigma-oversampled grid
                   at n mod G, unnormalised FFT, W^3 Kaiser-Bessel taps per
                   point; the adjoint is the exact transpose)
  Toeplitz A^H A   (F^H F v)[n] = sum_m t(n - m) v[m],
                   t(d) = Nvox^(-1) sum_j exp(+i k_j . d), d in (-N, N)^3,
                   embedded in a 2N circulant per axis with every d = -N
                   plane set to zero; Khat = FFT_2N(c) is real.
  preconditioner   the density-compensation preconditioner of Sec. 3.4 on
                   volumes: T. Chan's optimal circulant of the N^3 Toeplitz
                   part of F^H F (first column: the wrapped diagonals
                   averaged, per axis d in {q, q - N} with weights (N - q)/N
                   and q/N), eigenvalues lam = Re FFT_N(column), and
                   M^-1 v = IFFT_N(FFT_N(v) s^(-1/2)), s = max(a max(lam, 0) + b, b/4).

Every formula is evaluated as written, axis by axis, with NumPy products as
the only library steps.
"""
from __future__ import annotations

import math

import numpy as np

from . import kb
from .nudft import centred
from .nufft import apodisation, grid_size, point_taps


# --------------------------------------------------------------- exact NUDFT
def _axis_exp(traj, shape, sign):
    k = np.asarray(traj, dtype=np.float64)
    nz, ny, nx = shape
    Ex = np.exp(sign * 1j * np.outer(k[:, 0], centred(nx)))   # (M, nx)
    Ey = np.exp(sign * 1j * np.outer(k[:, 1], centred(ny)))   # (M, ny)
    Ez = np.exp(sign * 1j * np.outer(k[:, 2], centred(nz)))   # (M, nz)
    return Ex, Ey, Ez


def nudft_forward(x, smaps, traj):
    """A x with the exact 3D NUDFT; x (nz, ny, nx), smaps (L, nz, ny, nx),
    traj (M, 3) -> y (L, M) complex128."""
    x = np.asarray(x, dtype=np.complex128)
    smaps = np.asarray(smaps, dtype=np.complex128)
    nz, ny, nx = x.shape
    Ex, Ey, Ez = _axis_exp(traj, x.shape, -1.0)
    y = np.empty((smaps.shape[0], Ex.shape[0]), dtype=np.complex128)
    for l in range(smaps.shape[0]):
        v = smaps[l] * x
        sx = v @ Ex.T                                  # (nz, ny, M): sum over n_x
        sy = np.einsum("zyj,jy->zj", sx, Ey)           # sum over n_y
        y[l] = np.einsum("zj,jz->j", sy, Ez)           # sum over n_z
    return y / math.sqrt(nz * ny * nx)


def nudft_adjoint(y, smaps, traj):
    """A^H y with the exact 3D NUDFT; y (L, M) -> x (nz, ny, nx)."""
    y = np.asarray(y, dtype=np.complex128)
    smaps = np.asarray(smaps, dtype=np.complex128)
    L, nz, ny, nx = smaps.shape
    Ex, Ey, Ez = _axis_exp(traj, (nz, ny, nx), +1.0)
    x = np.zeros((nz, ny, nx), dtype=np.complex128)
    for l in range(L):
        wz = Ez * y[l][:, None]                        # (M, nz)
        zy = np.einsum("jz,jy->zyj", wz, Ey)           # (nz, ny, M)
        x += np.conj(smaps[l]) * (zy @ Ex)             # sum over j
    return x / math.sqrt(nz * ny * nx)


def nudft_normal(x, smaps, traj):
    return nudft_adjoint(nudft_forward(x, smaps, traj), smaps, traj)


# ------------------------------------------------------------ gridding NUFFT
def _taps3(traj, G, W, b):
    """Per axis a = 0 (x), 1 (y), 2 (z): grid indices (M, W) and weights (M, W)."""
    traj = np.asarray(traj, dtype=np.float64)
    out = []
    w = np.arange(W)
    for a in range(3):
        i0, d = point_taps(traj[:, a], G[a], W)
        out.append((np.mod(i0[:, None] + w[None, :], G[a]), kb.phi(d[:, None] - w[None, :], W, b)))
    return out


def _apod3(shape, G, W, b):
    nz, ny, nx = shape
    return (apodisation(nz, G[2], W, b)[:, None, None] * apodisation(ny, G[1], W, b)[None, :, None]
            * apodisation(nx, G[0], W, b)[None, None, :])


def _grid_sizes(shape, sigma):
    nz, ny, nx = shape
    return (grid_size(nx, sigma), grid_size(ny, sigma), grid_size(nz, sigma))


def forward(x, smaps, traj, W: int, sigma: float):
    """A x by 3D gridding; returns (L, M) complex128."""
    x = np.asarray(x, dtype=np.complex128)
    smaps = np.asarray(smaps, dtype=np.complex128)
    L, nz, ny, nx = smaps.shape
    G = _grid_sizes((nz, ny, nx), sigma)
    b = kb.beta(W, sigma)
    ap = _apod3((nz, ny, nx), G, W, b)
    pos = [np.mod(centred(n).astype(np.int64), g) for n, g in ((nx, G[0]), (ny, G[1]), (nz, G[2]))]
    (ix, wx), (iy, wy), (iz, wz) = _taps3(traj, G, W, b)
    M = ix.shape[0]
    y = np.zeros((L, M), dtype=np.complex128)
    for l in range(L):
        grid = np.zeros((G[2], G[1], G[0]), dtype=np.complex128)
        grid[np.ix_(pos[2], pos[1], pos[0])] = smaps[l] * x * ap
        Gh = np.fft.fftn(grid)
        acc = np.zeros(M, dtype=np.complex128)
        for c in range(W):
            for a in range(W):
                for e in range(W):
                    acc += wz[:, c] * wy[:, a] * wx[:, e] * Gh[iz[:, c], iy[:, a], ix[:, e]]
        y[l] = acc
    return y / math.sqrt(nz * ny * nx)


def spread(y_l, traj, G, W, b):
    """Type-1 gridding of one coil's samples onto the (Gz, Gy, Gx) grid."""
    (ix, wx), (iy, wy), (iz, wz) = _taps3(traj, G, W, b)
    size = G[0] * G[1] * G[2]
    H = np.zeros(size, dtype=np.complex128)
    for c in range(W):
        for a in range(W):
            for e in range(W):
                flat = (iz[:, c] * G[1] + iy[:, a]) * G[0] + ix[:, e]
                v = y_l * wz[:, c] * wy[:, a] * wx[:, e]
                H += np.bincount(flat, weights=v.real, minlength=size)
                H += 1j * np.bincount(flat, weights=v.imag, minlength=size)
    return H.reshape(G[2], G[1], G[0])


def adjoint(y, smaps, traj, W: int, sigma: float):
    """A^H y by 3D gridding; y (L, M) -> (nz, ny, nx) complex128."""
    y = np.asarray(y, dtype=np.complex128)
    smaps = np.asarray(smaps, dtype=np.complex128)
    L, nz, ny, nx = smaps.shape
    G = _grid_sizes((nz, ny, nx), sigma)
    b = kb.beta(W, sigma)
    ap = _apod3((nz, ny, nx), G, W, b)
    pos = [np.mod(centred(n).astype(np.int64), g) for n, g in ((nx, G[0]), (ny, G[1]), (nz, G[2]))]
    x = np.zeros((nz, ny, nx), dtype=np.complex128)
    for l in range(L):
        H = spread(y[l], traj, G, W, b)
        V = np.fft.ifftn(H) * H.size                   # unnormalised exp(+2 pi i m n / G)
        x += np.conj(smaps[l]) * V[np.ix_(pos[2], pos[1], pos[0])] * ap
    return x / math.sqrt(nz * ny * nx)


# ------------------------------------------------------------- Toeplitz 3D
def _circ_offsets(n: int) -> np.ndarray:
    p = np.arange(2 * n, dtype=np.int64)
    return np.where(p < n, p, p - 2 * n).astype(np.float64)


def kernel(traj, shape) -> np.ndarray:
    """Circulant first column c (2nz, 2ny, 2nx): c[p] = t(d(p)), zero on every d = -N plane."""
    nz, ny, nx = shape
    k = np.asarray(traj, dtype=np.float64)
    Ex = np.exp(1j * np.outer(k[:, 0], _circ_offsets(nx)))   # (M, 2nx)
    Ey = np.exp(1j * np.outer(k[:, 1], _circ_offsets(ny)))   # (M, 2ny)
    Ez = np.exp(1j * np.outer(k[:, 2], _circ_offsets(nz)))   # (M, 2nz)
    c = np.empty((2 * nz, 2 * ny, 2 * nx), dtype=np.complex128)
    for pz in range(2 * nz):
        c[pz] = (Ey * Ez[:, pz:pz + 1]).T @ Ex
    c /= nz * ny * nx
    c[nz, :, :] = 0.0
    c[:, ny, :] = 0.0
    c[:, :, nx] = 0.0
    return c


def khat(c: np.ndarray) -> np.ndarray:
    """Khat = FFT_2N(c); real because c is Hermitian."""
    return np.fft.fftn(c).real


def normal(x, smaps, Kh) -> np.ndarray:
    """A^H A x via the 2N^3 circulant embedding; Kh (2nz, 2ny, 2nx) real."""
    x = np.asarray(x, dtype=np.complex128)
    smaps = np.asarray(smaps, dtype=np.complex128)
    L, nz, ny, nx = smaps.shape
    out = np.zeros((nz, ny, nx), dtype=np.complex128)
    for l in range(L):
        pad = np.zeros((2 * nz, 2 * ny, 2 * nx), dtype=np.complex128)
        pad[:nz, :ny, :nx] = smaps[l] * x
        w = np.fft.ifftn(Kh * np.fft.fftn(pad))[:nz, :ny, :nx]
        out += np.conj(smaps[l]) * w
    return out


# ------------------------------------------------- density preconditioner
def chan_column(c, shape) -> np.ndarray:
    """First column (nz, ny, nx) of Chan's optimal circulant for the N^3
    Toeplitz operator with kernel t (given as the 2N circulant column c)."""
    nz, ny, nx = shape
    choices = []
    for n in (nz, ny, nx):
        q = np.arange(n)
        choices.append(((np.mod(q, 2 * n), (n - q) / n), (np.mod(q - n, 2 * n), q / n)))
    out = np.zeros(shape, dtype=np.complex128)
    for pz, wz in choices[0]:
        for py, wy in choices[1]:
            for px, wx in choices[2]:
                out += (wz[:, None, None] * wy[None, :, None] * wx[None, None, :]) * c[np.ix_(pz, py, px)]
    return out


def chan_symbol(c, shape) -> np.ndarray:
    """Eigenvalues of the Chan circulant: Re FFT_N(chan_column)."""
    return np.fft.fftn(chan_column(c, shape)).real


def precond_apply(v, lam, a: float, b: float) -> np.ndarray:
    """M^-1 v for H = a A^H A + b I on volumes."""
    s = a * np.maximum(lam, 0.0) + b
    return np.fft.ifftn(np.fft.fftn(v) / np.sqrt(np.maximum(s, 0.25 * b)))
