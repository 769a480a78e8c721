"""Coil-sensitivity (S-map) estimation (test infrastructure, FP64).

Sec. 4.1 estimates the S-maps from the centre of k-space under a 20 x 20
Hamming window, takes them to the image domain and masks them to the
object.  Written out here with the readings the paper leaves open:

  window   separable Hamming in Cartesian grid units u = k n / (2 pi):
           h(u) = 0.54 + 0.46 cos(2 pi u / width) for |u| <= width / 2, else 0,
           w_j = h(u_x) h(u_y);
  images   c_l = A_1^H (w d y_l), the single-coil adjoint NUFFT (S = 1) of the
           windowed samples of coil l (same gridding parameters as the rest),
           d the optional per-sample density-compensation weights (1 if none:
           trajectories that oversample the centre then bias the estimate);
  maps     S_l = c_l / sqrt(sum_l |c_l|^2) (root-sum-of-squares normalisation);
  mask     pixels where that root-sum-of-squares is at least thresh times its
           maximum; S_l = 0 elsewhere.
"""
from __future__ import annotations

import numpy as np

from . import nufft


def hamming_centre(traj, n: int, width: float = 20.0) -> np.ndarray:
    """Weights w_j of the separable Hamming window over the k-space centre."""
    u = np.asarray(traj, dtype=np.float64) * n / (2.0 * np.pi)
    h = np.where(np.abs(u) <= width / 2.0, 0.54 + 0.46 * np.cos(2.0 * np.pi * u / width), 0.0)
    return h[:, 0] * h[:, 1]


def coil_images(y, traj, n: int, W: int, sigma: float, width: float = 20.0, dcf=None) -> np.ndarray:
    """(L, n, n): c_l = A_1^H (w d y_l)."""
    y = np.asarray(y, dtype=np.complex128)
    w = hamming_centre(traj, n, width)
    if dcf is not None:
        w = w * np.asarray(dcf, dtype=np.float64)
    ones = np.ones((1, n, n), dtype=np.complex128)
    return np.stack([nufft.adjoint((w * y[l])[None], ones, traj, W, sigma) for l in range(y.shape[0])])


def estimate(y, traj, n: int, W: int, sigma: float, width: float = 20.0, thresh: float = 0.05, dcf=None):
    """(S, mask): S (L, n, n) normalised to root-sum-of-squares 1 on the mask, 0 off it."""
    c = coil_images(y, traj, n, W, sigma, width, dcf)
    rss = np.sqrt(np.sum(np.abs(c) ** 2, axis=0))
    mask = rss >= thresh * rss.max() if rss.max() > 0 else np.zeros(rss.shape, dtype=bool)
    safe = np.where(mask, rss, 1.0)
    return np.where(mask[None], c / safe[None], 0.0), mask
