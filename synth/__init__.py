"""Seeded synthetic inputs shaped like 2D multicoil brain scans.

This module only draws inputs: images, coil-sensitivity maps, k-space
trajectories, density-compensation weights and unit-variance noise.  It holds
none of the reconstruction arithmetic (no Fourier operator, no gridding, no
solver), so both the CPU oracle and the CUDA path can be fed from it without
sharing any of the method's code.

The paper (Sec. 4.1) simulates acquisitions from fastMRI brain k-space with a
spiral pattern; fastMRI is not available here, so seeded phantoms with the same
shapes (320x320 images, 16 coils, variable-density spirals) stand in for it.

Conventions
-----------
* images are (ny, nx), row-major; pixel (iy, ix) sits at the centred
  coordinate n = (ix - nx/2, iy - ny/2);
* coil maps are (L, ny, nx) and normalised so that sum_l |S_l|^2 = 1 per pixel;
* trajectories are (M, 2) float32 with columns (kx, ky) in radians per pixel,
  inside [-pi, pi).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "phantom", "coil_maps", "traj_radial", "traj_spiral", "dcf_voronoi",
    "complex_noise", "noise_scale_snr", "noise_scale_image_rule",
    "mu_schedule_geometric", "paper_schedule", "tiny_case", "brain_case",
    "odd_case", "phantom3d", "coil_maps3d", "traj_stack_of_spirals", "volume_case",
    "traj_spiral_frames", "dynamic_phantom",
]


def _grid_coords(n):
    """Normalised coordinates in [-1, 1): pixel i maps to (i - n/2)/(n/2)."""
    return (np.arange(n, dtype=np.float64) - n // 2) / (n / 2.0)


def phantom(seed: int, n: int) -> np.ndarray:
    """Random-ellipse phantom with a smooth random phase, complex128 (n, n).

    An outer "skull" ellipse (semi-axes 0.9, 0.8 of the half field of view)
    holds 8-12 random ellipses: centres U(-0.6, 0.6), semi-axes U(0.05, 0.4),
    angle U(0, pi), amplitude U(0.1, 1).  The phase is exp(i*pi*p(x, y)) with p
    a random second-order polynomial scaled to max|p| <= 1 on the grid.
    """
    rng = np.random.default_rng(seed)
    c = _grid_coords(n)
    X, Y = np.meshgrid(c, c, indexing="xy")
    skull = (X / 0.9) ** 2 + (Y / 0.8) ** 2 <= 1.0
    mag = 0.25 * skull.astype(np.float64)
    for _ in range(int(rng.integers(8, 13))):
        cx, cy = rng.uniform(-0.6, 0.6, size=2)
        ax, ay = rng.uniform(0.05, 0.4, size=2)
        th = rng.uniform(0.0, math.pi)
        amp = rng.uniform(0.1, 1.0)
        xr = (X - cx) * math.cos(th) + (Y - cy) * math.sin(th)
        yr = -(X - cx) * math.sin(th) + (Y - cy) * math.cos(th)
        mag += amp * (((xr / ax) ** 2 + (yr / ay) ** 2) <= 1.0)
    mag *= skull
    coef = rng.normal(size=6)
    p = (coef[0] + coef[1] * X + coef[2] * Y + coef[3] * X * X
         + coef[4] * X * Y + coef[5] * Y * Y)
    p /= max(np.abs(p).max(), 1e-12)
    return mag * np.exp(1j * math.pi * p)


def coil_maps(seed: int, n: int, L: int) -> np.ndarray:
    """Smooth coil sensitivities, complex128 (L, n, n), with RSS = 1 per pixel.

    Coil l is a Gaussian bump (std 0.8 in half-FOV units) centred on a circle
    of radius 1.4 half-FOV units at angle 2*pi*l/L plus a small jitter, with a
    phase 2*pi*l/L plus a small random linear ramp.
    """
    rng = np.random.default_rng(seed + 7919)
    c = _grid_coords(n)
    X, Y = np.meshgrid(c, c, indexing="xy")
    maps = np.empty((L, n, n), dtype=np.complex128)
    for l in range(L):
        ang = 2 * math.pi * l / L + rng.uniform(-0.2, 0.2)
        cx, cy = 1.4 * math.cos(ang), 1.4 * math.sin(ang)
        amp = np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2 * 0.8 ** 2))
        rx, ry = rng.uniform(-0.5, 0.5, size=2)
        maps[l] = amp * np.exp(1j * (2 * math.pi * l / L + rx * X + ry * Y))
    rss = np.sqrt((np.abs(maps) ** 2).sum(axis=0))
    return maps / rss[None]


def _wrap_pi(k):
    """Map values into [-pi, pi)."""
    return (k + math.pi) % (2 * math.pi) - math.pi


def traj_radial(n_spokes: int, n_readout: int) -> np.ndarray:
    """Golden-angle radial trajectory, float32 (n_spokes*n_readout, 2).

    Spoke s has angle s*pi*(sqrt(5)-1)/2 (about 111.246 degrees); readout
    sample r sits at radius -pi + 2*pi*r/n_readout.
    """
    golden = math.pi * (math.sqrt(5.0) - 1.0) / 2.0
    th = np.arange(n_spokes, dtype=np.float64)[:, None] * golden
    kr = -math.pi + 2 * math.pi * np.arange(n_readout, dtype=np.float64)[None, :] / n_readout
    kx = _wrap_pi(kr * np.cos(th)).reshape(-1)
    ky = _wrap_pi(kr * np.sin(th)).reshape(-1)
    return np.stack([kx, ky], axis=1).astype(np.float32)


def traj_spiral(n_interleaves: int, n_samples: int, n: int, accel: float = 8.0) -> np.ndarray:
    """Variable-density spiral, float32 (n_interleaves*n_samples, 2).

    k(t) = pi * t^1.5 * exp(i*(2*pi*T*t + 2*pi*i_l/n_interleaves)), t in [0, 1).
    T sets the spacing between neighbouring interleaves at the k-space edge to
    accel times the Nyquist spacing 2*pi/n: 1.5*pi/(n_interleaves*T) = accel*2*pi/n.
    """
    T = 1.5 * n / (2.0 * accel * n_interleaves)
    t = np.arange(n_samples, dtype=np.float64) / n_samples
    il = np.arange(n_interleaves, dtype=np.float64)[:, None]
    k = math.pi * t[None, :] ** 1.5 * np.exp(1j * (2 * math.pi * T * t[None, :]
                                                  + 2 * math.pi * il / n_interleaves))
    k = k.reshape(-1)
    return np.stack([_wrap_pi(k.real), _wrap_pi(k.imag)], axis=1).astype(np.float32)


def _polygon_area(v):
    c = v.mean(axis=0)
    a = np.arctan2(v[:, 1] - c[1], v[:, 0] - c[0])
    v = v[np.argsort(a)]
    x, y = v[:, 0], v[:, 1]
    return 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))


def dcf_voronoi(traj: np.ndarray) -> np.ndarray:
    """Voronoi-cell density-compensation weights, float32 (M,).

    Cells are bounded by mirroring the points across the four edges of the
    [-pi, pi)^2 box; coincident points (the centre of radial spokes) share the
    area of their common cell equally.  Weights are normalised to mean 1.
    """
    from scipy.spatial import Voronoi  # input preparation only

    k = traj.astype(np.float64)
    uniq, inv, counts = np.unique(np.round(k, 9), axis=0, return_inverse=True,
                                  return_counts=True)
    inv = inv.reshape(-1)
    pts = [uniq]
    for ax in (0, 1):
        for edge in (-math.pi, math.pi):
            m = uniq.copy()
            m[:, ax] = 2 * edge - m[:, ax]
            pts.append(m)
    vor = Voronoi(np.concatenate(pts, axis=0))
    area = np.empty(len(uniq))
    for i in range(len(uniq)):
        reg = vor.regions[vor.point_region[i]]
        if len(reg) == 0 or -1 in reg:
            area[i] = np.nan
        else:
            area[i] = _polygon_area(vor.vertices[reg])
    fill = np.nanmedian(area) if np.isfinite(area).any() else 1.0
    area = np.where(np.isfinite(area), area, fill)
    w = area[inv] / counts[inv]
    return (w / w.mean()).astype(np.float32)


def complex_noise(seed: int, shape) -> np.ndarray:
    """Circular complex Gaussian noise with unit variance per complex sample."""
    rng = np.random.default_rng(seed + 104729)
    return (rng.normal(size=shape) + 1j * rng.normal(size=shape)) / math.sqrt(2.0)


def noise_scale_snr(signal_energy: float, n_samples: int, snr_db: float) -> float:
    """Standard deviation giving the requested SNR for a signal of the given
    total energy spread over n_samples complex samples."""
    return math.sqrt(signal_energy / n_samples * 10.0 ** (-snr_db / 10.0))


def noise_scale_image_rule(max_coil_energy: float) -> float:
    """Noise std from the rule of Sec. 4.1: variance 1e-4 * max_n sum_l |x_l(n)|^2,
    where x_l = S_l x are the coil images (read in the image domain)."""
    return math.sqrt(1e-4 * max_coil_energy)


def mu_schedule_geometric(mu_first: float, mu_last: float, K: int) -> np.ndarray:
    """Geometric schedule from mu_first to mu_last over K outer iterations."""
    if K == 1:
        return np.array([mu_first], dtype=np.float64)
    return mu_first * (mu_last / mu_first) ** (np.arange(K) / (K - 1.0))


def paper_schedule(sigma0: float, xi: float, delta: float, lam: float, K: int):
    """Annealing rule of Sec. 3.3 read as sigma_k = sigma0 * xi^(delta*(k-1)),
    gamma_k = lam * sigma_k (k = 1..K); returns (mu, sigma) with mu_k = 1/gamma_k."""
    k = np.arange(1, K + 1, dtype=np.float64)
    sigma = sigma0 * xi ** (delta * (k - 1))
    gamma = lam * sigma
    return 1.0 / gamma, sigma


def tiny_case(seed: int = 0):
    """64x64 image, 4 coils, 16 golden-angle spokes x 128 readout samples,
    KB width 4, oversampling 2, HQS 10 x 5 with mu 1e-1 -> 1e-3."""
    n, L = 64, 4
    return dict(n=n, L=L, W=4, sigma=2.0,
                x=phantom(seed, n), smaps=coil_maps(seed, n, L),
                traj=traj_radial(16, 128), noise=complex_noise(seed, (L, 16 * 128)),
                snr_db=30.0, K=10, cg_iters=5,
                mu=mu_schedule_geometric(1e-1, 1e-3, 10))


def brain_case(seed: int = 0, n: int = 320, L: int = 16, n_interleaves: int = 16,
               n_samples: int = 2048, W: int = 6):
    """320x320 image, 16 coils, variable-density spiral 16 x 2048, KB width 6,
    oversampling 2; data-consistency solve at mu = 1e-2."""
    traj = traj_spiral(n_interleaves, n_samples, n)
    return dict(n=n, L=L, W=W, sigma=2.0,
                x=phantom(seed, n), smaps=coil_maps(seed, n, L), traj=traj,
                noise=complex_noise(seed, (L, traj.shape[0])), mu=1e-2, cg_iters=30)


def odd_case(seed: int = 0, n: int = 16, L: int = 3, M: int = 37, W: int = 4):
    """Small awkward shapes: few coils, a ragged point count and a cluster of
    points at the k-space centre (a hot tile)."""
    rng = np.random.default_rng(seed + 31)
    k = rng.uniform(-math.pi, math.pi, size=(M, 2))
    k[: M // 3] *= 0.02
    return dict(n=n, L=L, W=W, sigma=2.0, x=phantom(seed, n),
                smaps=coil_maps(seed, n, L), traj=k.astype(np.float32),
                noise=complex_noise(seed, (L, M)))


# ------------------------------------------------------------------ volumes
def phantom3d(seed: int, shape) -> np.ndarray:
    """Random-ellipsoid phantom with a smooth random phase, complex128 (nz, ny, nx).

    An outer ellipsoid (semi-axes 0.9, 0.8, 0.85 of the half field of view in
    x, y, z) holds 8-12 random axis-aligned ellipsoids: centres U(-0.5, 0.5),
    semi-axes U(0.08, 0.4), amplitude U(0.1, 1); the phase is exp(i*pi*p) with p
    a random linear-plus-quadratic polynomial scaled to max|p| <= 1.
    """
    nz, ny, nx = shape
    rng = np.random.default_rng(seed + 104729)
    Z, Y, X = np.meshgrid(_grid_coords(nz), _grid_coords(ny), _grid_coords(nx), indexing="ij")
    head = (X / 0.9) ** 2 + (Y / 0.8) ** 2 + (Z / 0.85) ** 2 <= 1.0
    mag = 0.25 * head.astype(np.float64)
    for _ in range(int(rng.integers(8, 13))):
        c = rng.uniform(-0.5, 0.5, size=3)
        a = rng.uniform(0.08, 0.4, size=3)
        amp = rng.uniform(0.1, 1.0)
        mag += amp * ((((X - c[0]) / a[0]) ** 2 + ((Y - c[1]) / a[1]) ** 2
                       + ((Z - c[2]) / a[2]) ** 2) <= 1.0)
    mag *= head
    coef = rng.normal(size=7)
    p = (coef[0] + coef[1] * X + coef[2] * Y + coef[3] * Z + coef[4] * X * X
         + coef[5] * Y * Y + coef[6] * Z * Z)
    p /= max(np.abs(p).max(), 1e-12)
    return mag * np.exp(1j * math.pi * p)


def coil_maps3d(seed: int, shape, L: int) -> np.ndarray:
    """Smooth coil sensitivities, complex128 (L, nz, ny, nx), RSS = 1 per voxel.

    Coil l is a Gaussian bump (std 0.9 half-FOV units) centred on a ring of
    radius 1.4 at angle 2*pi*l/L, alternately raised to z = +-0.5, with phase
    2*pi*l/L plus a small random linear ramp.
    """
    nz, ny, nx = shape
    rng = np.random.default_rng(seed + 15485863)
    Z, Y, X = np.meshgrid(_grid_coords(nz), _grid_coords(ny), _grid_coords(nx), indexing="ij")
    maps = np.empty((L,) + tuple(shape), dtype=np.complex128)
    for l in range(L):
        ang = 2 * math.pi * l / L + rng.uniform(-0.2, 0.2)
        cx, cy, cz = 1.4 * math.cos(ang), 1.4 * math.sin(ang), 0.5 * (-1) ** l
        amp = np.exp(-((X - cx) ** 2 + (Y - cy) ** 2 + (Z - cz) ** 2) / (2 * 0.9 ** 2))
        r = rng.uniform(-0.5, 0.5, size=3)
        maps[l] = amp * np.exp(1j * (2 * math.pi * l / L + r[0] * X + r[1] * Y + r[2] * Z))
    rss = np.sqrt((np.abs(maps) ** 2).sum(axis=0))
    return maps / rss[None]


def traj_stack_of_spirals(n_planes: int, n_interleaves: int, n_samples: int, n: int,
                          accel: float = 8.0) -> np.ndarray:
    """Stack of variable-density spirals, float32 (n_planes*n_interleaves*n_samples, 3).

    Plane p sits at kz = 2*pi*(p - n_planes/2)/n_planes (Cartesian along z,
    Nyquist-spaced when n_planes equals the slice count) and holds the
    traj_spiral pattern for an n-wide field of view, rotated by p times the
    golden angle so that neighbouring planes interleave.  Columns (kx, ky, kz).
    """
    base = traj_spiral(n_interleaves, n_samples, n, accel).astype(np.float64)
    kxy = base[:, 0] + 1j * base[:, 1]
    golden = math.pi * (3.0 - math.sqrt(5.0))
    out = []
    for p in range(n_planes):
        r = kxy * np.exp(1j * golden * p)
        kz = 2 * math.pi * (p - n_planes / 2) / n_planes
        out.append(np.stack([_wrap_pi(r.real), _wrap_pi(r.imag), np.full(r.shape, kz)], axis=1))
    return np.concatenate(out).astype(np.float32)


def volume_case(seed: int = 0, shape=(64, 64, 64), L: int = 16, n_interleaves: int = 8,
                n_samples: int = 1024, W: int = 6):
    """Volume of shape (nz, ny, nx), L coils, stack of nz spirals of
    n_interleaves x n_samples each (8-fold undersampled in-plane), KB width W,
    oversampling 2."""
    nz, ny, nx = shape
    traj = traj_stack_of_spirals(nz, n_interleaves, n_samples, max(ny, nx))
    return dict(shape=tuple(shape), L=L, W=W, sigma=2.0, x=phantom3d(seed, shape),
                smaps=coil_maps3d(seed, shape, L), traj=traj)


# ----------------------------------------------------------------- 2D + time
def traj_spiral_frames(n_frames: int, n_interleaves: int, n_samples: int, n: int,
                       accel: float = 8.0):
    """Per-frame trajectories of a dynamic (2D + time) acquisition: frame t
    holds the traj_spiral pattern rotated by t times the golden angle, so
    consecutive frames sample complementary k-space.  List of float32 (M, 2)."""
    base = traj_spiral(n_interleaves, n_samples, n, accel).astype(np.float64)
    kxy = base[:, 0] + 1j * base[:, 1]
    golden = math.pi * (3.0 - math.sqrt(5.0))
    out = []
    for t in range(n_frames):
        r = kxy * np.exp(1j * golden * t)
        out.append(np.stack([_wrap_pi(r.real), _wrap_pi(r.imag)], axis=1).astype(np.float32))
    return out


def dynamic_phantom(seed: int, n: int, n_frames: int) -> np.ndarray:
    """Frames (T, n, n) complex128: the phantom of `seed` plus a bright disc
    (radius 0.12, amplitude 0.5) moving on a circle of radius 0.25 half-FOV
    units, one turn over the T frames."""
    base = phantom(seed, n)
    c = _grid_coords(n)
    X, Y = np.meshgrid(c, c, indexing="xy")
    out = np.empty((n_frames, n, n), dtype=np.complex128)
    for t in range(n_frames):
        ang = 2 * math.pi * t / n_frames
        disc = ((X - 0.25 * math.cos(ang)) ** 2 + (Y - 0.25 * math.sin(ang)) ** 2) <= 0.12 ** 2
        out[t] = base + 0.5 * disc
    return out
