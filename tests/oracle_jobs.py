"""Per-slice oracle work for the headline-size parity tests, run in worker
processes started with the 'spawn' method (the test process has already
initialised CUDA, so it must not fork).  Each job takes plain NumPy arrays and
calls only the oracle; nothing here touches the CUDA library."""
from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np

from oracle import hqs as ohqs
from oracle import nufft, solvers, toeplitz


def pool(jobs: int):
    workers = max(1, min(jobs, (os.cpu_count() or 2) // 2, 8))
    return cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))


def rel(a, b) -> float:
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def c64(a):
    return np.asarray(a).astype(np.complex64).astype(np.complex128)


def pcg_fixed(smaps, Kh, lam, mu, rhs, iters, seed):
    """`iters` DC-preconditioned CG iterations from zero on (A^H A + mu I) u = rhs
    (rhs already rounded to complex64), and the deviation of the same run when
    rhs is perturbed by the float32 unit roundoff (the derived bound's input)."""
    H = lambda v: toeplitz.normal(v, smaps, Kh) + mu * v
    M = lambda v: toeplitz.precond_apply(v, lam, 1.0, mu)
    want, info = solvers.pcg(H, rhs, np.zeros_like(rhs), M, max_iter=iters, tol=0.0)
    rng = np.random.default_rng(seed)
    bp = rhs * (1 + 2.0 ** -24 * rng.normal(size=rhs.shape))
    pert, _ = solvers.pcg(H, bp, np.zeros_like(rhs), M, max_iter=iters, tol=0.0)
    return want, info["res_hist"], rel(pert, want)


def normal_rhs(smaps, Kh, mu, x):
    """rhs = (A^H A + mu I) x, rounded to complex64: a right-hand side whose
    exact solution is the phantom x."""
    return c64(toeplitz.normal(x, smaps, Kh) + mu * x)


def true_residual(smaps, Kh, mu, rhs, u):
    """||rhs - (A^H A + mu I) u|| / ||rhs|| in FP64."""
    r = rhs - (toeplitz.normal(u, smaps, Kh) + mu * u)
    return float(np.linalg.norm(r) / np.linalg.norm(rhs))


def slice_operators(traj, n):
    c = toeplitz.kernel(traj, n, n)
    return toeplitz.khat(c), toeplitz.chan_symbol(c, n, n)


def hqs_slice(case, y, mu, sigma, K, cg, seed):
    """The annealed HQS run of one slice (Gaussian smoothing, DC-preconditioned
    CG), and its deviation when A^H y is perturbed by the float32 unit roundoff."""
    n = case["n"]
    Kh, lam = slice_operators(case["traj"], n)
    b0 = nufft.adjoint(y, case["smaps"], case["traj"], case["W"], case["sigma"])
    AHA = lambda v: toeplitz.normal(v, case["smaps"], Kh)
    want, _, _ = ohqs.hqs(AHA, b0, np.zeros((n, n)), mu, sigma, K, cg_iters=cg, lam=lam)
    rng = np.random.default_rng(seed)
    b0p = b0 * (1 + 2.0 ** -24 * rng.normal(size=b0.shape))
    pert, _, _ = ohqs.hqs(AHA, b0p, np.zeros((n, n)), mu, sigma, K, cg_iters=cg, lam=lam)
    return want, rel(pert, want)


def dc_slice(case, mu, iters, seed):
    """Operators of one slice, rhs = (A^H A + mu I) x_phantom, and `iters`
    fixed PCG iterations with their perturbation deviation."""
    n = case["n"]
    Kh, lam = slice_operators(case["traj"], n)
    rhs = normal_rhs(case["smaps"], Kh, mu, case["x"])
    want, hist, dev = pcg_fixed(case["smaps"], Kh, lam, mu, rhs, iters, seed)
    return rhs, want, hist, dev
