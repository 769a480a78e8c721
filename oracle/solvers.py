"""Krylov solvers for the data-consistency step (test infrastructure, FP64).

Sec. 3.4 computes the P-metric proximal step "with a subiteration solver"; the
solver used here is preconditioned conjugate gradients on the Hermitian
positive-definite system H u = rhs with H = a A^H A + b I, and its flexible
variant (Notay 2000, truncation 1) for a nonlinear preconditioner.

Iteration protocol (shared with the GPU path by specification, not by code):
    r = rhs - H x;  stop if ||r|| <= tol*||rhs||;  z = M^-1 r;  p = z;  rz = Re<r, z>
    repeat:
        q = H p;  pq = Re<p, q>  (pq <= 0 -> breakdown)
        alpha = rz / pq;  x += alpha p;  r -= alpha q
        stop if ||r|| <= tol*||rhs|| or max_iter reached
        z = M^-1 r;  rz' = Re<r, z>;  beta = rz'/rz;  p = z + beta p
A zero right-hand side returns x = 0 after no iterations.
"""
from __future__ import annotations

import numpy as np


def vdot_re(a, b) -> float:
    return float(np.vdot(a, b).real)


def pcg(apply_H, rhs, x0, apply_Minv=None, max_iter=30, tol=0.0):
    """Returns (x, info) with info = dict(iters, res_hist, status)."""
    rhs = np.asarray(rhs, dtype=np.complex128)
    x = np.array(x0, dtype=np.complex128, copy=True)
    Minv = apply_Minv if apply_Minv is not None else (lambda v: v)
    bnorm = float(np.linalg.norm(rhs))
    if bnorm == 0.0:
        return np.zeros_like(x), dict(iters=0, res_hist=[0.0], status="ok")
    r = rhs - apply_H(x)
    hist = [float(np.linalg.norm(r)) / bnorm]
    if hist[-1] <= tol:
        return x, dict(iters=0, res_hist=hist, status="ok")
    z = Minv(r)
    p = z.copy()
    rz = vdot_re(r, z)
    it = 0
    status = "max_iter"
    while it < max_iter:
        q = apply_H(p)
        pq = vdot_re(p, q)
        if not pq > 0.0:
            status = "breakdown"
            break
        alpha = rz / pq
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        hist.append(float(np.linalg.norm(r)) / bnorm)
        if hist[-1] <= tol:
            status = "ok"
            break
        if it == max_iter:
            break
        z = Minv(r)
        rz_new = vdot_re(r, z)
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    if tol == 0.0 and status == "max_iter":
        status = "ok"          # fixed-iteration mode
    return x, dict(iters=it, res_hist=hist, status=status)


def fcg(apply_H, rhs, x0, apply_B, apply_Minv=None, max_iter=100, tol=1e-4,
        stall_window=5, stall_factor=0.9):
    """Flexible CG with a (possibly nonlinear) preconditioner B and fallback.

    Notay's truncated flexible CG (one direction kept): alpha_k =
    Re<p_k, r_k> / Re<p_k, H p_k> (exact line search along p_k, which keeps
    r_{k+1} orthogonal to p_k whatever B is), beta_k = Re<z_{k+1}, r_{k+1} -
    r_k> / Re<z_k, r_k> (Polak-Ribiere form), p_{k+1} = z_{k+1} + beta_k p_k.
    If Re<z, r> <= 0, Re<p, Hp> <= 0, or ||r|| has not dropped by the factor
    stall_factor over the last stall_window iterations (CG residual norms are
    not monotone, so the window is several iterations), the method restarts
    as plain PCG with apply_Minv from the current iterate for the remaining
    iterations.  Returns (x, info) with info['fallback'].
    """
    rhs = np.asarray(rhs, dtype=np.complex128)
    x = np.array(x0, dtype=np.complex128, copy=True)
    bnorm = float(np.linalg.norm(rhs))
    if bnorm == 0.0:
        return np.zeros_like(x), dict(iters=0, res_hist=[0.0], status="ok", fallback=False)
    r = rhs - apply_H(x)
    hist = [float(np.linalg.norm(r)) / bnorm]
    if hist[-1] <= tol:
        return x, dict(iters=0, res_hist=hist, status="ok", fallback=False)
    z = apply_B(r)
    rz = vdot_re(r, z)
    it = 0
    fallback = rz <= 0.0
    if not fallback:
        p = z.copy()
        while it < max_iter:
            q = apply_H(p)
            pq = vdot_re(p, q)
            if not pq > 0.0:
                fallback = True
                break
            alpha = vdot_re(p, r) / pq
            x = x + alpha * p
            r_old = r
            r = r - alpha * q
            it += 1
            hist.append(float(np.linalg.norm(r)) / bnorm)
            if hist[-1] <= tol:
                return x, dict(iters=it, res_hist=hist, status="ok", fallback=False)
            if it == max_iter:
                break
            if it >= stall_window and hist[-1] > stall_factor * hist[-1 - stall_window]:
                fallback = True
                break
            z = apply_B(r)
            rz_new = vdot_re(r, z)
            if not rz_new > 0.0:
                fallback = True
                break
            beta = vdot_re(z, r - r_old) / rz
            rz = rz_new
            p = z + beta * p
    if fallback and it < max_iter:
        x, inf2 = pcg(apply_H, rhs, x, apply_Minv, max_iter - it, tol)
        hist.extend(inf2["res_hist"][1:])
        return x, dict(iters=it + inf2["iters"], res_hist=hist, status=inf2["status"],
                       fallback=True)
    status = "ok" if hist[-1] <= tol else "max_iter"
    return x, dict(iters=it, res_hist=hist, status=status, fallback=fallback)


def cg_energy(apply_H, rhs, x) -> float:
    """Quadratic CG minimises: 0.5 x^H H x - Re<rhs, x>."""
    return 0.5 * vdot_re(x, apply_H(x)) - vdot_re(rhs, x)


def power_iteration(apply_N, shape, iters=50, rtol=1e-6, seed=0):
    """Largest eigenvalue of a Hermitian PSD operator (used for alpha = 1/||A^H A||)."""
    rng = np.random.default_rng(seed)
    v = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    v /= np.linalg.norm(v)
    lam = 0.0
    for _ in range(iters):
        w = apply_N(v)
        lam_new = vdot_re(v, w)
        v = w / np.linalg.norm(w)
        if lam and abs(lam_new - lam) <= rtol * abs(lam_new):
            lam = lam_new
            break
        lam = lam_new
    return lam
