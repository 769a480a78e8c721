"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
library special cases, closed forms, invariants and brute force on tiny inputs.

Each test targets a mistake that would otherwise go unseen (a dropped scale,
a wrong sign or index, a transposed operand).
"""
import math

import numpy as np
import pytest

from oracle import hqs, kb, nudft, nufft, solvers, toeplitz
import synth


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def rand_c(rng, shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


# ---------------------------------------------------------------- Kaiser-Bessel
def test_i0_series_matches_library():
    special = pytest.importorskip("scipy.special")
    z = np.linspace(0.0, 40.0, 401)
    assert np.max(np.abs(kb.i0(z) / special.i0(z) - 1.0)) < 1e-14


def test_i0_small_argument_closed_form():
    # I0(z) = 1 + z^2/4 + z^4/64 + O(z^6): exact at tiny z
    z = np.array([1e-4, 3e-4])
    assert np.allclose(kb.i0(z), 1 + z ** 2 / 4 + z ** 4 / 64, rtol=1e-16, atol=0)


@pytest.mark.parametrize("W,sigma", [(4, 2.0), (6, 2.0), (5, 1.5)])
def test_phihat_matches_quadrature(W, sigma):
    # int_{-W/2}^{W/2} phi(t) cos(2 pi nu t) dt with t = (W/2) sin(theta):
    # the substitution removes the square-root edge, Gauss-Legendre converges fast.
    b = kb.beta(W, sigma)
    th, wq = np.polynomial.legendre.leggauss(400)
    th = th * (math.pi / 2)
    wq = wq * (math.pi / 2)
    t = (W / 2) * np.sin(th)
    jac = (W / 2) * np.cos(th)
    for nu in [0.0, 0.05, 0.2, 0.37, 0.9, 1.7]:
        quad = np.sum(wq * jac * kb.phi(t, W, b) * np.cos(2 * math.pi * nu * t))
        got = kb.phihat(np.array([nu]), W, b)[0]
        # relative to the value, or to the peak where the value is in a side lobe
        # (the quadrature sums terms of the peak's size there)
        scale = max(abs(quad), 1e-5 * kb.phihat(np.array([0.0]), W, b)[0])
        assert abs(got - quad) < 1e-10 * scale


def test_beta_formula_values():
    # Beatty et al. (2005): W=6, sigma=2 -> pi*sqrt(9*2.25-0.8)
    assert abs(kb.beta(6, 2.0) - math.pi * math.sqrt(19.45)) < 1e-14
    assert abs(kb.beta(4, 2.0) - math.pi * math.sqrt(8.2)) < 1e-14


# ---------------------------------------------------------------- exact NUDFT
def test_nudft_matches_brute_force_loop():
    rng = np.random.default_rng(1)
    n, L, M = 8, 2, 20
    x = rand_c(rng, (n, n))
    S = rand_c(rng, (L, n, n))
    traj = rng.uniform(-math.pi, math.pi, size=(M, 2)).astype(np.float32)
    y = nudft.forward(x, S, traj)
    ref = np.zeros((L, M), dtype=np.complex128)
    k = traj.astype(np.float64)
    for l in range(L):
        for j in range(M):
            acc = 0j
            for iy in range(n):
                for ix in range(n):
                    ph = k[j, 0] * (ix - n // 2) + k[j, 1] * (iy - n // 2)
                    acc += S[l, iy, ix] * x[iy, ix] * complex(math.cos(ph), -math.sin(ph))
            ref[l, j] = acc / n
    assert rel(y, ref) < 1e-14
    # adjoint brute force
    yy = rand_c(rng, (L, M))
    xa = nudft.adjoint(yy, S, traj)
    ref_a = np.zeros((n, n), dtype=np.complex128)
    for l in range(L):
        for iy in range(n):
            for ix in range(n):
                ph = k[:, 0] * (ix - n // 2) + k[:, 1] * (iy - n // 2)
                ref_a[iy, ix] += np.conj(S[l, iy, ix]) * np.sum(yy[l] * np.exp(1j * ph))
    assert rel(xa, ref_a / n) < 1e-14


def cartesian_traj(n):
    m = np.arange(n) - n // 2
    MY, MX = np.meshgrid(m, m, indexing="ij")
    return np.stack([2 * math.pi * MX.ravel() / n, 2 * math.pi * MY.ravel() / n], 1), MY, MX


def test_nudft_cartesian_equals_library_fft():
    n = 12
    rng = np.random.default_rng(2)
    x = rand_c(rng, (n, n))
    S = np.ones((1, n, n), dtype=np.complex128)
    traj, MY, MX = cartesian_traj(n)
    y = nudft.forward(x, S, traj).reshape(n, n)
    X = np.fft.fft2(np.fft.ifftshift(x), norm="ortho")
    assert rel(y, X[np.mod(MY, n), np.mod(MX, n)]) < 1e-13


def test_parseval_cartesian_rss_maps():
    n, L = 16, 3
    x = synth.phantom(3, n)
    S = synth.coil_maps(3, n, L)
    traj, _, _ = cartesian_traj(n)
    y = nudft.forward(x, S, traj)
    assert abs(np.linalg.norm(y) / np.linalg.norm(x) - 1) < 1e-13
    yn = nufft.forward(x, S, traj, 4, 2.0)
    assert abs(np.linalg.norm(yn) / np.linalg.norm(x) - 1) < 2e-3


@pytest.mark.parametrize("op", ["nudft", "nufft4", "nufft6"])
def test_adjointness(op):
    rng = np.random.default_rng(4)
    n, L, M = 16, 3, 150
    x = rand_c(rng, (n, n))
    y = rand_c(rng, (L, M))
    S = rand_c(rng, (L, n, n))
    traj = rng.uniform(-math.pi, math.pi, size=(M, 2)).astype(np.float32)
    if op == "nudft":
        Ax, Ahy = nudft.forward(x, S, traj), nudft.adjoint(y, S, traj)
    else:
        W = int(op[-1])
        Ax, Ahy = nufft.forward(x, S, traj, W, 2.0), nufft.adjoint(y, S, traj, W, 2.0)
    lhs = np.vdot(y, Ax)
    rhs = np.vdot(Ahy, x)
    assert abs(lhs - rhs) / abs(lhs) < 1e-12


# ---------------------------------------------------------------- gridding accuracy
def test_nufft_vs_nudft_error_bound_and_monotone_in_width():
    c = synth.tiny_case(0)
    x, S, traj = c["x"], c["smaps"], c["traj"]
    ex = nudft.forward(x, S, traj)
    errs = {W: rel(nufft.forward(x, S, traj, W, 2.0), ex) for W in (4, 6, 8)}
    assert errs[4] <= 2e-3
    assert errs[6] < errs[4] / 10 and errs[8] < errs[6]
    y = c["noise"]
    ea = rel(nufft.adjoint(y, S, traj, 4, 2.0), nudft.adjoint(y, S, traj))
    assert ea <= 2e-3


def test_nufft_rectangular_image_against_nudft():
    # ny != nx: a per-axis quantity (grid size, apodisation, tap table) applied to the
    # wrong axis changes the result or its shape
    rng = np.random.default_rng(31)
    ny, nx, L, M = 24, 16, 2, 300
    x, S = rand_c(rng, (ny, nx)), rand_c(rng, (L, ny, nx))
    traj = rng.uniform(-math.pi, math.pi, size=(M, 2))
    y = rand_c(rng, (L, M))
    assert rel(nufft.forward(x, S, traj, 6, 2.0), nudft.forward(x, S, traj)) < 1e-4
    assert rel(nufft.adjoint(y, S, traj, 6, 2.0), nudft.adjoint(y, S, traj)) < 1e-4


def test_nufft_odd_shapes_and_hot_centre():
    c = synth.odd_case(0)
    ex = nudft.forward(c["x"], c["smaps"], c["traj"])
    assert rel(nufft.forward(c["x"], c["smaps"], c["traj"], 4, 2.0), ex) < 2e-3


# ---------------------------------------------------------------- Toeplitz
def test_toeplitz_embedding_equals_dense_normal_operator():
    rng = np.random.default_rng(5)
    n, L, M = 12, 2, 90
    x = rand_c(rng, (n, n))
    S = rand_c(rng, (L, n, n))
    traj = rng.uniform(-math.pi, math.pi, size=(M, 2)).astype(np.float32)
    c = toeplitz.kernel(traj, n, n)
    Kh = toeplitz.khat(c)
    assert np.max(np.abs(np.fft.fft2(c).imag)) < 1e-12 * np.max(np.abs(Kh))
    assert rel(toeplitz.normal(x, S, Kh), nudft.normal(x, S, traj)) < 1e-12


def test_toeplitz_kernel_brute_force_entry():
    rng = np.random.default_rng(6)
    n, M = 6, 11
    traj = rng.uniform(-math.pi, math.pi, size=(M, 2)).astype(np.float32)
    c = toeplitz.kernel(traj, n, n)
    k = traj.astype(np.float64)
    for (py, px) in [(0, 0), (1, 4), (7, 2), (11, 11), (n, 3)]:
        dy = py if py < n else py - 2 * n
        dx = px if px < n else px - 2 * n
        want = 0.0 if (py == n or px == n) else np.sum(np.exp(1j * (k[:, 0] * dx + k[:, 1] * dy))) / n ** 2
        assert abs(c[py, px] - want) < 1e-14


def test_density_symbols_are_one_on_full_cartesian():
    n = 16
    traj, _, _ = cartesian_traj(n)
    c = toeplitz.kernel(traj, n, n)
    for lam in (toeplitz.strang_symbol(c, n, n), toeplitz.chan_symbol(c, n, n)):
        assert np.max(np.abs(lam - 1.0)) < 1e-12
    v = rand_c(np.random.default_rng(7), (n, n))
    lam = toeplitz.chan_symbol(c, n, n)
    assert rel(toeplitz.precond_apply(v, lam, 2.0, 0.5), v / math.sqrt(2.5)) < 1e-13


def _dft_matrix(ny, nx):
    # E[k, m] = exp(-2 pi i (ky my / ny + kx mx / nx)), k and m flattened row-major (y, x)
    my, mx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    return np.exp(-2j * np.pi * (np.outer(my.ravel(), my.ravel()) / ny + np.outer(mx.ravel(), mx.ravel()) / nx))


def test_precond_apply_is_inverse_square_root_of_its_circulant():
    # Brute force on a 5 x 4 grid with a random, partly negative symbol (frequency ky
    # along axis 0, in DFT order): two applies followed by the dense circulant whose
    # eigenvalues are a max(lam, 0) + b give v back.  A transposed or mirrored symbol
    # (lam[-k]), a dropped clamp or a full instead of a square-root inverse fails.
    rng = np.random.default_rng(29)
    ny, nx = 5, 4
    lam = rng.uniform(-0.5, 3.0, size=(ny, nx))
    E = _dft_matrix(ny, nx)
    C = E.conj().T @ np.diag((0.7 * np.maximum(lam, 0.0) + 0.2).ravel()) @ E / (ny * nx)
    v = rand_c(rng, (ny, nx))
    z = toeplitz.precond_apply(toeplitz.precond_apply(v, lam, 0.7, 0.2), lam, 0.7, 0.2)
    assert rel((C @ z.ravel()).reshape(ny, nx), v) < 1e-13


def test_precond_apply_floor_on_plane_waves():
    # Plane waves are the circulant's eigenvectors.  With a < 0 the symbol
    # a lam + b falls below b / 4 where lam is large: there the multiplier is the
    # floor's (b / 4)^(-1/2) = 2 / sqrt(b); where lam < 0 it is b^(-1/2).
    ny, nx = 6, 5
    lam = np.full((ny, nx), 0.5)
    lam[2, 3], lam[4, 1] = 10.0, -3.0
    a, b = -0.1, 0.4
    my, mx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    for (ky, kx), want in (((2, 3), 2.0 / math.sqrt(b)), ((4, 1), 1.0 / math.sqrt(b)),
                           ((0, 0), 1.0 / math.sqrt(a * 0.5 + b))):
        e = np.exp(2j * np.pi * (ky * my / ny + kx * mx / nx))
        assert rel(toeplitz.precond_apply(e, lam, a, b), want * e) < 1e-13


def test_chan_circulant_averages_wrapped_diagonals():
    # T. Chan (1988): the Frobenius-optimal circulant approximation of a matrix
    # has first column c[q] = mean over n of T[(n + q) mod N, n].  Build the
    # dense block-Toeplitz matrix of F^H F on a tiny grid and compare.
    rng = np.random.default_rng(17)
    n, M = 5, 23
    traj = rng.uniform(-math.pi, math.pi, size=(M, 2)).astype(np.float32)
    c = toeplitz.kernel(traj, n, n)
    S = np.ones((1, n, n))
    T = dense_matrix(lambda v: nudft.normal(v, S, traj), n)   # (n*n, n*n)
    want = np.zeros((n, n), dtype=np.complex128)
    for qy in range(n):
        for qx in range(n):
            acc = 0j
            for my in range(n):
                for mx in range(n):
                    row = ((my + qy) % n) * n + (mx + qx) % n
                    acc += T[row, my * n + mx]
            want[qy, qx] = acc / (n * n)
    assert rel(toeplitz.chan_column(c, n, n), want) < 1e-12
    lam = toeplitz.chan_symbol(c, n, n)
    assert lam.min() > -1e-12       # a PSD Toeplitz gives a PSD Chan circulant


# ---------------------------------------------------------------- solvers
def small_problem(seed=8, n=16, L=2, M=200):
    rng = np.random.default_rng(seed)
    x = synth.phantom(seed, n)
    S = synth.coil_maps(seed, n, L)
    traj = rng.uniform(-math.pi, math.pi, size=(M, 2)).astype(np.float32)
    c = toeplitz.kernel(traj, n, n)
    Kh = toeplitz.khat(c)
    lam = toeplitz.chan_symbol(c, n, n)
    AHA = lambda v: toeplitz.normal(v, S, Kh)
    y = nudft.forward(x, S, traj) + 0.01 * rand_c(rng, (L, M))
    b0 = nudft.adjoint(y, S, traj)
    return dict(n=n, S=S, traj=traj, Kh=Kh, lam=lam, AHA=AHA, b0=b0, x=x)


def dense_matrix(apply, n):
    cols = []
    for i in range(n * n):
        e = np.zeros(n * n, dtype=np.complex128)
        e[i] = 1
        cols.append(apply(e.reshape(n, n)).ravel())
    return np.stack(cols, axis=1)


def test_pcg_matches_dense_solve():
    P = small_problem()
    n, mu = P["n"], 1e-2
    H = lambda v: P["AHA"](v) + mu * v
    Hd = dense_matrix(H, n)
    assert np.allclose(Hd, Hd.conj().T, atol=1e-12)
    ref = np.linalg.solve(Hd, P["b0"].ravel()).reshape(n, n)
    x, info = solvers.pcg(H, P["b0"], np.zeros((n, n)), None, max_iter=500, tol=1e-12)
    assert info["status"] == "ok" and rel(x, ref) < 1e-10
    Minv = lambda v: toeplitz.precond_apply(v, P["lam"], 1.0, mu)
    x2, info2 = solvers.pcg(H, P["b0"], np.zeros((n, n)), Minv, max_iter=500, tol=1e-12)
    assert rel(x2, ref) < 1e-10
    # true residual agrees with the recursive one at the end
    assert rel(H(x2), P["b0"]) < 1e-11


def test_cg_energy_decreases_monotonically():
    P = small_problem(9)
    n, mu = P["n"], 1e-3
    H = lambda v: P["AHA"](v) + mu * v
    Minv = lambda v: toeplitz.precond_apply(v, P["lam"], 1.0, mu)
    energies = []
    for it in range(0, 25):
        x, _ = solvers.pcg(H, P["b0"], np.zeros((n, n)), Minv, max_iter=it, tol=0.0)
        energies.append(solvers.cg_energy(H, P["b0"], x))
    assert all(e2 <= e1 + 1e-12 * abs(e1) for e1, e2 in zip(energies, energies[1:]))


def test_fcg_with_linear_preconditioner_matches_pcg():
    P = small_problem(10)
    n, mu = P["n"], 1e-2
    H = lambda v: P["AHA"](v) + mu * v
    Minv = lambda v: toeplitz.precond_apply(v, P["lam"], 1.0, mu)
    x1, i1 = solvers.pcg(H, P["b0"], np.zeros((n, n)), Minv, max_iter=200, tol=1e-10)
    x2, i2 = solvers.fcg(H, P["b0"], np.zeros((n, n)), Minv, Minv, max_iter=200, tol=1e-10)
    assert rel(x2, x1) < 1e-8 and not i2["fallback"]
    # a useless preconditioner (negated) must trigger the fallback and still converge
    x3, i3 = solvers.fcg(H, P["b0"], np.zeros((n, n)), lambda v: -v, Minv,
                         max_iter=200, tol=1e-10)
    assert i3["fallback"] and rel(x3, x1) < 1e-8


def test_fcg_fallback_continues_from_the_current_iterate():
    # B is the DC preconditioner for its first three calls (so three flexible-CG
    # iterations equal three PCG iterations) and then returns -r (<z, r> < 0): the
    # fallback is DC-PCG started at x_3 for the remaining iterations
    P = small_problem(18)
    n, mu = P["n"], 1e-2
    H = lambda v: P["AHA"](v) + mu * v
    Minv = lambda v: toeplitz.precond_apply(v, P["lam"], 1.0, mu)
    calls = [0]

    def B(v):
        calls[0] += 1
        return Minv(v) if calls[0] <= 3 else -v

    x0 = 0.3 * synth.phantom(5, n)
    x, info = solvers.fcg(H, P["b0"], x0, B, Minv, max_iter=12, tol=0.0)
    x3, _ = solvers.pcg(H, P["b0"], x0, Minv, max_iter=3, tol=0.0)
    want, _ = solvers.pcg(H, P["b0"], x3, Minv, max_iter=9, tol=0.0)
    assert info["fallback"] and info["iters"] == 12
    assert rel(x, want) < 1e-10


def test_pcg_zero_rhs_and_converged_start():
    P = small_problem(11)
    n = P["n"]
    H = lambda v: P["AHA"](v) + 0.1 * v
    x, info = solvers.pcg(H, np.zeros((n, n)), np.ones((n, n)), None, 10, 1e-4)
    assert info["iters"] == 0 and np.all(x == 0)
    ref, _ = solvers.pcg(H, P["b0"], np.zeros((n, n)), None, 500, 1e-12)
    x, info = solvers.pcg(H, P["b0"], ref, None, 10, 1e-6)
    assert info["iters"] == 0


def test_power_iteration_matches_eigvalsh():
    P = small_problem(12, n=10, M=80)
    Nd = dense_matrix(P["AHA"], P["n"])
    want = np.linalg.eigvalsh((Nd + Nd.conj().T) / 2).max()
    got = solvers.power_iteration(P["AHA"], (P["n"], P["n"]), iters=3000, rtol=1e-13)
    assert abs(got / want - 1) < 1e-6


# ---------------------------------------------------------------- denoiser and HQS
def test_gaussian_denoiser_matches_fft_convolution():
    rng = np.random.default_rng(13)
    v = rand_c(rng, (20, 24))
    s = 1.3
    g = hqs.gaussian_taps(s)
    r = (len(g) - 1) // 2
    ker = np.zeros((20, 24))
    for i in range(-r, r + 1):
        for j in range(-r, r + 1):
            ker[i % 20, j % 24] += g[i + r] * g[j + r]
    # correlation with a symmetric kernel equals convolution
    want = np.fft.ifft2(np.fft.fft2(v) * np.fft.fft2(ker))
    assert rel(hqs.gaussian_denoise(v, s), want) < 1e-13
    assert np.allclose(hqs.gaussian_denoise(v, 0.05), v)
    assert abs(hqs.gaussian_denoise(v, 2.0).sum() - v.sum()) < 1e-10


@pytest.mark.parametrize("s", [2.0, 3.0, 4.0])
def test_gaussian_taps_variance_of_the_truncated_normal(s):
    # taps sampled from a normal of std s and cut at +-3 s: their variance is the
    # truncated normal's, s^2 (1 - 6 phi(3) / (2 Phi(3) - 1)) = 0.97334 s^2 (the
    # sampling at integer offsets changes it by far less than the tolerance here)
    g = hqs.gaussian_taps(s)
    r = (len(g) - 1) // 2
    i = np.arange(-r, r + 1)
    assert r == 3 * s and abs(g.sum() - 1.0) < 1e-15
    var = float(np.sum(g * i * i))
    pdf3 = math.exp(-4.5) / math.sqrt(2 * math.pi)
    want = s * s * (1 - 6 * pdf3 / math.erf(3 / math.sqrt(2)))
    assert abs(var / want - 1) < 0.03


def test_denoiser_std_tracks_the_noise_level():
    # the blur is kappa = 1.5 px at the first noise level and scales with sigma_k
    assert abs(hqs.denoiser_std(0.2, 0.2) - 1.5) < 1e-15
    assert abs(hqs.denoiser_std(0.05, 0.2) - 0.375) < 1e-15


def test_hqs_and_pgd_closed_form_when_AHA_is_identity():
    # With A^H A = I every prox system is ((1 + (c0 + c1) mu_k)) u = b0 + mu_k (c0 + c1) x,
    # solved exactly by the first CG step, and a PGD step is x - gamma_k (c0 + c1)(x - b0);
    # with the shrink D(u, s) = u / (1 + s) both loops are scalar recursions per pixel,
    # so each step's mu_k, sigma_k, gamma_k and the metric enter visibly.
    rng = np.random.default_rng(33)
    b0, x0 = rand_c(rng, (6, 6)), rand_c(rng, (6, 6))
    I = lambda v: v
    D = lambda u, s: u / (1 + s)
    mu = [0.3, 0.1, 0.05, 0.02]
    sig = [0.4, 0.2, 0.1, 0.05]
    gam = [0.2, 0.15, 0.1, 0.05]
    for c0, c1 in [(1.0, 0.0), (2.0, -0.4), (4.0, -10 * 0.4 / 3)]:
        c = c0 + c1
        x, u, _ = hqs.hqs(I, b0, x0, mu, sig, 4, cg_iters=3, c0=c0, c1=c1, denoiser=D)
        want = x0
        for m, sg in zip(mu, sig):
            want = (b0 + m * c * want) / (1 + c * m) / (1 + sg)
        assert rel(x, want) < 1e-13
        xp = hqs.pgd(I, b0, x0, gam, sig, 4, c0=c0, c1=c1, denoiser=D)
        want = x0
        for g, sg in zip(gam, sig):
            want = (want - g * c * (want - b0)) / (1 + sg)
        assert rel(xp, want) < 1e-13


def test_hqs_warm_start_keeps_a_consistent_solution():
    # noise-free data b0 = A^H A x_t and x_0 = x_t: x_t solves every prox system, so
    # warm-started CG leaves it in place (three iterations could not reach it from 0)
    P = small_problem(34)
    n = P["n"]
    xt = synth.phantom(34, n)
    b0 = P["AHA"](xt)
    x, u, _ = hqs.hqs(P["AHA"], b0, xt, [0.05, 0.02], [1.0, 1.0], 2, cg_iters=3,
                      denoiser=lambda v, s: v, lam=P["lam"])
    assert rel(x, xt) < 1e-10 and rel(u, xt) < 1e-10


def test_pgd_fixed_point_in_the_f1_metric():
    # P = 2 I - alpha A^H A, D(v) = v / (1 + tau): the PGD limit solves
    # (tau I + gamma P A^H A) x = gamma P A^H y
    P = small_problem(35)
    n, tau, K = P["n"], 0.5, 300
    lmax = solvers.power_iteration(P["AHA"], (n, n), iters=500, rtol=1e-12)
    alpha = 1.0 / lmax
    gamma = 0.9 / (2.0 * lmax)
    D = lambda u, s: u / (1 + tau)
    x = hqs.pgd(P["AHA"], P["b0"], np.zeros((n, n)), [gamma] * K, [1.0] * K, K, c0=2.0, c1=-alpha,
                denoiser=D)
    Pm = lambda v: 2.0 * v - alpha * P["AHA"](v)
    Hd = dense_matrix(lambda v: tau * v + gamma * Pm(P["AHA"](v)), n)
    want = np.linalg.solve(Hd, (gamma * Pm(P["b0"])).ravel()).reshape(n, n)
    assert rel(x, want) < 1e-8


def test_hqs_fixed_point_linear_shrink_prop1():
    # D(v) = v/(1+tau) is the prox of (tau/2)||.||^2.  With P = Id and constant
    # mu, HQS converges to u* solving (A^H A + mu tau/(1+tau) I) u = A^H y,
    # x* = u*/(1+tau); PGD converges to (gamma A^H A + tau I) x = gamma A^H y.
    P = small_problem(14)
    n, mu, tau, K = P["n"], 0.05, 0.5, 120
    D = lambda u, s: u / (1 + tau)
    x, u, _ = hqs.hqs(P["AHA"], P["b0"], np.zeros((n, n)), [mu] * K, [1.0] * K, K,
                      cg_iters=60, denoiser=D, lam=P["lam"])
    Hd = dense_matrix(lambda v: P["AHA"](v) + mu * tau / (1 + tau) * v, n)
    ustar = np.linalg.solve(Hd, P["b0"].ravel()).reshape(n, n)
    assert rel(u, ustar) < 1e-8
    assert rel(x, ustar / (1 + tau)) < 1e-8
    gamma = 1.0 / mu
    xp = hqs.pgd(P["AHA"], P["b0"], np.zeros((n, n)), [0.5] * 400, [1.0] * 400, 400,
                 denoiser=D)
    Hp = dense_matrix(lambda v: 0.5 * P["AHA"](v) + tau * v, n)
    xpstar = np.linalg.solve(Hp, 0.5 * P["b0"].ravel()).reshape(n, n)
    assert rel(xp, xpstar) < 1e-8
    assert gamma > 0


def test_hqs_fixed_point_gaussian_smoothing():
    # circulant smoothing G: fixed point solves (A^H A + mu (I - G)) u = A^H y
    P = small_problem(15)
    n, mu, s, K = P["n"], 0.05, 0.8, 150
    D = lambda u, _s: hqs.gaussian_denoise(u, s)
    x, u, _ = hqs.hqs(P["AHA"], P["b0"], np.zeros((n, n)), [mu] * K, [1.0] * K, K,
                      cg_iters=60, denoiser=D, lam=P["lam"])
    Hd = dense_matrix(lambda v: P["AHA"](v) + mu * (v - hqs.gaussian_denoise(v, s)), n)
    ustar = np.linalg.solve(Hd, P["b0"].ravel()).reshape(n, n)
    assert rel(u, ustar) < 1e-7


def test_hqs_pmetric_prox_is_argmin():
    # one prox step with P = c0 I + c1 A^H A must satisfy the optimality
    # condition gamma A^H (A u - y) + P (u - x) = 0 (Sec. 3.4 definition).
    P = small_problem(16)
    n, mu = P["n"], 0.05
    alpha = 1.0 / solvers.power_iteration(P["AHA"], (n, n), iters=500, rtol=1e-12)
    x0 = synth.phantom(99, n)
    for c0, c1 in [(1.0, 0.0), (2.0, -alpha), (4.0, -10.0 * alpha / 3.0)]:
        D = lambda u, s: u
        _, u, _ = hqs.hqs(P["AHA"], P["b0"], x0, [mu], [1.0], 1, cg_iters=200,
                          c0=c0, c1=c1, denoiser=D, lam=P["lam"])
        gamma = 1.0 / mu
        grad = gamma * (P["AHA"](u) - P["b0"]) + c0 * (u - x0) + c1 * P["AHA"](u - x0)
        assert np.linalg.norm(grad) < 1e-8 * np.linalg.norm(gamma * P["b0"])


def test_prox_coefficients():
    assert hqs.prox_coefficients(0.1, 1.0, 0.0) == (1.0, 0.1)
    a, b = hqs.prox_coefficients(0.1, 2.0, -0.5)
    assert abs(a - 0.95) < 1e-15 and abs(b - 0.2) < 1e-15


def test_density_preconditioner_cuts_iterations_on_vd_spiral():
    # the design property the preconditioner is chosen for (not a parity pin)
    n, L = 64, 4
    traj = synth.traj_spiral(16, 512, n)
    S = synth.coil_maps(0, n, L)
    c = toeplitz.kernel(traj, n, n)
    Kh = toeplitz.khat(c)
    lam = toeplitz.chan_symbol(c, n, n)
    AHA = lambda v: toeplitz.normal(v, S, Kh)
    y = nudft.forward(synth.phantom(0, n), S, traj) + 0.01 * synth.complex_noise(0, (L, traj.shape[0]))
    b0 = nudft.adjoint(y, S, traj)
    mu = 1e-2
    H = lambda v: AHA(v) + mu * v
    _, i_plain = solvers.pcg(H, b0, np.zeros((n, n)), None, 300, 1e-4)
    _, i_dc = solvers.pcg(H, b0, np.zeros((n, n)),
                          lambda v: toeplitz.precond_apply(v, lam, 1.0, mu), 300, 1e-4)
    assert i_dc["iters"] < 0.8 * i_plain["iters"]


# ---------------------------------------------------------------- conv net
from oracle import convnet


def small_net(seed=0, layers=((2, 3), (3, 2))):
    rng = np.random.default_rng(seed)
    return [(rng.normal(size=(co, ci, 3, 3)), rng.normal(size=co)) for ci, co in layers]


def test_conv3x3_matches_brute_force():
    rng = np.random.default_rng(20)
    x = rng.normal(size=(2, 3, 5, 4))
    W = rng.normal(size=(2, 3, 3, 3))
    b = rng.normal(size=2)
    out = convnet.conv3x3(x, W, b)
    ref = np.zeros_like(out)
    for n in range(2):
        for o in range(2):
            for y in range(5):
                for xx in range(4):
                    acc = b[o]
                    for i in range(3):
                        for dy in range(3):
                            for dx in range(3):
                                yy, xc = y + dy - 1, xx + dx - 1
                                if 0 <= yy < 5 and 0 <= xc < 4:
                                    acc += W[o, i, dy, dx] * x[n, i, yy, xc]
                    ref[n, o, y, xx] = acc
    assert np.max(np.abs(out - ref)) < 1e-12


def test_conv3x3_single_channel_equals_library_correlation():
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(21)
    x = rng.normal(size=(1, 1, 9, 7))
    W = rng.normal(size=(1, 1, 3, 3))
    out = convnet.conv3x3(x, W, np.zeros(1))[0, 0]
    ref = signal.correlate2d(x[0, 0], W[0, 0], mode="same", boundary="fill")
    assert np.max(np.abs(out - ref)) < 1e-12


def test_convnet_gradient_matches_finite_differences():
    rng = np.random.default_rng(22)
    params = small_net(1, layers=((2, 4), (4, 4), (4, 2)))
    x = rng.normal(size=(3, 2, 6, 5))
    t = rng.normal(size=(3, 2, 6, 5))
    loss, grads = convnet.loss_and_grad(params, x, t)
    g = np.concatenate([np.concatenate([dW.ravel(), db.ravel()]) for dW, db in grads])
    layers = [(p[0].shape[1], p[0].shape[0]) for p in params]
    vec = convnet.flatten(params)
    h = 1e-6
    # 25 random parameters and every bias (a handful among the weights)
    biases, k0 = [], 0
    for W, b in params:
        k0 += W.size
        biases += list(range(k0, k0 + b.size))
        k0 += b.size
    for k in list(rng.choice(vec.size, size=25, replace=False)) + biases:
        vp, vm = vec.copy(), vec.copy()
        vp[k] += h
        vm[k] -= h
        lp, _ = convnet.loss_and_grad(convnet.unflatten(vp, layers), x, t)
        lm, _ = convnet.loss_and_grad(convnet.unflatten(vm, layers), x, t)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(fd)), (k, fd, g[k])


def test_adam_first_step_closed_form():
    # after one step from m = v = 0: update = lr * g / (|g| + eps) elementwise
    g = np.array([0.5, -2.0, 1e-3])
    p, m, v = convnet.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, 0.1)
    assert np.allclose(p, -0.1 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_learned_preconditioner_starts_as_dc_preconditioner():
    # zero last layer: the learned preconditioner reduces to the DC one
    P = small_problem(23)
    params = convnet.init_params(0)
    assert convnet.num_params() == 19682
    r = P["b0"]
    z = convnet.learned_precond(r, P["lam"], 1.0, 0.05, params)
    assert rel(z, toeplitz.precond_apply(r, P["lam"], 1.0, 0.05)) < 1e-15


def test_learned_preconditioner_is_positively_homogeneous():
    # the network sees zdc / s, which does not change when r is scaled, and its output
    # is scaled back by s: z(c r) = c z(r) for c > 0, whatever the weights and biases
    P = small_problem(24)
    rng = np.random.default_rng(24)
    vec = convnet.flatten(convnet.init_params(1))
    vec = vec + 0.05 * rng.normal(size=vec.shape)          # last layer and biases non-zero
    params = convnet.unflatten(vec)
    r = P["b0"]
    z1 = convnet.learned_precond(r, P["lam"], 1.0, 0.05, params)
    z2 = convnet.learned_precond(3.7 * r, P["lam"], 1.0, 0.05, params)
    assert rel(z1, toeplitz.precond_apply(r, P["lam"], 1.0, 0.05)) > 1e-3
    assert rel(z2, 3.7 * z1) < 1e-13


def test_learned_preconditioner_scale_is_the_rms_of_the_dc_output():
    # last layer: zero weights and bias (c, 0), so net(.) = c + 0i everywhere and
    # z - zdc = s c: s must be the root-mean-square of zdc over the complex pixels
    P = small_problem(25)
    params = convnet.init_params(2)
    W4, b4 = params[-1]
    params[-1] = (np.zeros_like(W4), np.array([0.7, 0.0]))
    r = P["b0"]
    zdc = toeplitz.precond_apply(r, P["lam"], 1.0, 0.05)
    z = convnet.learned_precond(r, P["lam"], 1.0, 0.05, params)
    s = math.sqrt(float(np.sum(zdc.real ** 2 + zdc.imag ** 2)) / zdc.size)
    assert rel(z - zdc, np.full(zdc.shape, 0.7 * s)) < 1e-13


# ------------------------------------------------------------------ S-maps (Sec. 4.1)
def test_smaps_window_closed_form():
    from oracle import smaps
    n = 64
    # u = 0, +-5, +-10, 12 Cartesian units on each axis
    us = np.array([0.0, 5.0, -5.0, 10.0, -10.0, 12.0])
    traj = np.stack([us * 2 * np.pi / n, np.zeros_like(us)], axis=1)
    w = smaps.hamming_centre(traj, n, 20)
    assert np.allclose(w, [1.0, 0.54, 0.54, 0.08, 0.08, 0.0], atol=1e-12)
    # separable: off the axes the weight is the product of the two axes' values
    pts = np.array([[5.0, 5.0], [-5.0, 10.0], [0.0, 12.0], [0.0, -5.0]]) * 2 * np.pi / n
    assert np.allclose(smaps.hamming_centre(pts, n, 20), [0.54 ** 2, 0.54 * 0.08, 0.0, 0.54], atol=1e-12)


def test_smaps_estimate_normalised_masked_and_phase_covariant():
    from oracle import nufft as onufft, smaps
    n, L = 48, 4
    traj = synth.traj_radial(32, 96)
    x = synth.phantom(2, n)
    S = synth.coil_maps(2, n, L)
    y = onufft.forward(x, S, traj, 4, 2.0)
    est, mask = smaps.estimate(y, traj, n, 4, 2.0, thresh=0.3)
    rss = np.sqrt(np.sum(np.abs(est) ** 2, axis=0))
    assert mask.any() and not mask.all()
    assert np.allclose(rss[mask], 1.0, atol=1e-12) and np.all(rss[~mask] == 0.0)
    # a common complex factor on the data only rotates every map by its phase
    c = 3.0 * np.exp(0.7j)
    est2, mask2 = smaps.estimate(c * y, traj, n, 4, 2.0, thresh=0.3)
    assert np.array_equal(mask, mask2)
    assert np.allclose(est2, np.exp(0.7j) * est, atol=1e-12)
    # one coil: unit modulus on the mask
    est1, m1 = smaps.estimate(y[:1], traj, n, 4, 2.0, thresh=0.3)
    assert np.allclose(np.abs(est1[0][m1]), 1.0, atol=1e-12)


def test_smaps_estimate_recovers_smooth_maps_of_a_smooth_object():
    """For a smooth positive object and maps with root-sum-of-squares 1, the
    windowed, density-compensated low-resolution coil images are ~ S_l times
    a positive blur of the object, so the normalised estimate returns S_l on
    the object; without the density weights the radial centre dominates and
    the estimate is much worse."""
    from oracle import nufft as onufft, smaps
    n, L = 64, 6
    yy, xx = np.mgrid[0:n, 0:n] - n / 2
    x = np.exp(-(xx ** 2 + yy ** 2) / (2 * (0.3 * n) ** 2)).astype(np.complex128)
    S = synth.coil_maps(5, n, L)
    traj = synth.traj_radial(64, 2 * n)
    y = onufft.forward(x, S, traj, 6, 2.0)
    dcf = synth.dcf_voronoi(traj)
    est, mask = smaps.estimate(y, traj, n, 6, 2.0, thresh=0.3, dcf=dcf)
    err = np.linalg.norm((est - S)[:, mask]) / np.linalg.norm(S[:, mask])
    raw, mraw = smaps.estimate(y, traj, n, 6, 2.0, thresh=0.3)
    err_raw = np.linalg.norm((raw - S)[:, mraw]) / np.linalg.norm(S[:, mraw])
    print(f"S-map recovery: {err:.3f} with density weights, {err_raw:.3f} without")
    assert err < 0.1 and err < err_raw, (err, err_raw)
