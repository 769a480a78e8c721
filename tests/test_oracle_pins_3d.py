"""Pins of the volumetric (3D) oracle against facts that do not come from it:
brute-force loops on tiny volumes, the 2D operator (pinned on its own) as the
one-slice special case, the library FFT on Cartesian samples, adjointness, and
the Kaiser-Bessel error decreasing with the kernel width.  Shapes are
anisotropic throughout so that a transposed axis fails.
"""
import math

import numpy as np
import pytest

from oracle import hqs, nudft, nufft3d, solvers, toeplitz
import synth


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def rand_c(rng, shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


def rand_traj(rng, M):
    return rng.uniform(-math.pi, math.pi, size=(M, 3)).astype(np.float32)


def test_nudft3d_matches_brute_force_loop():
    rng = np.random.default_rng(11)
    nz, ny, nx, L, M = 3, 4, 5, 2, 7
    x = rand_c(rng, (nz, ny, nx))
    S = rand_c(rng, (L, nz, ny, nx))
    traj = rand_traj(rng, M)
    k = traj.astype(np.float64)
    ref = np.zeros((L, M), dtype=np.complex128)
    for l in range(L):
        for j in range(M):
            acc = 0j
            for iz in range(nz):
                for iy in range(ny):
                    for ix in range(nx):
                        ph = (k[j, 0] * (ix - nx // 2) + k[j, 1] * (iy - ny // 2)
                              + k[j, 2] * (iz - nz // 2))
                        acc += S[l, iz, iy, ix] * x[iz, iy, ix] * complex(math.cos(ph), -math.sin(ph))
            ref[l, j] = acc / math.sqrt(nz * ny * nx)
    assert rel(nufft3d.nudft_forward(x, S, traj), ref) < 1e-14
    yy = rand_c(rng, (L, M))
    ref_a = np.zeros((nz, ny, nx), dtype=np.complex128)
    for l in range(L):
        for iz in range(nz):
            for iy in range(ny):
                for ix in range(nx):
                    ph = k[:, 0] * (ix - nx // 2) + k[:, 1] * (iy - ny // 2) + k[:, 2] * (iz - nz // 2)
                    ref_a[iz, iy, ix] += np.conj(S[l, iz, iy, ix]) * np.sum(yy[l] * np.exp(1j * ph))
    assert rel(nufft3d.nudft_adjoint(yy, S, traj), ref_a / math.sqrt(nz * ny * nx)) < 1e-14


def test_nudft3d_one_slice_is_the_2d_operator():
    rng = np.random.default_rng(12)
    ny, nx, L, M = 6, 10, 3, 40
    x = rand_c(rng, (ny, nx))
    S = rand_c(rng, (L, ny, nx))
    traj = rand_traj(rng, M)                      # any kz: the one slice sits at n_z = 0
    y3 = nufft3d.nudft_forward(x[None], S[:, None], traj)
    assert rel(y3, nudft.forward(x, S, traj[:, :2])) < 1e-14
    yy = rand_c(rng, (L, M))
    assert rel(nufft3d.nudft_adjoint(yy, S[:, None], traj)[0], nudft.adjoint(yy, S, traj[:, :2])) < 1e-14


def test_nudft3d_cartesian_equals_library_fft():
    nz, ny, nx = 4, 6, 8
    rng = np.random.default_rng(13)
    x = rand_c(rng, (nz, ny, nx))
    mz, my, mx = (np.arange(n) - n // 2 for n in (nz, ny, nx))
    MZ, MY, MX = np.meshgrid(mz, my, mx, indexing="ij")
    traj = np.stack([2 * math.pi * MX.ravel() / nx, 2 * math.pi * MY.ravel() / ny,
                     2 * math.pi * MZ.ravel() / nz], 1)
    y = nufft3d.nudft_forward(x, np.ones((1, nz, ny, nx)), traj).reshape(nz, ny, nx)
    X = np.fft.fftn(np.fft.ifftshift(x), norm="ortho")
    assert rel(y, X[np.mod(MZ, nz), np.mod(MY, ny), np.mod(MX, nx)]) < 1e-13


@pytest.mark.parametrize("op", ["nudft", "nufft4", "nufft6"])
def test_adjointness_3d(op):
    rng = np.random.default_rng(14)
    shape, L, M = (8, 12, 10), 2, 300
    x = rand_c(rng, shape)
    y = rand_c(rng, (L, M))
    S = rand_c(rng, (L,) + shape)
    traj = rand_traj(rng, M)
    if op == "nudft":
        Ax, Ahy = nufft3d.nudft_forward(x, S, traj), nufft3d.nudft_adjoint(y, S, traj)
    else:
        W = int(op[-1])
        Ax, Ahy = nufft3d.forward(x, S, traj, W, 2.0), nufft3d.adjoint(y, S, traj, W, 2.0)
    lhs, rhs = np.vdot(y, Ax), np.vdot(Ahy, x)
    assert abs(lhs - rhs) / abs(lhs) < 1e-12


def test_nufft3d_vs_nudft_error_bound_and_monotone_in_width():
    c = synth.volume_case(0, (8, 16, 12), 3, 4, 128)
    x, S, traj = c["x"], c["smaps"], c["traj"]
    ex = nufft3d.nudft_forward(x, S, traj)
    errs = {W: rel(nufft3d.forward(x, S, traj, W, 2.0), ex) for W in (4, 6, 8)}
    # one-dimensional KB aliasing error at W = 4, sigma = 2 is ~2e-4 per axis
    assert errs[4] <= 2e-3
    assert errs[6] < errs[4] / 10 and errs[8] < errs[6]
    y = synth.complex_noise(1, ex.shape)
    ea = {W: rel(nufft3d.adjoint(y, S, traj, W, 2.0), nufft3d.nudft_adjoint(y, S, traj)) for W in (4, 6)}
    assert ea[4] <= 2e-3 and ea[6] < ea[4] / 10


def test_toeplitz3d_equals_dense_normal_operator():
    rng = np.random.default_rng(15)
    shape, L, M = (4, 6, 5), 2, 80
    x = rand_c(rng, shape)
    S = rand_c(rng, (L,) + shape)
    traj = rand_traj(rng, M)
    c = nufft3d.kernel(traj, shape)
    Kh = nufft3d.khat(c)
    assert np.max(np.abs(np.fft.fftn(c).imag)) < 1e-12 * np.max(np.abs(Kh))
    assert rel(nufft3d.normal(x, S, Kh), nufft3d.nudft_normal(x, S, traj)) < 1e-12


def test_toeplitz3d_kernel_brute_force_entries():
    rng = np.random.default_rng(16)
    shape, M = (3, 4, 5), 9
    traj = rand_traj(rng, M)
    c = nufft3d.kernel(traj, shape)
    k = traj.astype(np.float64)
    nz, ny, nx = shape
    for p in [(0, 0, 0), (1, 2, 3), (5, 7, 9), (4, 1, 6), (nz, 2, 2), (1, ny, 2), (2, 1, nx)]:
        d = [q if q < n else q - 2 * n for q, n in zip(p, shape)]
        zero = any(q == n for q, n in zip(p, shape))
        want = 0.0 if zero else np.sum(np.exp(1j * (k[:, 0] * d[2] + k[:, 1] * d[1] + k[:, 2] * d[0]))) / (nz * ny * nx)
        assert abs(c[p] - want) < 1e-14


def test_toeplitz3d_one_slice_is_the_2d_embedding():
    rng = np.random.default_rng(17)
    ny, nx, L, M = 6, 8, 2, 50
    x = rand_c(rng, (ny, nx))
    S = rand_c(rng, (L, ny, nx))
    traj = rand_traj(rng, M)
    K3 = nufft3d.khat(nufft3d.kernel(traj, (1, ny, nx)))
    K2 = toeplitz.khat(toeplitz.kernel(traj[:, :2], ny, nx))
    assert rel(nufft3d.normal(x[None], S[:, None], K3)[0], toeplitz.normal(x, S, K2)) < 1e-13


# ------------------------------------------------- density preconditioner
def test_chan3d_averages_wrapped_diagonals_of_the_dense_normal_matrix():
    # T. Chan (1988): the Frobenius-optimal (three-level) circulant has first
    # column c[q] = mean over m of T[(m + q) mod N, m], T the dense matrix of F^H F.
    rng = np.random.default_rng(18)
    shape, M = (2, 3, 4), 17
    nvox = int(np.prod(shape))
    traj = rand_traj(rng, M)
    S = np.ones((1,) + shape)
    T = np.zeros((nvox, nvox), dtype=np.complex128)
    for i in range(nvox):
        e = np.zeros(nvox, dtype=np.complex128)
        e[i] = 1
        T[:, i] = nufft3d.nudft_normal(e.reshape(shape), S, traj).ravel()
    nz, ny, nx = shape
    want = np.zeros(shape, dtype=np.complex128)
    for q in np.ndindex(*shape):
        acc = 0j
        for m in np.ndindex(*shape):
            r = [(mm + qq) % n for mm, qq, n in zip(m, q, shape)]
            acc += T[(r[0] * ny + r[1]) * nx + r[2], (m[0] * ny + m[1]) * nx + m[2]]
        want[q] = acc / nvox
    c = nufft3d.kernel(traj, shape)
    assert rel(nufft3d.chan_column(c, shape), want) < 1e-12
    assert nufft3d.chan_symbol(c, shape).min() > -1e-12


def test_chan3d_one_slice_is_the_2d_symbol():
    rng = np.random.default_rng(19)
    ny, nx, M = 6, 8, 60
    traj = rand_traj(rng, M)
    lam3 = nufft3d.chan_symbol(nufft3d.kernel(traj, (1, ny, nx)), (1, ny, nx))[0]
    lam2 = toeplitz.chan_symbol(toeplitz.kernel(traj[:, :2], ny, nx), ny, nx)
    assert rel(lam3, lam2) < 1e-13


def test_chan3d_symbol_is_one_on_full_cartesian_sampling():
    shape = (4, 6, 8)
    mz, my, mx = (np.arange(n) - n // 2 for n in shape)
    MZ, MY, MX = np.meshgrid(mz, my, mx, indexing="ij")
    traj = np.stack([2 * math.pi * MX.ravel() / shape[2], 2 * math.pi * MY.ravel() / shape[1],
                     2 * math.pi * MZ.ravel() / shape[0]], 1)
    lam = nufft3d.chan_symbol(nufft3d.kernel(traj, shape), shape)
    assert np.max(np.abs(lam - 1.0)) < 1e-12
    v = rand_c(np.random.default_rng(20), shape)
    assert rel(nufft3d.precond_apply(v, lam, 2.0, 0.5), v / math.sqrt(2.5)) < 1e-13


def test_precond3d_floor_and_clamp_on_plane_waves():
    # plane waves are the 3D circulant's eigenvectors: where lam < 0 the multiplier is
    # b^(-1/2) (the clamp), where a lam + b < b / 4 (a < 0) it is 2 / sqrt(b) (the floor),
    # elsewhere (a lam + b)^(-1/2); frequency kz is the first axis
    nz, ny, nx = 3, 4, 5
    lam = np.full((nz, ny, nx), 0.5)
    lam[1, 2, 3], lam[2, 0, 4] = 10.0, -3.0
    mz, my, mx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for a, b, k, want in ((-0.1, 0.4, (1, 2, 3), 2.0 / math.sqrt(0.4)),
                          (0.7, 0.2, (2, 0, 4), 1.0 / math.sqrt(0.2)),
                          (0.7, 0.2, (1, 2, 3), 1.0 / math.sqrt(7.2)),
                          (0.7, 0.2, (0, 3, 1), 1.0 / math.sqrt(0.55))):
        e = np.exp(2j * np.pi * (k[0] * mz / nz + k[1] * my / ny + k[2] * mx / nx))
        assert rel(nufft3d.precond_apply(e, lam, a, b), want * e) < 1e-13


def test_density_preconditioner_cuts_3d_iterations_on_stacked_spirals():
    # the design property the preconditioner is chosen for (not a parity pin)
    c = synth.volume_case(3, (8, 32, 32), 4, 8, 256)
    K = nufft3d.khat(nufft3d.kernel(c["traj"], c["shape"]))
    lam = nufft3d.chan_symbol(nufft3d.kernel(c["traj"], c["shape"]), c["shape"])
    y = nufft3d.nudft_forward(c["x"], c["smaps"], c["traj"])
    b0 = nufft3d.nudft_adjoint(y, c["smaps"], c["traj"])
    mu = 1e-2
    H = lambda v: nufft3d.normal(v, c["smaps"], K) + mu * v
    z0 = np.zeros(c["shape"])
    _, i_plain = solvers.pcg(H, b0, z0, None, 300, 1e-4)
    _, i_dc = solvers.pcg(H, b0, z0, lambda v: nufft3d.precond_apply(v, lam, 1.0, mu), 300, 1e-4)
    assert i_dc["iters"] < 0.8 * i_plain["iters"], (i_dc["iters"], i_plain["iters"])


# ------------------------------------------------------------ HQS on volumes
def test_gaussian_denoise3d_matches_fft_convolution():
    rng = np.random.default_rng(21)
    shape, sd = (8, 10, 12), 1.3
    v = rand_c(rng, shape)
    g = hqs.gaussian_taps(sd)
    r = (len(g) - 1) // 2
    kern = np.zeros(shape)
    for i in range(-r, r + 1):
        for j in range(-r, r + 1):
            for k in range(-r, r + 1):
                kern[i % shape[0], j % shape[1], k % shape[2]] += g[i + r] * g[j + r] * g[k + r]
    # out[n] = sum_d g(d) v[n + d]: correlation with the (symmetric) kernel
    want = np.fft.ifftn(np.fft.fftn(v) * np.conj(np.fft.fftn(kern)))
    assert rel(hqs.gaussian_denoise(v, sd), want) < 1e-13
    assert rel(hqs.gaussian_denoise(v, 0.05), v) == 0.0


def test_hqs_on_a_one_slice_volume_is_the_2d_run():
    # every piece of the volumetric loop (normal operator, Chan preconditioner,
    # Gaussian smoothing) reduces to its 2D counterpart on one slice
    rng = np.random.default_rng(22)
    ny, nx, L, M, K = 12, 16, 2, 300, 4
    x = rand_c(rng, (ny, nx))
    S = rand_c(rng, (L, ny, nx))
    traj = rand_traj(rng, M)
    y = nudft.forward(x, S, traj[:, :2]) + 0.05 * rand_c(rng, (L, M))
    mu = np.geomspace(1e-1, 1e-2, K)
    sg = np.geomspace(0.2, 0.05, K)
    c2 = toeplitz.kernel(traj[:, :2], ny, nx)
    K2, lam2 = toeplitz.khat(c2), toeplitz.chan_symbol(c2, ny, nx)
    b2 = nudft.adjoint(y, S, traj[:, :2])
    x2, _, _ = hqs.hqs(lambda v: toeplitz.normal(v, S, K2), b2, np.zeros((ny, nx)), mu, sg, K, cg_iters=4,
                       lam=lam2)
    c3 = nufft3d.kernel(traj, (1, ny, nx))
    K3, lam3 = nufft3d.khat(c3), nufft3d.chan_symbol(c3, (1, ny, nx))
    b3 = nufft3d.nudft_adjoint(y, S[:, None], traj)
    x3, _, _ = hqs.hqs(lambda v: nufft3d.normal(v, S[:, None], K3), b3, np.zeros((1, ny, nx)), mu, sg, K,
                       cg_iters=4, lam=lam3, precond_apply=nufft3d.precond_apply)
    assert rel(x3[0], x2) < 1e-12


def test_hqs3d_fixed_point_linear_shrink_prop1():
    # Proposition 1 on a volume: D(v) = v/(1+tau) is the prox of (tau/2)||.||^2, so with
    # P = Id and constant mu the u-iterate converges to u* solving
    # (A^H A + mu tau/(1+tau) I) u = A^H y, and x* = u*/(1+tau); the system is formed
    # densely from the exact NUDFT and solved by the library solver
    rng = np.random.default_rng(23)
    shape, L, M = (4, 6, 6), 2, 120
    nvox = int(np.prod(shape))
    S = rand_c(rng, (L,) + shape)
    traj = rand_traj(rng, M)
    y = rand_c(rng, (L, M))
    c = nufft3d.kernel(traj, shape)
    Kh, lam = nufft3d.khat(c), nufft3d.chan_symbol(c, shape)
    AHA = lambda v: nufft3d.normal(v, S, Kh)
    b0 = nufft3d.nudft_adjoint(y, S, traj)
    mu, tau, K = 0.05, 0.5, 150
    D = lambda u, s: u / (1 + tau)
    # more inner CG iterations than unknowns: every DC step is solved exactly
    x, u, _ = hqs.hqs(AHA, b0, np.zeros(shape), [mu] * K, [1.0] * K, K, cg_iters=nvox + 16, denoiser=D, lam=lam,
                      precond_apply=nufft3d.precond_apply)
    H = np.zeros((nvox, nvox), dtype=np.complex128)
    for i in range(nvox):
        e = np.zeros(nvox, dtype=np.complex128)
        e[i] = 1
        H[:, i] = (nufft3d.nudft_normal(e.reshape(shape), S, traj) + mu * tau / (1 + tau) * e.reshape(shape)).ravel()
    ustar = np.linalg.solve(H, b0.ravel()).reshape(shape)
    assert rel(u, ustar) < 1e-8
    assert rel(x, ustar / (1 + tau)) < 1e-8
