"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.  Bar (float32 path vs float64 oracle, equal parameters):
relative L2 <= 1e-5; against the exact NUDFT at width 4, sigma 2: <= 2e-3."""
import math

import numpy as np
import pytest

import synth
from helpers import make_plan, quantised, rel, to_dev, to_host
from oracle import hqs as ohqs
from oracle import nudft, nufft, solvers, toeplitz

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def hq():
    import paper_2411_01955_gb300 as m
    return m


def cases():
    return {
        "tiny": synth.tiny_case(0),
        "odd": synth.odd_case(0),
        "odd_w6": dict(synth.odd_case(1, n=32, L=5, M=301, W=6)),
        # 20 coils: two coil chunks in every FFT pass; odd kernel width
        "l20_w5": dict(synth.odd_case(2, n=32, L=20, M=400, W=5)),
        # 16 and 32 coils with G = 2n: the NUFFT passes with the image in the lower half
        # of each line (one and two 16-coil chunks)
        "l16": dict(synth.odd_case(5, n=64, L=16, M=900, W=6)),
        "l32_w4": dict(synth.odd_case(6, n=32, L=32, M=500, W=4)),
    }


@pytest.fixture(scope="module", params=["tiny", "odd", "odd_w6", "l20_w5", "l16", "l32_w4"])
def case(request):
    return quantised(cases()[request.param])


def test_forward_matches_oracle(case):
    plan, traj, smaps = make_plan(case)
    x = to_dev(case["x"])
    y = torch.empty((case["smaps"].shape[0], case["traj"].shape[0]), dtype=torch.complex64, device="cuda")
    hq().forward(plan, x, y)
    got = to_host(y)
    want = nufft.forward(case["x"], case["smaps"], case["traj"], case["W"], case["sigma"])
    assert rel(got, want) <= TOL
    if case["W"] == 4:
        assert rel(got, nudft.forward(case["x"], case["smaps"], case["traj"])) <= 2e-3


def test_adjoint_matches_oracle(case):
    plan, traj, smaps = make_plan(case)
    yv = case["noise"].astype(np.complex64).astype(np.complex128)
    y = to_dev(yv)
    x = torch.empty((case["n"], case["n"]), dtype=torch.complex64, device="cuda")
    hq().adjoint(plan, y, x)
    got = to_host(x)
    want = nufft.adjoint(yv, case["smaps"], case["traj"], case["W"], case["sigma"])
    assert rel(got, want) <= TOL
    if case["W"] == 4:
        assert rel(got, nudft.adjoint(yv, case["smaps"], case["traj"])) <= 2e-3


def test_adjoint_axpy_and_zero_start(case):
    plan, _, _ = make_plan(case)
    n = case["n"]
    yv = case["noise"].astype(np.complex64).astype(np.complex128)
    z = case["x"]
    x = torch.empty((n, n), dtype=torch.complex64, device="cuda")
    hq().adjoint_axpy(plan, to_dev(yv), 0.3, to_dev(z), x)
    want = nufft.adjoint(yv, case["smaps"], case["traj"], case["W"], case["sigma"]) + 0.3 * z
    assert rel(to_host(x), want) <= TOL
    zz = to_dev(z)                        # in place: z and x the same buffer
    hq().adjoint_axpy(plan, to_dev(yv), 0.3, zz, zz)
    assert rel(to_host(zz), want) <= TOL
    # zero start ignores the incoming x and matches a solve from zeros
    for mode in (0, 1):
        a = to_dev(np.full((n, n), 7.0 + 1j))
        b = torch.zeros_like(a)
        ia = hq().dc_solve(plan, 1.0, 1e-2, x, a, max_iter=6, rel_tol=0.0,
                           mode=mode | hq().HQS_SOLVE_X0_ZERO)
        ib = hq().dc_solve(plan, 1.0, 1e-2, x, b, max_iter=6, rel_tol=0.0, mode=mode)
        assert ia.iterations == ib.iterations == 6
        assert rel(to_host(a), to_host(b)) <= 1e-6


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_adjoint_hot_tiles_and_repeatable(tile):
    """Tile-owned spreading with tiles of several items: 1000 of 3000 points
    within 0.02 pi of the k-space centre give the centre tiles far more than
    one item's 256 candidates, so their items write partial slots and the
    last to arrive sums them.  The adjoint matches the oracle, and two calls
    are bitwise equal (no atomics, a fixed summation order)."""
    case = quantised(dict(synth.odd_case(4, n=64, L=6, M=3000, W=6)))
    plan, _, _ = make_plan(case)
    hq().plan_set_tuning(plan, hq().HQS_TUNE_SPREAD_TILE, tile)
    yv = case["noise"].astype(np.complex64).astype(np.complex128)
    want = nufft.adjoint(yv, case["smaps"], case["traj"], case["W"], case["sigma"])
    x1 = torch.empty((case["n"], case["n"]), dtype=torch.complex64, device="cuda")
    x2 = torch.empty_like(x1)
    hq().adjoint(plan, to_dev(yv), x1)
    hq().adjoint(plan, to_dev(yv), x2)
    assert rel(to_host(x1), want) <= TOL
    torch.cuda.synchronize()
    assert torch.equal(x1, x2)


def test_gpu_operator_pair_is_adjoint(case):
    plan, _, _ = make_plan(case)
    rng = np.random.default_rng(3)
    n, L, M = case["n"], case["smaps"].shape[0], case["traj"].shape[0]
    xv = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    yv = rng.normal(size=(L, M)) + 1j * rng.normal(size=(L, M))
    Ax = torch.empty((L, M), dtype=torch.complex64, device="cuda")
    Ahy = torch.empty((n, n), dtype=torch.complex64, device="cuda")
    hq().forward(plan, to_dev(xv), Ax)
    hq().adjoint(plan, to_dev(yv), Ahy)
    x32 = xv.astype(np.complex64).astype(np.complex128)
    y32 = yv.astype(np.complex64).astype(np.complex128)
    lhs = np.vdot(y32, to_host(Ax))
    rhs = np.vdot(to_host(Ahy), x32)
    assert abs(lhs - rhs) / abs(lhs) < 1e-5


def oracle_toeplitz(case):
    n = case["n"]
    c = toeplitz.kernel(case["traj"], n, n)
    return toeplitz.khat(c), toeplitz.chan_symbol(c, n, n)


def test_toeplitz_normal_matches_oracle(case):
    plan, _, _ = make_plan(case)
    Kh, _ = oracle_toeplitz(case)
    out = torch.empty((case["n"], case["n"]), dtype=torch.complex64, device="cuda")
    hq().toeplitz_normal(plan, to_dev(case["x"]), out)
    want = toeplitz.normal(case["x"], case["smaps"], Kh)
    assert rel(to_host(out), want) <= TOL


def test_precond_apply_matches_oracle(case):
    plan, _, _ = make_plan(case)
    _, lam = oracle_toeplitz(case)
    r = case["x"]
    z = torch.empty_like(to_dev(r))
    for a, b in [(1.0, 1e-2), (0.8, 0.05), (-0.3, 2.0)]:
        hq().precond_apply(plan, a, b, to_dev(r), z)
        want = toeplitz.precond_apply(r, lam, a, b)
        assert rel(to_host(z), want) <= TOL, (a, b)


def test_dc_solve_fixed_iterations_matches_oracle(case):
    plan, _, _ = make_plan(case)
    Kh, lam = oracle_toeplitz(case)
    n = case["n"]
    mu = 1e-2
    rhs = nufft.adjoint(case["noise"], case["smaps"], case["traj"], case["W"], case["sigma"])
    rhs = rhs.astype(np.complex64).astype(np.complex128)
    H = lambda v: toeplitz.normal(v, case["smaps"], Kh) + mu * v
    for precond in (hq().HQS_PRECOND_DC, hq().HQS_PRECOND_NONE):
        Minv = (lambda v: toeplitz.precond_apply(v, lam, 1.0, mu)) if precond else None
        want, winfo = solvers.pcg(H, rhs, np.zeros((n, n)), Minv, max_iter=5, tol=0.0)
        x = torch.zeros((n, n), dtype=torch.complex64, device="cuda")
        info = hq().dc_solve(plan, 1.0, mu, to_dev(rhs), x, max_iter=5, rel_tol=0.0, precond=precond)
        assert info.iterations == 5 and info.status == 0
        assert rel(to_host(x), want) <= TOL
        got_hist = np.array(info.history())
        assert np.allclose(got_hist, winfo["res_hist"], rtol=1e-4, atol=0)


@pytest.mark.parametrize("precond", [1, 0])
def test_fused_dc_solve_matches_oracle(case, precond):
    """The persistent cooperative solve follows the same recursion as the oracle."""
    plan, _, _ = make_plan(case)
    Kh, lam = oracle_toeplitz(case)
    n, mu = case["n"], 1e-2
    rhs = nufft.adjoint(case["noise"], case["smaps"], case["traj"], case["W"], case["sigma"])
    rhs = rhs.astype(np.complex64).astype(np.complex128)
    H = lambda v: toeplitz.normal(v, case["smaps"], Kh) + mu * v
    Minv = (lambda v: toeplitz.precond_apply(v, lam, 1.0, mu)) if precond else None
    want, winfo = solvers.pcg(H, rhs, np.zeros((n, n)), Minv, max_iter=5, tol=0.0)
    x = torch.zeros((n, n), dtype=torch.complex64, device="cuda")
    info = hq().dc_solve(plan, 1.0, mu, to_dev(rhs), x, max_iter=5, rel_tol=0.0, precond=precond,
                         mode=hq().HQS_SOLVE_FUSED)
    assert info.iterations == 5 and info.status == 0
    assert rel(to_host(x), want) <= TOL
    assert np.allclose(np.array(info.history()), winfo["res_hist"], rtol=1e-4, atol=0)
    # to tolerance: same iteration count as the per-stage path (+-1), true residual
    xp = torch.zeros_like(x)
    ip = hq().dc_solve(plan, 1.0, mu, to_dev(rhs), xp, max_iter=200, rel_tol=1e-4, precond=precond)
    xf = torch.zeros_like(x)
    inf = hq().dc_solve(plan, 1.0, mu, to_dev(rhs), xf, max_iter=200, rel_tol=1e-4, precond=precond,
                        mode=hq().HQS_SOLVE_FUSED)
    assert inf.status == 0 and abs(inf.iterations - ip.iterations) <= 1
    true_res = np.linalg.norm(rhs - H(to_host(xf))) / np.linalg.norm(rhs)
    assert true_res <= 1.2e-4
    # deterministic: a second fused solve is bitwise identical
    xf2 = torch.zeros_like(x)
    hq().dc_solve(plan, 1.0, mu, to_dev(rhs), xf2, max_iter=200, rel_tol=1e-4, precond=precond,
                  mode=hq().HQS_SOLVE_FUSED)
    torch.cuda.synchronize()
    assert torch.equal(xf, xf2)


def test_dc_solve_converges_to_tolerance(case):
    plan, _, _ = make_plan(case)
    Kh, lam = oracle_toeplitz(case)
    n, mu = case["n"], 1e-2
    rhs = nufft.adjoint(case["noise"], case["smaps"], case["traj"], case["W"], case["sigma"])
    rhs = rhs.astype(np.complex64).astype(np.complex128)
    x = torch.zeros((n, n), dtype=torch.complex64, device="cuda")
    info = hq().dc_solve(plan, 1.0, mu, to_dev(rhs), x, max_iter=200, rel_tol=1e-4)
    assert info.status == 0 and info.rel_residual <= 1e-4
    H = lambda v: toeplitz.normal(v, case["smaps"], Kh) + mu * v
    true_res = np.linalg.norm(rhs - H(to_host(x))) / np.linalg.norm(rhs)
    assert true_res <= 1.2e-4
    hist = info.history()
    assert len(hist) == info.iterations + 1


@pytest.mark.parametrize("mode", [0, 1])
def test_dc_solve_edge_cases(mode):
    case = quantised(synth.tiny_case(1))
    plan, _, _ = make_plan(case)
    n = case["n"]
    import functools
    solve = functools.partial(hq().dc_solve, mode=mode)
    # zero right-hand side: exact zero solution, no iterations
    x = to_dev(np.ones((n, n), dtype=np.complex64))
    info = solve(plan, 1.0, 0.1, torch.zeros_like(x), x, max_iter=10, rel_tol=1e-4)
    assert info.iterations == 0 and info.status == 0
    assert float(torch.abs(x).max()) == 0.0
    # max_iter = 0 returns the start point untouched
    x0 = to_dev(case["x"])
    x = x0.clone()
    info = solve(plan, 1.0, 0.1, to_dev(case["x"] * 2), x, max_iter=0, rel_tol=1e-4, check=False)
    assert info.iterations == 0 and torch.equal(x, x0)
    # non-positive b is rejected
    with pytest.raises(hq().HqsError):
        solve(plan, 1.0, 0.0, x0, x, max_iter=5)
    # non-finite input is reported as breakdown, not a fault
    bad = case["x"].copy()
    bad[3, 4] = np.nan
    info = solve(plan, 1.0, 0.1, to_dev(bad), torch.zeros_like(x0), max_iter=5, rel_tol=1e-4,
                 check=False)
    assert info.status == hq().HQS_ERR_BREAKDOWN


def test_empty_trajectory():
    case = quantised(synth.tiny_case(2))
    case["traj"] = np.zeros((0, 2), dtype=np.float32)
    plan, _, _ = make_plan(case)
    n = case["n"]
    x = torch.empty((n, n), dtype=torch.complex64, device="cuda")
    hq().adjoint(plan, torch.zeros((case["smaps"].shape[0], 0), dtype=torch.complex64, device="cuda"), x)
    assert float(torch.abs(x).max()) == 0.0
    out = torch.empty_like(x)
    hq().toeplitz_normal(plan, to_dev(case["x"]), out)
    assert float(torch.abs(out).max()) == 0.0
    # H = b I: one CG step solves it
    xs = torch.zeros_like(x)
    info = hq().dc_solve(plan, 1.0, 0.5, to_dev(case["x"]), xs, max_iter=5, rel_tol=1e-6)
    assert rel(to_host(xs), case["x"] / 0.5) < 1e-6


def test_gaussian_denoiser_matches_oracle():
    rng = np.random.default_rng(5)
    v = (rng.normal(size=(64, 96)) + 1j * rng.normal(size=(64, 96))).astype(np.complex64)
    v = v.astype(np.complex128)
    out = torch.empty((64, 96), dtype=torch.complex64, device="cuda")
    for s in [0.05, 0.5, 1.5, 4.0]:
        hq().gaussian_denoise(to_dev(v), out, s)
        assert rel(to_host(out), ohqs.gaussian_denoise(v, s)) <= TOL, s
    hq().gaussian_denoise(to_dev(v), out, 0.3, gauss=(1.5, 0.1))   # s = 1.5*0.3/0.1
    assert rel(to_host(out), ohqs.gaussian_denoise(v, 4.5)) <= TOL


def test_hqs_run_matches_oracle_tiny_config():
    """Annealed HQS, 10 outer x 5 CG iterations, Gaussian-smoothing denoiser.

    Truncated, warm-started CG with mu falling to 1e-3 amplifies rounding
    (a relative input perturbation grows ~3e3-fold over the ten steps), so
    the bounds are derived, not assumed: each outer step, started on the GPU
    from the oracle's x_k, must match the oracle's x_{k+1} within
    max(1e-5, 4 d_k), d_k the oracle's own one-step deviation when its inputs
    (A^H y and x_k) are perturbed by the float32 unit roundoff 2^-24; the
    whole run within 4x the oracle's deviation under the same perturbation
    of A^H y."""
    case = quantised(synth.tiny_case(0))
    plan, _, _ = make_plan(case)
    n, K = case["n"], case["K"]
    Kh, lam = oracle_toeplitz(case)
    y = nufft.forward(case["x"], case["smaps"], case["traj"], case["W"], case["sigma"])
    sd = synth.noise_scale_snr(float(np.sum(np.abs(y) ** 2)), y.size, case["snr_db"])
    y = (y + sd * case["noise"]).astype(np.complex64).astype(np.complex128)
    mu = case["mu"].astype(np.float32)
    sigma = mu.copy()   # sigma_k tied to mu_k
    mu64, sg64 = mu.astype(np.float64), sigma.astype(np.float64)
    b0 = nufft.adjoint(y, case["smaps"], case["traj"], case["W"], case["sigma"])
    AHA = lambda v: toeplitz.normal(v, case["smaps"], Kh)
    want, _, hist = ohqs.hqs(AHA, b0, np.zeros((n, n)), mu64, sg64, K, cg_iters=case["cg_iters"], lam=lam)
    gauss = (1.5, float(sigma[0]))
    # per outer step from the oracle's iterate
    rng = np.random.default_rng(0)
    eps = 2.0 ** -24
    xk = np.zeros((n, n), dtype=np.complex128)
    for k in range(K):
        xg = to_dev(xk)
        hq().hqs_run(plan, to_dev(y), xg, mu, sigma, K=k + 1, k0=k, cg_iters=case["cg_iters"], gauss=gauss)
        step, _, _ = ohqs.hqs(AHA, b0, xk, mu64, sg64, k + 1, k0=k, cg_iters=case["cg_iters"], lam=lam)
        b0p = b0 * (1 + eps * rng.normal(size=b0.shape))
        xkp = xk * (1 + eps * rng.normal(size=xk.shape))
        pstep, _, _ = ohqs.hqs(AHA, b0p, xkp, mu64, sg64, k + 1, k0=k, cg_iters=case["cg_iters"], lam=lam)
        tol_k = max(TOL, 4 * rel(pstep, step))
        assert rel(to_host(xg), step) <= tol_k, (k, rel(to_host(xg), step), tol_k)
        xk = hist[k].astype(np.complex64).astype(np.complex128)
    # whole run
    x = torch.zeros((n, n), dtype=torch.complex64, device="cuda")
    hq().hqs_run(plan, to_dev(y), x, mu, sigma, K=K, cg_iters=case["cg_iters"])
    b0p = b0 * (1 + eps * rng.normal(size=b0.shape))
    pert, _, _ = ohqs.hqs(AHA, b0p, np.zeros((n, n)), mu64, sg64, K, cg_iters=case["cg_iters"], lam=lam)
    bound = 4 * rel(pert, want)
    err = rel(to_host(x), want)
    assert err <= bound, (err, bound)
    # resume: 5 + 5 iterations reproduce the straight run (up to the float-atomic
    # summation order of A^H y, recomputed by each call)
    xa = torch.zeros((n, n), dtype=torch.complex64, device="cuda")
    hq().hqs_run(plan, to_dev(y), xa, mu, sigma, K=5, cg_iters=case["cg_iters"], gauss=gauss)
    hq().hqs_run(plan, to_dev(y), xa, mu, sigma, K=K, k0=5, cg_iters=case["cg_iters"], gauss=gauss)
    assert rel(to_host(xa), to_host(x)) <= bound


@pytest.mark.parametrize("metric", ["f1", "chebyshev"])
def test_hqs_run_pmetric_matches_oracle(metric):
    """Annealed HQS in the P-metrics of Sec. 3.4 (10 outer x 5 CG iterations,
    Gaussian smoothing, the 64^2 workload): P = c0 I + c1 A^H A with
    (c0, c1) = (2, -alpha) (F-1) and (4, -10 alpha / 3) (Chebyshev), alpha =
    1 / ||A^H A|| from the oracle's power iteration.  The prox solves
    ((1 + c1 mu) A^H A + c0 mu I) u = A^H y + mu (c0 x + c1 A^H A x), so this
    checks the extra A^H A x term of the right-hand side and the solve's
    coefficients against the oracle.  Bounds derived as in the P = Id test:
    each step from the oracle's x_k within max(1e-5, 4 d_k), the whole run
    within 4x the oracle's deviation under a 2^-24 perturbation of A^H y."""
    case = quantised(synth.tiny_case(0))
    plan, _, _ = make_plan(case)
    n, K = case["n"], case["K"]
    Kh, lam = oracle_toeplitz(case)
    AHA = lambda v: toeplitz.normal(v, case["smaps"], Kh)
    lmax = solvers.power_iteration(AHA, (n, n), iters=300, rtol=1e-12)
    alpha = 1.0 / lmax
    c0, c1 = {"f1": (2.0, -alpha), "chebyshev": (4.0, -10.0 * alpha / 3.0)}[metric]
    c1 = float(np.float32(c1))     # the value the library receives
    y = nufft.forward(case["x"], case["smaps"], case["traj"], case["W"], case["sigma"])
    sd = synth.noise_scale_snr(float(np.sum(np.abs(y) ** 2)), y.size, case["snr_db"])
    y = (y + sd * case["noise"]).astype(np.complex64).astype(np.complex128)
    mu = case["mu"].astype(np.float32)
    sigma = mu.copy()
    mu64, sg64 = mu.astype(np.float64), sigma.astype(np.float64)
    b0 = nufft.adjoint(y, case["smaps"], case["traj"], case["W"], case["sigma"])
    cg = case["cg_iters"]
    run = lambda b, x0, k1, k0=0: ohqs.hqs(AHA, b, x0, mu64, sg64, k1, k0=k0, cg_iters=cg, c0=c0, c1=c1, lam=lam)
    want, _, hist = run(b0, np.zeros((n, n)), K)
    gauss = (1.5, float(sigma[0]))
    rng = np.random.default_rng(4)
    eps = 2.0 ** -24
    xk = np.zeros((n, n), dtype=np.complex128)
    for k in range(K):
        xg = to_dev(xk)
        hq().hqs_run(plan, to_dev(y), xg, mu, sigma, K=k + 1, k0=k, cg_iters=cg, c0=c0, c1=c1, gauss=gauss)
        step, _, _ = run(b0, xk, k + 1, k)
        pstep, _, _ = run(b0 * (1 + eps * rng.normal(size=b0.shape)), xk * (1 + eps * rng.normal(size=xk.shape)),
                          k + 1, k)
        tol_k = max(TOL, 4 * rel(pstep, step))
        err = rel(to_host(xg), step)
        assert err <= tol_k, (metric, k, err, tol_k)
        xk = hist[k].astype(np.complex64).astype(np.complex128)
    x = torch.zeros((n, n), dtype=torch.complex64, device="cuda")
    hq().hqs_run(plan, to_dev(y), x, mu, sigma, K=K, cg_iters=cg, c0=c0, c1=c1)
    pert, _, _ = run(b0 * (1 + eps * rng.normal(size=b0.shape)), np.zeros((n, n)), K)
    bound = 4 * rel(pert, want)
    err = rel(to_host(x), want)
    print(f"HQS {metric}: whole run {err:.2e} (bound {bound:.2e})")
    assert err <= max(TOL, bound), (err, bound)


def test_hqs_denoiser_callback_and_failure():
    case = quantised(synth.tiny_case(0))
    plan, _, _ = make_plan(case)
    n = case["n"]
    y = to_dev(case["noise"])
    calls = []

    def shrink(tin, tout, s):
        calls.append(s)
        tout.copy_(tin * 0.5)
        return 0

    x = torch.zeros((n, n), dtype=torch.complex64, device="cuda")
    hq().hqs_run(plan, y, x, [0.1, 0.05], [1.0, 0.5], cg_iters=3, denoiser=shrink)
    assert calls == [1.0, 0.5]
    with pytest.raises(hq().HqsError) as ei:
        hq().hqs_run(plan, y, x, [0.1], [1.0], cg_iters=3, denoiser=lambda a, b, s: 7)
    assert ei.value.status == hq().HQS_ERR_CALLBACK


def test_power_iteration_matches_oracle():
    case = quantised(synth.tiny_case(0))
    plan, _, _ = make_plan(case)
    Kh, _ = oracle_toeplitz(case)
    n = case["n"]
    want = solvers.power_iteration(lambda v: toeplitz.normal(v, case["smaps"], Kh), (n, n),
                                   iters=200, rtol=1e-9)
    got = hq().power_iteration(plan, iters=200)
    assert abs(got / want - 1) < 1e-3


def test_fused_solve_reports_a_barrier_timeout_and_recovers():
    """The persistent solve's failure path, made to happen without a GPU
    fault: with the test hook armed, one CTA leaves before the first grid
    barrier, the others' bounded waits (cut to about 10 ms) run out, and the
    solve returns HQS_ERR_TIMEOUT; the next solve on the same plan runs
    normally and matches a solve on a fresh plan bit for bit."""
    case = quantised(synth.tiny_case(0))
    plan, _, _ = make_plan(case)
    n, mu = case["n"], 1e-2
    rhs = to_dev(nufft.adjoint(case["noise"], case["smaps"], case["traj"], case["W"], case["sigma"]))
    fused = hq().HQS_SOLVE_FUSED | hq().HQS_SOLVE_X0_ZERO
    hq().plan_set_tuning(plan, hq().HQS_TUNE_DEBUG_BARRIER_SKIP, 1)
    x = torch.zeros((n, n), dtype=torch.complex64, device="cuda")
    info = hq().dc_solve(plan, 1.0, mu, rhs, x, max_iter=300, rel_tol=1e-4, mode=fused, check=False)
    assert info.rc == hq().HQS_ERR_TIMEOUT and info.status == hq().HQS_ERR_TIMEOUT
    x2 = torch.zeros_like(x)
    info2 = hq().dc_solve(plan, 1.0, mu, rhs, x2, max_iter=300, rel_tol=1e-4, mode=fused)
    assert info2.status == 0 and info2.rel_residual <= 1e-4
    plan_b, _, _ = make_plan(case)
    x3 = torch.zeros_like(x)
    hq().dc_solve(plan_b, 1.0, mu, rhs, x3, max_iter=300, rel_tol=1e-4, mode=fused)
    torch.cuda.synchronize()
    assert torch.equal(x2, x3)
    with pytest.raises(hq().HqsError):
        hq().plan_set_tuning(plan, hq().HQS_TUNE_DEBUG_BARRIER_SKIP, 2)


@pytest.mark.parametrize("grid", [0, 37, 100])
def test_fused_line_balanced_passes(grid):
    """16 coils: the persistent solve deals (row, coil) and (column, coil)
    lines to the CTAs in contiguous ranges that straddle rows and columns
    (uneven for 37 and 100 CTAs); it must follow the oracle's recursion."""
    case = quantised(dict(synth.odd_case(3, n=64, L=16, M=1500, W=6)))
    plan, _, _ = make_plan(case)
    hq().plan_set_tuning(plan, hq().HQS_TUNE_FUSED_GRID, grid)
    Kh, lam = oracle_toeplitz(case)
    n, mu = case["n"], 1e-2
    rhs = nufft.adjoint(case["noise"], case["smaps"], case["traj"], case["W"], case["sigma"])
    rhs = rhs.astype(np.complex64).astype(np.complex128)
    H = lambda v: toeplitz.normal(v, case["smaps"], Kh) + mu * v
    Minv = lambda v: toeplitz.precond_apply(v, lam, 1.0, mu)
    want, winfo = solvers.pcg(H, rhs, np.zeros((n, n)), Minv, max_iter=6, tol=0.0)
    x = torch.zeros((n, n), dtype=torch.complex64, device="cuda")
    info = hq().dc_solve(plan, 1.0, mu, to_dev(rhs), x, max_iter=6, rel_tol=0.0,
                         mode=hq().HQS_SOLVE_FUSED)
    assert info.iterations == 6 and info.status == 0
    assert rel(to_host(x), want) <= TOL
    assert np.allclose(np.array(info.history()), winfo["res_hist"], rtol=1e-4, atol=0)
    xf = torch.zeros_like(x)
    inf = hq().dc_solve(plan, 1.0, mu, to_dev(rhs), xf, max_iter=200, rel_tol=1e-4,
                        mode=hq().HQS_SOLVE_FUSED | hq().HQS_SOLVE_X0_ZERO)
    assert inf.status == 0
    assert np.linalg.norm(rhs - H(to_host(xf))) / np.linalg.norm(rhs) <= 1.2e-4


@pytest.mark.parametrize("metric", ["id", "f1", "chebyshev"])
def test_pgd_run_matches_oracle(metric):
    """PnP-PGD, 10 steps, gamma = 0.9 / ||A^H A||, Gaussian-smoothing denoiser,
    gradient step in the metric P = c0 I + c1 A^H A (Id, F-1, Chebyshev with
    alpha = 1 / ||A^H A||).  Bound derived as for HQS: 4x the oracle's own
    deviation when A^H y is perturbed by the float32 unit roundoff, at least
    1e-5."""
    from oracle import hqs as ohqs
    from oracle import solvers as osolvers
    case = quantised(synth.tiny_case(0))
    plan, _, _ = make_plan(case)
    n, K = case["n"], 10
    Kh, _ = oracle_toeplitz(case)
    AHA = lambda v: toeplitz.normal(v, case["smaps"], Kh)
    lmax = osolvers.power_iteration(AHA, (n, n), iters=200, rtol=1e-10)
    alpha = 1.0 / lmax
    c0, c1 = {"id": (1.0, 0.0), "f1": (2.0, -alpha), "chebyshev": (4.0, -10.0 * alpha / 3.0)}[metric]
    gamma = np.full(K, 0.9 / lmax / c0, dtype=np.float32)
    sigma = np.full(K, 0.5, dtype=np.float32)
    y = nufft.forward(case["x"], case["smaps"], case["traj"], case["W"], case["sigma"])
    y = (y + 0.02 * np.sqrt(np.mean(np.abs(y) ** 2)) * case["noise"]).astype(np.complex64).astype(np.complex128)
    b0 = nufft.adjoint(y, case["smaps"], case["traj"], case["W"], case["sigma"])
    c1f = float(np.float32(c1))
    want = ohqs.pgd(AHA, b0, np.zeros((n, n)), gamma.astype(np.float64), sigma.astype(np.float64), K,
                    c0=c0, c1=c1f)
    rng = np.random.default_rng(1)
    b0p = b0 * (1 + 2.0 ** -24 * rng.normal(size=b0.shape))
    pert = ohqs.pgd(AHA, b0p, np.zeros((n, n)), gamma.astype(np.float64), sigma.astype(np.float64), K,
                    c0=c0, c1=c1f)
    tol = max(TOL, 4 * rel(pert, want))
    x = torch.zeros((n, n), dtype=torch.complex64, device="cuda")
    hq().pgd_run(plan, to_dev(y), x, gamma, sigma, c0=c0, c1=c1f)
    err = rel(to_host(x), want)
    print(f"PGD {metric}: rel err {err:.2e} (bound {tol:.2e})")
    assert err <= tol


@pytest.mark.parametrize("use_dcf", [True, False], ids=["dcf", "no_dcf"])
def test_estimate_smaps_matches_oracle(use_dcf):
    """S-map estimation (Sec. 4.1) against the oracle: the mask agrees except
    for pixels whose root-sum-of-squares lies within 1e-4 of the threshold
    (a float decision), and the maps on the common mask to 1e-5."""
    from oracle import smaps as osmaps
    n, L = 64, 4
    traj = synth.traj_radial(32, 128).astype(np.float32)
    x = synth.phantom(4, n).astype(np.complex64).astype(np.complex128)
    S = synth.coil_maps(4, n, L).astype(np.complex64).astype(np.complex128)
    y = nufft.forward(x, S, traj, 6, 2.0).astype(np.complex64).astype(np.complex128)
    dcf = synth.dcf_voronoi(traj).astype(np.float32) if use_dcf else None
    want, mask = osmaps.estimate(y, traj, n, 6, 2.0, thresh=0.3, dcf=dcf)
    out = torch.empty((L, n, n), dtype=torch.complex64, device="cuda")
    hq().estimate_smaps(to_dev(traj, np.float32), to_dev(y), n, out,
                        dcf=to_dev(dcf, np.float32) if use_dcf else None, kernel_width=6, thresh=0.3)
    got = to_host(out)
    gmask = np.sum(np.abs(got) ** 2, axis=0) > 0
    c = osmaps.coil_images(y, traj, n, 6, 2.0, dcf=dcf)
    rss = np.sqrt(np.sum(np.abs(c) ** 2, axis=0))
    band = np.abs(rss - 0.3 * rss.max()) <= 1e-4 * rss.max()
    assert np.all((gmask == mask) | band)
    both = gmask & mask
    assert rel(got[:, both], want[:, both]) <= 1e-5
    assert np.allclose(np.sqrt(np.sum(np.abs(got[:, both]) ** 2, axis=0)), 1.0, atol=1e-5)
