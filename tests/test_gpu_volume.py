"""Volumetric (3D) operator on the GPU against the FP64 oracle.

Tolerances.  The GPU and the oracle grid with the same Kaiser-Bessel kernel,
so they differ by float32 rounding only: a 3D transform of size G^3 adds about
log2(G^3) * 2^-24 relative error per pass and the W^3-tap sums about
2^-24 sqrt(W^3); with four passes that is ~1e-6, and the checks allow 1e-5.
The GPU's Toeplitz kernel is gridded with an 8-wide kernel on a 4N grid,
whose relative error is ~1e-7 (the oracle pins show 7e-8 for the operator at
W = 8), so the Toeplitz product against the exact oracle embedding is held to
the same 1e-5.  At the benchmark size the oracle cannot run whole: there the
forward and adjoint are checked at sampled points/voxels against the exact
NUDFT (difference = the W = 6 gridding error, ~1e-5), the Toeplitz kernel at
sampled offsets against its defining sum, and A^H A against the GPU's own
adjoint of its forward (two independent code paths, equal up to the gridding
error).
"""
import math

import numpy as np
import pytest

import synth
from helpers import rel, to_dev, to_host
from oracle import hqs as ohqs, nufft3d, solvers

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def hq():
    import paper_2411_01955_gb300 as m
    return m


def q(case):
    out = dict(case)
    out["x"] = case["x"].astype(np.complex64).astype(np.complex128)
    out["smaps"] = case["smaps"].astype(np.complex64).astype(np.complex128)
    out["traj"] = case["traj"].astype(np.float32)
    return out


CASES = {
    # anisotropic, 3 coils (a ragged coil chunk), 8 planes of 4 x 256 samples
    "aniso": lambda: q(synth.volume_case(1, (8, 16, 32), 3, 4, 256)),
    # 32^3 with 8 coils, width 4
    "cube32": lambda: q(dict(synth.volume_case(2, (32, 32, 32), 8, 4, 128), W=4)),
}


def plan_of(case, W=None):
    traj = to_dev(case["traj"], np.float32)
    smaps = to_dev(case["smaps"])
    return hq().plan3d_create(traj, case["shape"], smaps, W or case["W"], 2.0), traj, smaps


@pytest.mark.parametrize("name", list(CASES))
def test_forward_adjoint_3d_match_oracle(name):
    c = CASES[name]()
    plan, _, _ = plan_of(c)
    L, M = c["L"], c["traj"].shape[0]
    x = to_dev(c["x"])
    y = torch.empty((L, M), dtype=torch.complex64, device="cuda")
    hq().forward3d(plan, x, y)
    want = nufft3d.forward(c["x"], c["smaps"], c["traj"], c["W"], c["sigma"])
    ef = rel(to_host(y), want)
    yin = synth.complex_noise(5, (L, M)).astype(np.complex64).astype(np.complex128)
    xa = torch.empty(c["shape"], dtype=torch.complex64, device="cuda")
    hq().adjoint3d(plan, to_dev(yin), xa)
    ea = rel(to_host(xa), nufft3d.adjoint(yin, c["smaps"], c["traj"], c["W"], c["sigma"]))
    print(f"{name}: forward {ef:.2e}, adjoint {ea:.2e}")
    assert ef <= 1e-5 and ea <= 1e-5


@pytest.mark.parametrize("name", list(CASES))
def test_toeplitz_3d_matches_exact_embedding(name):
    c = CASES[name]()
    plan, _, _ = plan_of(c)
    K = nufft3d.khat(nufft3d.kernel(c["traj"], c["shape"]))
    T = [2 * v for v in c["shape"]]
    kg = torch.empty(T, dtype=torch.float32, device="cuda")
    hq().plan3d_khat(plan, kg)
    torch.cuda.synchronize()
    ek = rel(kg.cpu().numpy().astype(np.float64) * np.prod(T), K)
    out = torch.empty(c["shape"], dtype=torch.complex64, device="cuda")
    hq().toeplitz_normal3d(plan, to_dev(c["x"]), out)
    et = rel(to_host(out), nufft3d.normal(c["x"], c["smaps"], K))
    print(f"{name}: Khat {ek:.2e}, A^H A {et:.2e}")
    assert ek <= 1e-5 and et <= 1e-5


def test_adjointness_3d_on_gpu():
    c = CASES["aniso"]()
    plan, _, _ = plan_of(c)
    L, M = c["L"], c["traj"].shape[0]
    rng = np.random.default_rng(3)
    xv = (rng.normal(size=c["shape"]) + 1j * rng.normal(size=c["shape"])).astype(np.complex64)
    yv = (rng.normal(size=(L, M)) + 1j * rng.normal(size=(L, M))).astype(np.complex64)
    Ax = torch.empty((L, M), dtype=torch.complex64, device="cuda")
    Ahy = torch.empty(c["shape"], dtype=torch.complex64, device="cuda")
    hq().forward3d(plan, to_dev(xv), Ax)
    hq().adjoint3d(plan, to_dev(yv), Ahy)
    lhs = np.vdot(yv.astype(np.complex128), to_host(Ax))
    rhs = np.vdot(to_host(Ahy), xv.astype(np.complex128))
    assert abs(lhs - rhs) / abs(lhs) < 1e-5


def test_dc_solve_3d_matches_oracle_cg():
    c = CASES["aniso"]()
    plan, _, _ = plan_of(c)
    mu = 1e-2
    K = nufft3d.khat(nufft3d.kernel(c["traj"], c["shape"]))
    y = nufft3d.forward(c["x"], c["smaps"], c["traj"], c["W"], c["sigma"])
    rhs = nufft3d.adjoint(y, c["smaps"], c["traj"], c["W"], c["sigma"])
    rhs = rhs.astype(np.complex64).astype(np.complex128)
    H = lambda v: nufft3d.normal(v, c["smaps"], K) + mu * v
    xo, io = solvers.pcg(H, rhs, np.zeros_like(rhs), max_iter=200, tol=1e-4)
    x = torch.zeros(c["shape"], dtype=torch.complex64, device="cuda")
    info = hq().dc_solve3d(plan, 1.0, mu, to_dev(rhs), x, max_iter=200, rel_tol=1e-4,
                           precond=hq().HQS_PRECOND_NONE)
    got = to_host(x)
    true_res = float(np.linalg.norm(rhs - H(got)) / np.linalg.norm(rhs))
    print(f"3D DC solve: {info.iterations} iterations (oracle {io['iters']}), recursion {info.rel_residual:.2e}, "
          f"true {true_res:.2e}, vs oracle solution {rel(got, xo):.2e}")
    assert info.rc == hq().HQS_OK and info.rel_residual <= 1e-4
    assert abs(info.iterations - io["iters"]) <= max(2, io["iters"] // 10)
    assert true_res <= 2e-4
    # the CG recursion history starts at 1 for a zero start and decreases overall
    h = info.history()
    assert abs(h[0] - 1.0) < 1e-6 and h[-1] <= 1e-4


def test_dc_solve_3d_zero_rhs_and_start_at_solution():
    c = CASES["aniso"]()
    plan, _, _ = plan_of(c)
    x = torch.full(c["shape"], 1 + 1j, dtype=torch.complex64, device="cuda")
    info = hq().dc_solve3d(plan, 1.0, 1e-2, torch.zeros_like(x), x, max_iter=10, rel_tol=1e-4,
                           precond=hq().HQS_PRECOND_NONE)
    assert info.rc == hq().HQS_OK and info.iterations == 0
    assert float(x.abs().max()) == 0.0
    # nz = 8 has no 8-point transform: the density preconditioner is refused, not approximated
    with pytest.raises(hq().HqsError) as e:
        hq().dc_solve3d(plan, 1.0, 1e-2, torch.ones_like(x), x, max_iter=10, rel_tol=1e-4)
    assert e.value.status == hq().HQS_ERR_UNSUPPORTED


def pc_case():
    # every axis a transform size (16, 32, 32), 4 coils, 16 planes of 8 x 256 samples
    return q(synth.volume_case(4, (16, 32, 32), 4, 8, 256))


def test_precond_3d_matches_oracle():
    c = CASES["cube32"]()
    plan, _, _ = plan_of(c)
    lam = nufft3d.chan_symbol(nufft3d.kernel(c["traj"], c["shape"]), c["shape"])
    r = synth.complex_noise(8, c["shape"]).astype(np.complex64).astype(np.complex128)
    z = torch.empty(c["shape"], dtype=torch.complex64, device="cuda")
    for a, b in ((1.0, 1e-2), (2.0, 0.5)):
        hq().precond_apply3d(plan, a, b, to_dev(r), z)
        e = rel(to_host(z), nufft3d.precond_apply(r, lam, a, b))
        print(f"precond a={a} b={b}: {e:.2e}")
        assert e <= 1e-5


def test_dc_solve_3d_density_preconditioned_matches_oracle_pcg():
    c = pc_case()
    plan, _, _ = plan_of(c)
    mu = 1e-2
    kern = nufft3d.kernel(c["traj"], c["shape"])
    K = nufft3d.khat(kern)
    lam = nufft3d.chan_symbol(kern, c["shape"])
    y = nufft3d.forward(c["x"], c["smaps"], c["traj"], c["W"], c["sigma"])
    rhs = nufft3d.adjoint(y, c["smaps"], c["traj"], c["W"], c["sigma"])
    rhs = rhs.astype(np.complex64).astype(np.complex128)
    H = lambda v: nufft3d.normal(v, c["smaps"], K) + mu * v
    z0 = np.zeros_like(rhs)
    xo, io = solvers.pcg(H, rhs, z0, lambda v: nufft3d.precond_apply(v, lam, 1.0, mu), 200, 1e-4)
    _, ip = solvers.pcg(H, rhs, z0, None, 200, 1e-4)
    x = torch.zeros(c["shape"], dtype=torch.complex64, device="cuda")
    info = hq().dc_solve3d(plan, 1.0, mu, to_dev(rhs), x, max_iter=200, rel_tol=1e-4)
    got = to_host(x)
    xp = torch.zeros_like(x)
    plain = hq().dc_solve3d(plan, 1.0, mu, to_dev(rhs), xp, max_iter=200, rel_tol=1e-4,
                            precond=hq().HQS_PRECOND_NONE)
    true_res = float(np.linalg.norm(rhs - H(got)) / np.linalg.norm(rhs))
    print(f"3D DC-PCG: {info.iterations} iterations (oracle {io['iters']}; plain CG {plain.iterations}, "
          f"oracle {ip['iters']}), true residual {true_res:.2e}")
    assert info.rc == hq().HQS_OK and info.rel_residual <= 1e-4 and true_res <= 2e-4
    assert abs(info.iterations - io["iters"]) <= max(2, io["iters"] // 10)
    assert abs(plain.iterations - ip["iters"]) <= max(2, ip["iters"] // 10)
    assert info.iterations < plain.iterations


def test_volume_edge_cases():
    c = CASES["aniso"]()
    smaps = to_dev(c["smaps"])
    empty = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    plan = hq().plan3d_create(empty, c["shape"], smaps, 6, 2.0)
    x = to_dev(c["x"])
    out = torch.full(c["shape"], 7.0, dtype=torch.complex64, device="cuda")
    hq().adjoint3d(plan, torch.zeros((c["L"], 0), dtype=torch.complex64, device="cuda"), out)
    assert float(out.abs().max()) == 0.0
    out.fill_(7.0)
    hq().toeplitz_normal3d(plan, x, out)
    assert float(out.abs().max()) == 0.0
    traj = to_dev(c["traj"], np.float32)
    for shape, W, sg in [((8, 16, 24), 6, 2.0), ((8, 16, 32), 3, 2.0), ((8, 16, 32), 6, 1.5),
                         ((4, 16, 32), 6, 2.0)]:
        with pytest.raises(hq().HqsError) as e:
            hq().plan3d_create(traj, shape, to_dev(np.ones((c["L"],) + shape, np.complex64)), W, sg)
        assert e.value.status == hq().HQS_ERR_INVALID_ARG


# ------------------------------------------------------------ benchmark size
def test_volume_benchmark_size_sampled():
    shape, L = (64, 64, 64), 16
    c = q(synth.volume_case(0, shape, L, 8, 1024))
    plan, _, _ = plan_of(c)
    M = c["traj"].shape[0]
    x = to_dev(c["x"])
    y = torch.empty((L, M), dtype=torch.complex64, device="cuda")
    hq().forward3d(plan, x, y)
    yh = to_host(y)
    rng = np.random.default_rng(9)
    k = c["traj"].astype(np.float64)
    nz, ny, nx = shape
    ez, ey, ex = (np.arange(n) - n // 2 for n in shape)
    # forward: 48 sampled points, all coils, against the exact NUDFT sum
    js = rng.choice(M, 48, replace=False)
    Ex = np.exp(-1j * np.outer(k[js, 0], ex))
    Ey = np.exp(-1j * np.outer(k[js, 1], ey))
    Ez = np.exp(-1j * np.outer(k[js, 2], ez))
    phase = Ez[:, :, None, None] * Ey[:, None, :, None] * Ex[:, None, None, :]   # (48, nz, ny, nx)
    want = np.einsum("jzyx,lzyx->lj", phase, c["smaps"] * c["x"]) / math.sqrt(nz * ny * nx)
    ef = rel(yh[:, js], want)
    # adjoint: 32 sampled voxels against the exact sum over every point
    yin = synth.complex_noise(6, (L, M)).astype(np.complex64).astype(np.complex128)
    xa = torch.empty(shape, dtype=torch.complex64, device="cuda")
    hq().adjoint3d(plan, to_dev(yin), xa)
    xah = to_host(xa)
    vs = [tuple(int(rng.integers(0, shape[a])) for a in range(3)) for _ in range(32)]
    got, exp_ = [], []
    for (iz, iy, ix) in vs:
        ph = np.exp(1j * (k[:, 0] * (ix - nx // 2) + k[:, 1] * (iy - ny // 2) + k[:, 2] * (iz - nz // 2)))
        s = (yin @ ph)                                    # per coil
        exp_.append(np.sum(np.conj(c["smaps"][:, iz, iy, ix]) * s) / math.sqrt(nz * ny * nx))
        got.append(xah[iz, iy, ix])
    ea = rel(np.array(got), np.array(exp_))
    # Toeplitz kernel: sampled offsets of IFFT(Khat) against the defining sum
    T = [2 * v for v in shape]
    kg = torch.empty(T, dtype=torch.float32, device="cuda")
    hq().plan3d_khat(plan, kg)
    torch.cuda.synchronize()
    cfull = np.fft.ifftn(kg.cpu().numpy().astype(np.float64)) * np.prod(T)
    got_t, want_t = [], []
    for _ in range(24):
        p = tuple(int(rng.integers(0, t)) for t in T)
        d = [pp if pp < t // 2 else pp - t for pp, t in zip(p, T)]
        zero = any(pp == t // 2 for pp, t in zip(p, T))
        w = 0.0 if zero else np.sum(np.exp(1j * (k[:, 0] * d[2] + k[:, 1] * d[1] + k[:, 2] * d[0]))) / (nz * ny * nx)
        got_t.append(cfull[p])
        want_t.append(w)
    et = np.max(np.abs(np.array(got_t) - np.array(want_t))) / np.abs(cfull[0, 0, 0])
    # A^H A against the GPU adjoint of the GPU forward
    out = torch.empty(shape, dtype=torch.complex64, device="cuda")
    hq().toeplitz_normal3d(plan, x, out)
    ref = torch.empty(shape, dtype=torch.complex64, device="cuda")
    hq().adjoint3d(plan, y, ref)
    en = rel(to_host(out), to_host(ref))
    print(f"64^3 x 16 coils, {M} points: forward {ef:.2e}, adjoint {ea:.2e}, kernel {et:.2e}, "
          f"Toeplitz vs A^H(A x) {en:.2e}")
    assert ef <= 1e-4 and ea <= 1e-4 and et <= 1e-5 and en <= 1e-4


def test_volume_128_sampled():
    """128^3 x 8 coils, 128 planes of 8 x 512 samples (524 288 points): the
    256-point two-stage transforms of the Toeplitz passes and the 512-point
    kernel gridding, checked as at 64^3 (sampled exact sums, A^H A against
    A^H(A x))."""
    shape, L = (128, 128, 128), 8
    c = q(synth.volume_case(5, shape, L, 8, 512))
    plan, _, _ = plan_of(c)
    M = c["traj"].shape[0]
    x = to_dev(c["x"])
    y = torch.empty((L, M), dtype=torch.complex64, device="cuda")
    hq().forward3d(plan, x, y)
    yh = to_host(y)
    rng = np.random.default_rng(13)
    k = c["traj"].astype(np.float64)
    nz, ny, nx = shape
    ez, ey, ex = (np.arange(n) - n // 2 for n in shape)
    v = c["smaps"] * c["x"]
    got, want = [], []
    for j in rng.choice(M, 12, replace=False):
        t = np.einsum("lzyx,x->lzy", v, np.exp(-1j * k[j, 0] * ex))
        t = np.einsum("lzy,y->lz", t, np.exp(-1j * k[j, 1] * ey))
        want.append(np.einsum("lz,z->l", t, np.exp(-1j * k[j, 2] * ez)) / math.sqrt(nz * ny * nx))
        got.append(yh[:, j])
    ef = rel(np.array(got), np.array(want))
    yin = synth.complex_noise(4, (L, M)).astype(np.complex64).astype(np.complex128)
    xa = torch.empty(shape, dtype=torch.complex64, device="cuda")
    hq().adjoint3d(plan, to_dev(yin), xa)
    xah = to_host(xa)
    got, want = [], []
    for _ in range(8):
        iz, iy, ix = (int(rng.integers(0, n)) for n in shape)
        ph = np.exp(1j * (k[:, 0] * (ix - nx // 2) + k[:, 1] * (iy - ny // 2) + k[:, 2] * (iz - nz // 2)))
        want.append(np.sum(np.conj(c["smaps"][:, iz, iy, ix]) * (yin @ ph)) / math.sqrt(nz * ny * nx))
        got.append(xah[iz, iy, ix])
    ea = rel(np.array(got), np.array(want))
    T = [2 * n for n in shape]
    kg = torch.empty(T, dtype=torch.float32, device="cuda")
    hq().plan3d_khat(plan, kg)
    torch.cuda.synchronize()
    cfull = np.fft.ifftn(kg.cpu().numpy().astype(np.float64)) * np.prod(T)
    errs = []
    for _ in range(12):
        p = tuple(int(rng.integers(0, t)) for t in T)
        d = [pp if pp < t // 2 else pp - t for pp, t in zip(p, T)]
        zero = any(pp == t // 2 for pp, t in zip(p, T))
        w = 0.0 if zero else np.sum(np.exp(1j * (k[:, 0] * d[2] + k[:, 1] * d[1] + k[:, 2] * d[0]))) / (nz * ny * nx)
        errs.append(abs(cfull[p] - w))
    et = max(errs) / abs(cfull[0, 0, 0])
    out = torch.empty(shape, dtype=torch.complex64, device="cuda")
    hq().toeplitz_normal3d(plan, x, out)
    ref = torch.empty(shape, dtype=torch.complex64, device="cuda")
    hq().adjoint3d(plan, y, ref)
    en = rel(to_host(out), to_host(ref))
    print(f"128^3 x {L} coils, {M} points: forward {ef:.2e}, adjoint {ea:.2e}, kernel {et:.2e}, "
          f"Toeplitz vs A^H(A x) {en:.2e}")
    assert ef <= 1e-4 and ea <= 1e-4 and et <= 1e-5 and en <= 1e-4


@pytest.mark.parametrize("W,L", [(5, 1), (7, 2), (8, 3), (4, 16)])
def test_volume_widths_coils_and_edge_points(W, L):
    """Odd widths (5, 7), the widest kernel (8: two-coil spreading chunks), one
    and two coils, and points exactly at -pi, at the k-space centre and
    repeated: forward and adjoint against the gridding oracle, A^H A against
    the exact embedding."""
    shape = (8, 16, 16)
    base = synth.traj_stack_of_spirals(8, 2, 128, 16)
    edge = np.array([[-np.pi, -np.pi, -np.pi], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0], [np.pi - 1e-7, -np.pi, 0.5],
                     [-np.pi, 1.0, np.pi - 1e-7]], dtype=np.float32)
    c = q(dict(shape=shape, L=L, W=W, sigma=2.0, x=synth.phantom3d(6, shape), smaps=synth.coil_maps3d(6, shape, L),
               traj=np.concatenate([base, edge])))
    plan, _, _ = plan_of(c)
    M = c["traj"].shape[0]
    y = torch.empty((L, M), dtype=torch.complex64, device="cuda")
    hq().forward3d(plan, to_dev(c["x"]), y)
    ef = rel(to_host(y), nufft3d.forward(c["x"], c["smaps"], c["traj"], W, 2.0))
    yin = synth.complex_noise(3, (L, M)).astype(np.complex64).astype(np.complex128)
    xa = torch.empty(shape, dtype=torch.complex64, device="cuda")
    hq().adjoint3d(plan, to_dev(yin), xa)
    ea = rel(to_host(xa), nufft3d.adjoint(yin, c["smaps"], c["traj"], W, 2.0))
    K = nufft3d.khat(nufft3d.kernel(c["traj"], shape))
    out = torch.empty(shape, dtype=torch.complex64, device="cuda")
    hq().toeplitz_normal3d(plan, to_dev(c["x"]), out)
    et = rel(to_host(out), nufft3d.normal(c["x"], c["smaps"], K))
    print(f"W={W} L={L}: forward {ef:.2e}, adjoint {ea:.2e}, A^H A {et:.2e}")
    assert ef <= 1e-5 and ea <= 1e-5 and et <= 1e-5


def test_volume_192_largest_transforms():
    """192^3 x 2 coils: 384-point NUFFT / Toeplitz transforms and 768-point
    kernel gridding (the largest sizes), no density preconditioner (192 is not
    a transform size).  Sampled forward against the exact NUDFT sum, A^H A
    against the GPU's own A^H(A x), and the plain CG solve's true residual
    measured with that A^H A."""
    shape, L = (192, 192, 192), 2
    c = q(dict(shape=shape, L=L, W=4, sigma=2.0, x=synth.phantom3d(7, shape), smaps=synth.coil_maps3d(7, shape, L),
               traj=synth.traj_stack_of_spirals(64, 4, 512, 192)))
    plan, _, _ = plan_of(c)
    M = c["traj"].shape[0]
    x = to_dev(c["x"])
    y = torch.empty((L, M), dtype=torch.complex64, device="cuda")
    hq().forward3d(plan, x, y)
    yh = to_host(y)
    rng = np.random.default_rng(17)
    k = c["traj"].astype(np.float64)
    ez, ey, ex = (np.arange(n) - n // 2 for n in shape)
    v = c["smaps"] * c["x"]
    got, want = [], []
    for j in rng.choice(M, 8, replace=False):
        t = np.einsum("lzyx,x->lzy", v, np.exp(-1j * k[j, 0] * ex))
        t = np.einsum("lzy,y->lz", t, np.exp(-1j * k[j, 1] * ey))
        want.append(np.einsum("lz,z->l", t, np.exp(-1j * k[j, 2] * ez)) / math.sqrt(float(np.prod(shape))))
        got.append(yh[:, j])
    ef = rel(np.array(got), np.array(want))
    out = torch.empty(shape, dtype=torch.complex64, device="cuda")
    hq().toeplitz_normal3d(plan, x, out)
    ref = torch.empty(shape, dtype=torch.complex64, device="cuda")
    hq().adjoint3d(plan, y, ref)
    en = rel(to_host(out), to_host(ref))
    xs = torch.zeros(shape, dtype=torch.complex64, device="cuda")
    info = hq().dc_solve3d(plan, 1.0, 1e-2, ref, xs, max_iter=100, rel_tol=1e-3, precond=hq().HQS_PRECOND_NONE)
    hx = torch.empty_like(xs)
    hq().toeplitz_normal3d(plan, xs, hx)
    res = rel(to_host(hx) + 1e-2 * to_host(xs), to_host(ref))
    print(f"192^3 x {L} coils, {M} points: forward {ef:.2e}, Toeplitz vs A^H(A x) {en:.2e}; "
          f"CG {info.iterations} iterations, residual {res:.2e}")
    # W = 4: each gridding direction carries ~7e-4 (oracle pins), so A^H(A x) differs from the
    # Toeplitz product (kernel gridded at width 8) by up to ~1.5e-3
    assert ef <= 2e-3 and en <= 3e-3 and info.rc == hq().HQS_OK and res <= 2e-3


# ------------------------------------------------------------------ HQS on volumes
def test_gaussian_denoise3d_matches_oracle():
    rng = np.random.default_rng(31)
    v = (rng.normal(size=(8, 12, 16)) + 1j * rng.normal(size=(8, 12, 16))).astype(np.complex64)
    out = torch.empty(v.shape, dtype=torch.complex64, device="cuda")
    for s_, gauss in ((1.3, None), (0.6, (1.5, 0.3)), (0.05, None)):
        hq().gaussian_denoise3d(to_dev(v), out, s_, gauss=gauss)
        sd = s_ if gauss is None else gauss[0] * s_ / gauss[1]
        e = rel(to_host(out), ohqs.gaussian_denoise(v.astype(np.complex128), sd))
        assert e <= 1e-6, (s_, e)
    # in place
    x = to_dev(v)
    hq().gaussian_denoise3d(x, x, 1.3)
    assert rel(to_host(x), ohqs.gaussian_denoise(v.astype(np.complex128), 1.3)) <= 1e-6


def test_hqs_run3d_matches_oracle():
    """Annealed HQS on a volume, 6 outer x 5 PCG iterations, mu 1e-1 -> 1e-3,
    Gaussian smoothing.  As for the 2D run, truncated warm-started CG amplifies
    rounding, so the bounds are derived from the oracle's own sensitivity:
    each step (started from the oracle's x_k) within max(1e-5, 4 d_k), d_k the
    oracle's one-step deviation when A^H y and x_k are perturbed by 2^-22
    relative (four float32 unit roundoffs: the GPU's gridded Toeplitz kernel
    adds ~1e-7 to the FP32 rounding); the whole run within 4x the oracle's
    deviation under the same perturbation of A^H y."""
    c = pc_case()
    plan, _, _ = plan_of(c)
    K, cg = 6, 5
    kern = nufft3d.kernel(c["traj"], c["shape"])
    Kh, lam = nufft3d.khat(kern), nufft3d.chan_symbol(kern, c["shape"])
    y = nufft3d.forward(c["x"], c["smaps"], c["traj"], c["W"], c["sigma"])
    y = (y + 0.02 * np.abs(y).max() * synth.complex_noise(7, y.shape)).astype(np.complex64).astype(np.complex128)
    mu = np.geomspace(1e-1, 1e-3, K).astype(np.float32)
    sigma = mu.copy()
    mu64, sg64 = mu.astype(np.float64), sigma.astype(np.float64)
    b0 = nufft3d.adjoint(y, c["smaps"], c["traj"], c["W"], c["sigma"])
    AHA = lambda v: nufft3d.normal(v, c["smaps"], Kh)
    run = lambda b, x0, k1, k0=0: ohqs.hqs(AHA, b, x0, mu64, sg64, k1, k0=k0, cg_iters=cg, lam=lam,
                                           precond_apply=nufft3d.precond_apply)
    want, _, hist = run(b0, np.zeros(c["shape"]), K)
    rng = np.random.default_rng(0)
    eps = 2.0 ** -22
    xk = np.zeros(c["shape"], dtype=np.complex128)
    for k in range(K):
        xg = to_dev(xk)
        hq().hqs_run3d(plan, to_dev(y), xg, mu, sigma, K=k + 1, k0=k, cg_iters=cg, gauss=(1.5, float(sigma[0])))
        step, _, _ = run(b0, xk, k + 1, k)
        pstep, _, _ = run(b0 * (1 + eps * rng.normal(size=b0.shape)), xk * (1 + eps * rng.normal(size=xk.shape)),
                          k + 1, k)
        tol_k = max(1e-5, 4 * rel(pstep, step))
        assert rel(to_host(xg), step) <= tol_k, (k, rel(to_host(xg), step), tol_k)
        xk = hist[k].astype(np.complex64).astype(np.complex128)
    x = torch.zeros(c["shape"], dtype=torch.complex64, device="cuda")
    hq().hqs_run3d(plan, to_dev(y), x, mu, sigma, K=K, cg_iters=cg, gauss=(1.5, float(sigma[0])))
    pert, _, _ = run(b0 * (1 + eps * rng.normal(size=b0.shape)), np.zeros(c["shape"]), K)
    bound = max(1e-5, 4 * rel(pert, want))
    err = rel(to_host(x), want)
    print(f"3D HQS {K}x{cg}: rel error to the oracle {err:.2e} (bound {bound:.2e}); "
          f"to the ground truth {rel(to_host(x), c['x']):.3f}")
    assert err <= bound, (err, bound)


def test_hqs_run3d_callback_and_failure():
    c = CASES["aniso"]()
    plan, _, _ = plan_of(c)
    y = to_dev(synth.complex_noise(2, (c["L"], c["traj"].shape[0])))
    calls = []

    def shrink(tin, tout, s):
        calls.append((tuple(tin.shape), s))
        tout.copy_(tin * 0.5)
        return 0

    x = torch.zeros(c["shape"], dtype=torch.complex64, device="cuda")
    hq().hqs_run3d(plan, y, x, [0.1, 0.05], [1.0, 0.5], cg_iters=3, denoiser=shrink)
    assert calls == [(c["shape"], 1.0), (c["shape"], 0.5)]
    with pytest.raises(hq().HqsError) as ei:
        hq().hqs_run3d(plan, y, x, [0.1], [1.0], cg_iters=3, denoiser=lambda a, b, s: 7)
    assert ei.value.status == hq().HQS_ERR_CALLBACK
