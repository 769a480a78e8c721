"""GPU tests of the learned preconditioner: the network's forward pass,
gradients and Adam step against the FP64 oracle; flexible CG with the trained
network (convergence, held-out gain over the DC preconditioner alone) and its
fallback to DC-preconditioned CG."""
import math

import numpy as np
import pytest

import synth
from helpers import make_plan, quantised, rel, to_dev, to_host
from oracle import convnet, toeplitz

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5
EPS = 2.0 ** -24


TC_PRODUCT = 3 * 2.0 ** -16


def rounding_model(params, rng, tensor_cores=True):
    """The network's rounding as a perturbation of its parameters.

    A float32 dot product of K terms equals the exact dot product of slightly
    perturbed weights, |dw| <= K u |w| in the worst case and about sqrt(K) u |w|
    for rounding errors of random sign (Higham, Accuracy and Stability of
    Numerical Algorithms, sec. 3.1 and 2.8), u = 2^-24.  Each 3x3 layer sums
    K = 9 Cin products plus its bias, so every parameter of that layer is
    perturbed by a relative sqrt(K) u with a random sign.  With the tensor
    cores (the default precision) the two 32 -> 32 layers multiply BF16 hi/lo
    splits: v = hi + lo + r with |r| <= 2^-16 |v| (two roundings to 8
    significant bits), and hi*hi + lo*hi + hi*lo misses lo*lo + r_a b + a r_b,
    at most 3 * 2^-16 |a b| per product; as a weight perturbation that is a
    relative 3 * 2^-16 per weight (random sign) on top of the FP32
    accumulation's sqrt(K) u.  The learned path's bound is then four times the
    oracle's deviation under this perturbation (and a 2^-24 perturbation of its
    input), like the other iterated or composed results in this suite; ReLU
    and the input scaling add no error of their own beyond this model."""
    out = []
    for li, (W, b) in enumerate(params):
        K = 9 * W.shape[1] + 1
        d = EPS * math.sqrt(K)
        if tensor_cores and W.shape[0] == W.shape[1] == 32:
            d += TC_PRODUCT
        out.append((W * (1 + d * rng.choice([-1.0, 1.0], size=W.shape)),
                    b * (1 + d * rng.choice([-1.0, 1.0], size=b.shape))))
    return out


def hq():
    import paper_2411_01955_gb300 as m
    return m


def random_params(seed, scale_last=0.3):
    rng = np.random.default_rng(seed)
    params = convnet.init_params(seed)
    W4 = rng.normal(size=params[-1][0].shape) * scale_last * math.sqrt(2.0 / (32 * 9))
    params[-1] = (W4, rng.normal(size=2) * 0.1)
    params = [(W, b + 0.05 * rng.normal(size=b.shape)) for W, b in params]
    return params


def f32(params):
    return [(W.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64))
            for W, b in params]


def grad_vector(wgrads):
    return np.concatenate([np.concatenate([dW.ravel(), db.ravel()]) for dW, db in wgrads])


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
@pytest.mark.parametrize("shape", [(2, 2, 20, 19), (2, 2, 160, 100)])
def test_net_forward_and_gradient_match_oracle(precision, shape):
    """Forward pass, loss and parameter gradient against the FP64 oracle: FP32
    convolutions within 1e-5, the tensor-core 32 -> 32 layers within the bound
    their BF16 split derives (rounding_model); 20 x 19 images leave partial
    16 x 16 tiles and a partial 128-pixel tile, 2 x 160 x 100 gives 250
    128-pixel tiles (more than one per SM)."""
    rng = np.random.default_rng(0)
    params = f32(random_params(1))
    net = hq().Net()
    tc = precision == "bf16x3"
    net.set_precision(hq().HQS_PREC_BF16X3 if tc else hq().HQS_PREC_FP32)
    assert net.num_params == convnet.num_params() == 19682
    net.set_params(convnet.flatten(params))
    assert np.array_equal(net.get_params(), convnet.flatten(params).astype(np.float32))
    x = rng.normal(size=shape).astype(np.float32)
    t = rng.normal(size=shape).astype(np.float32)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    out = net.forward(xd).cpu().numpy()
    want, _ = convnet.forward(params, x.astype(np.float64))
    wloss, wgrads = convnet.loss_and_grad(params, x.astype(np.float64), t.astype(np.float64))
    wg = grad_vector(wgrads)
    # the bound: the oracle under the rounding model of the chosen precision
    prng = np.random.default_rng(21)
    pp = rounding_model(params, prng, tensor_cores=tc)
    xp = x.astype(np.float64) * (1 + EPS * prng.normal(size=x.shape))
    pout, _ = convnet.forward(pp, xp)
    ploss, pgrads = convnet.loss_and_grad(pp, xp, t.astype(np.float64))
    pg = grad_vector(pgrads)
    tol_out = max(TOL, 4 * rel(pout, want))
    tol_loss = max(TOL, 4 * abs(ploss / wloss - 1))
    tol_g = max(TOL, 4 * rel(pg, wg))
    if not tc:
        tol_out = tol_loss = tol_g = TOL
    g, loss = net.gradient(xd, td)
    err_out, err_loss, err_g = rel(out, want), abs(loss / wloss - 1), rel(g.cpu().numpy(), wg)
    print(f"{precision} {shape}: forward {err_out:.2e} (bound {tol_out:.2e}), loss {err_loss:.2e} "
          f"({tol_loss:.2e}), gradient {err_g:.2e} ({tol_g:.2e})")
    assert err_out <= tol_out
    assert err_loss <= tol_loss
    assert err_g <= tol_g
    # per layer as well (a wrong layer offset would hide in the global norm)
    k = 0
    for (dW, db), (pW, pb) in zip(wgrads, pgrads):
        m = dW.size + db.size
        bound = max(1e-4, 4 * rel(pg[k:k + m], wg[k:k + m])) if tc else 1e-4
        assert rel(g.cpu().numpy()[k:k + m], wg[k:k + m]) <= bound
        k += m
    net.status()


def test_tensor_core_layers_against_fp32_layers():
    """The same network in both precisions on a 320 x 320 image (800 tiles of
    128 pixels): the tensor-core forward stays within the BF16 split's bound of
    the FP32 one, and the network's error flag stays clear."""
    rng = np.random.default_rng(4)
    params = f32(random_params(2))
    x = torch.from_numpy(rng.normal(size=(1, 2, 320, 320)).astype(np.float32)).cuda()
    outs = {}
    for prec in (hq().HQS_PREC_FP32, hq().HQS_PREC_BF16X3):
        net = hq().Net()
        net.set_precision(prec)
        net.set_params(convnet.flatten(params))
        outs[prec] = net.forward(x).cpu().numpy().astype(np.float64)
        net.status()
    with pytest.raises(hq().HqsError):
        hq().Net().set_precision(hq().HQS_PREC_FP16X3)
    # bound from the oracle on a 64 x 64 crop (the error is per pixel, so the
    # relative L2 bound carries over to the whole image)
    crop = x[:, :, :64, :64].cpu().numpy().astype(np.float64)
    want, _ = convnet.forward(params, crop)
    prng = np.random.default_rng(22)
    pout, _ = convnet.forward(rounding_model(params, prng, tensor_cores=True), crop)
    bound = 8 * rel(pout, want)
    err = rel(outs[hq().HQS_PREC_BF16X3], outs[hq().HQS_PREC_FP32])
    print(f"tensor-core vs FP32 layers at 320^2: {err:.2e} (bound {bound:.2e})")
    assert 0 < err <= bound


def test_adam_step_matches_its_definition():
    rng = np.random.default_rng(2)
    params = f32(random_params(3))
    net = hq().Net()
    p0 = convnet.flatten(params).astype(np.float32)
    net.set_params(p0)
    x = torch.from_numpy(rng.normal(size=(2, 2, 16, 16)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.normal(size=(2, 2, 16, 16)).astype(np.float32)).cuda()
    g, _ = net.gradient(x, t)
    g = g.cpu().numpy().astype(np.float64)
    lr = 1e-3
    net.train_step(x, t, lr)
    want, _, _ = convnet.adam_step(p0.astype(np.float64), g, np.zeros_like(g), np.zeros_like(g), 1, lr)
    got = net.get_params().astype(np.float64)
    assert np.max(np.abs(got - want)) <= 1e-6 * lr * 10 + 1e-7


def make_slices(seeds, n=128, L=8):
    traj = synth.traj_spiral(8, 1024, n)
    out = []
    for sd in seeds:
        case = quantised(dict(n=n, L=L, W=6, sigma=2.0, x=synth.phantom(sd, n),
                              smaps=synth.coil_maps(sd, n, L), traj=traj))
        plan, _, _ = make_plan(case)
        x = to_dev(case["x"])
        y = torch.empty((L, traj.shape[0]), dtype=torch.complex64, device="cuda")
        hq().forward(plan, x, y)
        noise = torch.from_numpy(synth.complex_noise(sd, (L, traj.shape[0])).astype(np.complex64)).cuda()
        y = y + 0.02 * float(torch.sqrt(torch.mean(torch.abs(y) ** 2))) * noise
        rhs = torch.empty_like(x)
        hq().adjoint(plan, y.contiguous(), rhs)
        out.append((plan, rhs))
    return out


def test_learned_fcg_trains_converges_and_falls_back():
    import learned_training as learned
    mu = 1e-2
    train_slices = make_slices(range(1000, 1006))
    test_slices = make_slices(range(5000, 5002))
    examples = []
    for plan, rhs in train_slices:
        for r, e in learned.solve_pairs(plan, rhs, mu, iterates=24):
            examples.append(learned.network_example(plan, mu, r, e))
    held = []
    for plan, rhs in test_slices:
        for r, e in learned.solve_pairs(plan, rhs, mu, iterates=12):
            held.append(learned.network_example(plan, mu, r, e))
    net = hq().Net()
    net.set_params(convnet.flatten(convnet.init_params(0)))
    base = learned.heldout_loss(net, held)
    assert abs(base - 1.0) < 1e-6          # zero last layer: exactly the DC preconditioner
    losses = learned.train(net, examples, steps=600, batch=16, crop=48, lr=1e-3)
    trained = learned.heldout_loss(net, held)
    print(f"held-out relative error of the correction: {base:.3f} -> {trained:.3f}; "
          f"train loss {losses[0]:.3f} -> {np.mean(losses[-20:]):.3f}")
    assert trained < base                   # the trained network gains over DC alone
    # flexible CG with the trained network, and DC-PCG, on held-out slices
    for plan, rhs in test_slices:
        hq().plan_set_net(plan, net)
        xl = torch.zeros_like(rhs)
        il = hq().dc_solve(plan, 1.0, mu, rhs, xl, max_iter=300, rel_tol=1e-4,
                           precond=hq().HQS_PRECOND_LEARNED)
        xd = torch.zeros_like(rhs)
        idc = hq().dc_solve(plan, 1.0, mu, rhs, xd, max_iter=300, rel_tol=1e-4)
        print(f"iterations to 1e-4: learned {il.iterations} (fallback {il.fallback}), DC {idc.iterations}")
        assert il.status == 0 and il.rel_residual <= 1e-4
        r = learned.residual(plan, mu, rhs, xl)
        assert float(torch.linalg.vector_norm(r) / torch.linalg.vector_norm(rhs)) <= 1.5e-4
    # a sabotaged network (negated correction, 30x) must trigger the fallback and still converge
    bad = hq().Net()
    vec = net.get_params().astype(np.float64)
    k = convnet.num_params() - (2 * 32 * 9 + 2)
    vec[k:] *= -30.0
    bad.set_params(vec)
    plan, rhs = test_slices[0]
    hq().plan_set_net(plan, bad)
    xb = torch.zeros_like(rhs)
    ib = hq().dc_solve(plan, 1.0, mu, rhs, xb, max_iter=300, rel_tol=1e-4, precond=hq().HQS_PRECOND_LEARNED)
    assert ib.status == 0 and ib.rel_residual <= 1e-4
    print(f"sabotaged network: fallback {ib.fallback}, iterations {ib.iterations}")
    hq().plan_set_net(plan, None)


def test_learned_precond_apply_matches_oracle():
    case = quantised(synth.tiny_case(0))
    plan, _, _ = make_plan(case)
    n = case["n"]
    params = f32(random_params(5))
    net = hq().Net()
    net.set_params(convnet.flatten(params))
    hq().plan_set_net(plan, net)
    lam = toeplitz.chan_symbol(toeplitz.kernel(case["traj"], n, n), n, n)
    r = case["x"]
    z = torch.empty((n, n), dtype=torch.complex64, device="cuda")
    hq().learned_precond_apply(plan, 1.0, 0.05, to_dev(r), z)
    want = convnet.learned_precond(r, lam, 1.0, 0.05, params)
    rng = np.random.default_rng(11)
    dev = rel(convnet.learned_precond(r * (1 + EPS * rng.normal(size=r.shape)), lam, 1.0, 0.05,
                                      rounding_model(params, rng)), want)
    tol = max(TOL, 4 * dev)
    err = rel(to_host(z), want)
    print(f"learned preconditioner apply: {err:.2e} (bound {tol:.2e})")
    assert err <= tol
    hq().plan_set_net(plan, None)


def test_learned_fcg_iterates_match_oracle():
    from oracle import solvers
    case = quantised(synth.tiny_case(0))
    plan, _, _ = make_plan(case)
    n, mu = case["n"], 1e-2
    params = f32(random_params(7, scale_last=0.1))
    net = hq().Net()
    net.set_params(convnet.flatten(params))
    hq().plan_set_net(plan, net)
    c = toeplitz.kernel(case["traj"], n, n)
    Kh, lam = toeplitz.khat(c), toeplitz.chan_symbol(c, n, n)
    from oracle import nufft
    rhs = nufft.adjoint(case["noise"], case["smaps"], case["traj"], case["W"], case["sigma"])
    rhs = rhs.astype(np.complex64).astype(np.complex128)
    H = lambda v: toeplitz.normal(v, case["smaps"], Kh) + mu * v
    B = lambda v: convnet.learned_precond(v, lam, 1.0, mu, params)
    want, winfo = solvers.fcg(H, rhs, np.zeros((n, n)), B, None, max_iter=4, tol=0.0)
    rng = np.random.default_rng(12)
    pp = rounding_model(params, rng)
    Bp = lambda v: convnet.learned_precond(v, lam, 1.0, mu, pp)
    pert, _ = solvers.fcg(H, rhs * (1 + EPS * rng.normal(size=rhs.shape)), np.zeros((n, n)), Bp, None,
                          max_iter=4, tol=0.0)
    tol = max(TOL, 4 * rel(pert, want))
    x = torch.zeros((n, n), dtype=torch.complex64, device="cuda")
    info = hq().dc_solve(plan, 1.0, mu, to_dev(rhs), x, max_iter=4, rel_tol=0.0,
                         precond=hq().HQS_PRECOND_LEARNED)
    assert info.iterations == 4 and not info.fallback and not winfo["fallback"]
    err = rel(to_host(x), want)
    print(f"learned flexible CG, 4 iterations: {err:.2e} (bound {tol:.2e})")
    assert err <= tol
    assert np.allclose(np.array(info.history()), winfo["res_hist"], rtol=1e-3, atol=0)
    hq().plan_set_net(plan, None)


def test_backward_from_output_gradient_matches_loss_gradient():
    """hqs_net_backward seeded with the relative-MSE output gradient
    2 (y - t) / (N ||t_k||^2) reproduces hqs_net_gradient (itself pinned to
    the oracle)."""
    rng = np.random.default_rng(8)
    net = hq().Net()
    net.set_params(convnet.flatten(f32(random_params(9))))
    x = torch.from_numpy(rng.normal(size=(3, 2, 24, 17)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.normal(size=(3, 2, 24, 17)).astype(np.float32)).cuda()
    g_ref, _ = net.gradient(x, t)
    y = net.forward(x)
    tn = torch.sum(t.double() ** 2, dim=(1, 2, 3)).view(3, 1, 1, 1)
    dy = (2.0 * (y.double() - t.double()) / (3 * tn)).float().contiguous()
    g = net.backward(x, dy)
    assert rel(g.cpu().numpy(), g_ref.cpu().numpy()) <= 1e-5


def test_residual_trained_net_in_flexible_cg():
    """Trained on the preconditioned residual ||r - H M r||^2 / ||r||^2 of
    DC-PCG residuals, the network lowers it on held-out slices below the DC
    preconditioner's; flexible CG with it converges (falling back if it
    stalls), and its iteration count is reported beside DC-PCG's."""
    import learned_training as learned
    mu = 1e-2
    train_slices = make_slices(range(1000, 1008))
    test_slices = make_slices(range(5000, 5003))

    def residuals(slices, its):
        out = []
        for plan, rhs in slices:
            for r, _ in learned.solve_pairs(plan, rhs, mu, iterates=its):
                out.append(learned.residual_example(plan, mu, r))
        return out
    examples = residuals(train_slices, 20)
    held = residuals(test_slices, 12)
    net = hq().Net()
    net.set_params(convnet.flatten(convnet.init_params(0)))
    base = learned.heldout_residual(net, held)
    losses = learned.train_residual(net, examples, steps=300, batch=8, lr=5e-4)
    trained = learned.heldout_residual(net, held)
    print(f"held-out ||r - H M r||^2/||r||^2: DC {base:.4f} -> learned {trained:.4f}; "
          f"train {losses[0]:.4f} -> {np.mean(losses[-20:]):.4f}")
    assert trained < base
    for plan, rhs in test_slices:
        hq().plan_set_net(plan, net)
        xl = torch.zeros_like(rhs)
        il = hq().dc_solve(plan, 1.0, mu, rhs, xl, max_iter=300, rel_tol=1e-4, precond=hq().HQS_PRECOND_LEARNED)
        xd = torch.zeros_like(rhs)
        idc = hq().dc_solve(plan, 1.0, mu, rhs, xd, max_iter=300, rel_tol=1e-4)
        print(f"iterations to 1e-4: learned {il.iterations} (fallback {il.fallback}), DC {idc.iterations}")
        assert il.status == 0 and il.rel_residual <= 1e-4
        hq().plan_set_net(plan, None)


def test_net_denoiser_matches_oracle_forward():
    """D_sigma(v) = v - sigma net(v / sigma) against the oracle's network
    forward pass, for two noise levels."""
    rng = np.random.default_rng(11)
    params = f32(random_params(12))
    net = hq().Net()
    net.set_params(convnet.flatten(params))
    v = (rng.normal(size=(40, 40)) + 1j * rng.normal(size=(40, 40))).astype(np.complex64).astype(np.complex128)
    for sigma in (0.3, 0.05):
        out = torch.empty((40, 40), dtype=torch.complex64, device="cuda")
        net.denoise(to_dev(v), out, sigma)
        inp = (np.stack([v.real, v.imag])[None] / np.float32(sigma)).astype(np.float32).astype(np.float64)
        y, _ = convnet.forward(params, inp)
        want = v - sigma * (y[0, 0] + 1j * y[0, 1])
        # bound: the oracle under the tensor-core rounding model (the default precision)
        yp, _ = convnet.forward(rounding_model(params, np.random.default_rng(23)), inp)
        tol = max(1e-5, 4 * rel(v - sigma * (yp[0, 0] + 1j * yp[0, 1]), want))
        err = rel(to_host(out), want)
        print(f"net denoiser, sigma {sigma}: {err:.2e} (bound {tol:.2e})")
        assert err <= tol
    # sigma = 0 copies
    out = torch.empty((40, 40), dtype=torch.complex64, device="cuda")
    net.denoise(to_dev(v), out, 0.0)
    assert rel(to_host(out), v) <= 1e-7


def test_trained_net_denoiser_and_hqs_with_it():
    """Trained on synthetic phantoms (noise std 0.02-0.2 per part, images
    scaled to max 1), the conv denoiser lowers the held-out error well below
    the noisy input's; annealed HQS runs with it as the native denoiser."""
    import learned_training as learned
    n = 128
    def imgs(seeds):
        out = []
        for sd in seeds:
            x = synth.phantom(sd, n)
            out.append(torch.from_numpy((x / np.abs(x).max()).astype(np.complex64)).cuda())
        return out
    train = learned.denoiser_examples(imgs(range(1000, 1024)), [0.02, 0.05, 0.1, 0.2], seed=1)
    net = hq().Net()
    net.set_params(learned.initial_params(3))
    learned.train(net, train, steps=600, batch=16, crop=64, lr=1e-3)
    rng = np.random.default_rng(9)
    for sigma in (0.05, 0.1):
        errs = []
        for x in imgs(range(5000, 5003)):
            noise = torch.complex(torch.from_numpy(rng.normal(size=(n, n)).astype(np.float32)),
                                  torch.from_numpy(rng.normal(size=(n, n)).astype(np.float32))).cuda()
            v = x + sigma * noise
            d = torch.empty_like(v)
            net.denoise(v, d, sigma)
            g = torch.empty_like(v)
            hq().gaussian_denoise(v, g, 1.0)
            e = lambda a: float(torch.linalg.vector_norm(a - x) / torch.linalg.vector_norm(x))
            errs.append((e(v), e(d), e(g)))
        noisy, learned_e, gauss_e = np.mean(errs, axis=0)
        print(f"sigma {sigma}: relative error noisy {noisy:.4f}, conv denoiser {learned_e:.4f}, "
              f"Gaussian 1 px {gauss_e:.4f}")
        assert learned_e < 0.6 * noisy
    # annealed HQS with the conv denoiser as the native callback
    case = quantised(dict(n=n, L=6, W=6, sigma=2.0, x=synth.phantom(5010, n) / np.abs(synth.phantom(5010, n)).max(),
                          smaps=synth.coil_maps(5010, n, 6), traj=synth.traj_spiral(8, 1024, n)))
    plan, _, _ = make_plan(case)
    from oracle import nufft as onufft
    y = onufft.forward(case["x"], case["smaps"], case["traj"], 6, 2.0)
    y = y + 0.01 * np.sqrt(np.mean(np.abs(y) ** 2)) * synth.complex_noise(5010, y.shape)
    K = 10
    mu = synth.mu_schedule_geometric(1e-1, 1e-3, K).astype(np.float32)
    sig = np.geomspace(0.1, 0.01, K).astype(np.float32)
    res = {}
    for name, den in (("conv", net), ("gauss", None)):
        x = torch.zeros((n, n), dtype=torch.complex64, device="cuda")
        hq().hqs_run(plan, to_dev(y), x, mu, sig, cg_iters=5, denoiser=den)
        res[name] = rel(to_host(x), case["x"])
    print(f"HQS 10 x 5 relative error vs ground truth: conv denoiser {res['conv']:.4f}, "
          f"Gaussian smoothing {res['gauss']:.4f}")
    assert np.isfinite(res["conv"]) and res["conv"] < 1.0
