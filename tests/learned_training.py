"""Training data and training loop for the learned CG preconditioner (test
and benchmark infrastructure: the tests and the learned-preconditioner
benchmark workload train networks with it; the product library itself only
runs the network's forward, backward and Adam kernels).

Pairs come from the plain solver (Sec. 3.4's data-consistency system with
P = Id): for a right-hand side b, x* is solved to a tight tolerance with
DC-preconditioned CG, and the CG iterates x_i give residuals r_i = b - H x_i
and errors e_i = x* - x_i (H e_i = r_i).  The network sees the DC-
preconditioned residual zdc_i / s_i and learns (e_i - zdc_i) / s_i, so that
z = zdc + s net(zdc / s) approximates H^-1 r.  Training uses random crops
(the network is convolutional) and the library's Adam step.  All operator
work runs in the library; torch only slices and stacks tensors.
"""
from __future__ import annotations

import numpy as np
import torch

import paper_2411_01955_gb300 as hq


LAYERS = ((2, 32), (32, 32), (32, 32), (32, 2))   # (in, out) channels of the 3x3 convolutions


def initial_params(seed=0):
    """Flat float32 parameters in the library's layout (per layer: weights
    [out][in][3][3], then biases): He-normal hidden layers, zero biases, and a
    zero last layer, so the untrained network adds nothing to the DC
    preconditioner."""
    rng = np.random.default_rng(seed)
    parts = []
    for k, (ci, co) in enumerate(LAYERS):
        w = rng.normal(size=(co, ci, 3, 3)) * np.sqrt(2.0 / (ci * 9))
        if k == len(LAYERS) - 1:
            w = np.zeros_like(w)
        parts += [w.ravel(), np.zeros(co)]
    return np.concatenate(parts).astype(np.float32)


def residual(plan, mu, rhs, x):
    """r = rhs - (A^H A + mu I) x."""
    ax = torch.empty_like(x)
    hq.toeplitz_normal(plan, x, ax)
    return rhs - ax - mu * x


def solve_pairs(plan, rhs, mu, iterates=12, tol_ref=1e-6):
    """(r_i, e_i) for the first `iterates` DC-PCG iterates from x = 0."""
    xs = torch.zeros_like(rhs)
    hq.dc_solve(plan, 1.0, mu, rhs, xs, max_iter=hq.HQS_MAX_ITERS, rel_tol=tol_ref,
                mode=hq.HQS_SOLVE_FUSED | hq.HQS_SOLVE_X0_ZERO, check=False)
    pairs = []
    for i in range(iterates):
        xi = torch.zeros_like(rhs)
        hq.dc_solve(plan, 1.0, mu, rhs, xi, max_iter=i, rel_tol=0.0,
                    mode=hq.HQS_SOLVE_FUSED | hq.HQS_SOLVE_X0_ZERO, check=False)
        pairs.append((residual(plan, mu, rhs, xi), xs - xi))
    return pairs


def to_planar(z):
    return torch.stack([z.real, z.imag]).contiguous()


def network_example(plan, mu, r, e):
    """(input, target) planar (2, n, n) for one pair: zdc/s and (e - zdc)/s."""
    zdc = torch.empty_like(r)
    hq.precond_apply(plan, 1.0, mu, r, zdc)
    s = float(torch.sqrt(torch.mean(torch.abs(zdc) ** 2)))
    s = s if s > 0 else 1.0
    return to_planar(zdc / s), to_planar((e - zdc) / s)


def random_crops(examples, batch, crop, rng):
    xs, ts = [], []
    for _ in range(batch):
        inp, tgt = examples[int(rng.integers(len(examples)))]
        n = inp.shape[-1]
        y0, x0 = (int(v) for v in rng.integers(0, n - crop + 1, size=2))
        xs.append(inp[:, y0:y0 + crop, x0:x0 + crop])
        ts.append(tgt[:, y0:y0 + crop, x0:x0 + crop])
    return torch.stack(xs).contiguous(), torch.stack(ts).contiguous()


def train(net, examples, steps=400, batch=16, crop=64, lr=1e-3, seed=0, log_every=0):
    rng = np.random.default_rng(seed)
    losses = []
    for it in range(steps):
        x, t = random_crops(examples, batch, crop, rng)
        losses.append(net.train_step(x, t, lr))
        if log_every and it % log_every == 0:
            print(f"step {it} loss {losses[-1]:.4f}", flush=True)
    return losses


def heldout_loss(net, examples):
    """Mean relative error of the learned correction on full-size examples
    (1.0 = no better than the DC preconditioner alone)."""
    vals = []
    for inp, tgt in examples:
        out = net.forward(inp[None].contiguous())[0]
        vals.append(float(torch.sum((out - tgt) ** 2) / torch.sum(tgt ** 2)))
    return float(np.mean(vals))


# ---------------------------------------------------------------- residual loss
# The flexible CG this preconditioner serves converges fast when ||I - H M||
# is small on the residuals it meets, so the second training mode minimises
# the preconditioned residual itself: for z = zdc + s net(zdc / s),
#     loss = ||r - H z||^2 / ||r||^2,   dloss/dz = -2 H (r - H z) / ||r||^2
# (H Hermitian), and dloss/d(net output) = s dloss/dz.  Full images are used
# (H is a global operator); the two A^H A applies per example run in the
# library, the network's backward in the library from that output gradient.

def from_planar(p):
    return torch.complex(p[0], p[1])


def apply_H(plan, mu, v):
    out = torch.empty_like(v)
    hq.toeplitz_normal(plan, v, out)
    return out + mu * v


def residual_example(plan, mu, r):
    """Example of the residual-loss mode: the DC-preconditioned residual zdc,
    its RMS s and the network input zdc / s (planar)."""
    zdc = torch.empty_like(r)
    hq.precond_apply(plan, 1.0, mu, r, zdc)
    s = float(torch.sqrt(torch.mean(torch.abs(zdc) ** 2)))
    s = s if s > 0 else 1.0
    return dict(plan=plan, mu=mu, r=r, zdc=zdc, s=s, inp=to_planar(zdc / s))


def residual_loss(net, ex, out=None):
    """Preconditioned residual ||r - H z||^2 / ||r||^2 of one example, and the
    gradient with respect to the network output (planar)."""
    if out is None:
        out = net.forward(ex["inp"][None].contiguous())[0]
    z = ex["zdc"] + ex["s"] * from_planar(out)
    res = ex["r"] - apply_H(ex["plan"], ex["mu"], z)
    rn = float(torch.sum(torch.abs(ex["r"]) ** 2))
    loss = float(torch.sum(torch.abs(res) ** 2)) / rn
    g = -2.0 * apply_H(ex["plan"], ex["mu"], res) / rn
    return loss, ex["s"] * to_planar(g)


def train_residual(net, examples, steps=300, batch=8, lr=5e-4, seed=0, log_every=0):
    """Adam on the mean preconditioned residual over random batches of
    full-size examples (all of one image size)."""
    rng = np.random.default_rng(seed)
    losses = []
    for it in range(steps):
        idx = rng.integers(len(examples), size=batch)
        exs = [examples[int(i)] for i in idx]
        x = torch.stack([e["inp"] for e in exs]).contiguous()
        out = net.forward(x)
        dys, ls = [], []
        for k, e in enumerate(exs):
            l, dy = residual_loss(net, e, out[k])
            ls.append(l)
            dys.append(dy / batch)
        net.train_step_dy(x, torch.stack(dys).contiguous(), lr)
        losses.append(float(np.mean(ls)))
        if log_every and it % log_every == 0:
            print(f"step {it} residual loss {losses[-1]:.4f}", flush=True)
    return losses


def heldout_residual(net, examples):
    """Mean ||r - H M r||^2 / ||r||^2 over examples (M: DC + network)."""
    return float(np.mean([residual_loss(net, e)[0] for e in examples]))


# ---------------------------------------------------------------- conv denoiser
def denoiser_examples(images, sigmas, seed=0):
    """(input, target) pairs for D_sigma(v) = v - sigma net(v / sigma): v = x + sigma n
    with complex Gaussian n (unit variance per part); input v / sigma, target n."""
    rng = np.random.default_rng(seed)
    out = []
    for x in images:
        s = float(rng.choice(sigmas)) if np.ndim(sigmas) else float(sigmas)
        noise = torch.complex(torch.from_numpy(rng.normal(size=x.shape).astype(np.float32)),
                              torch.from_numpy(rng.normal(size=x.shape).astype(np.float32))).to(x.device)
        v = x + s * noise
        out.append((to_planar(v / s), to_planar(noise)))
    return out
