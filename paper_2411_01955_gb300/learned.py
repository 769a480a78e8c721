"""Training data and training loop for the learned CG preconditioner.

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

from . import _lib as hq


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
