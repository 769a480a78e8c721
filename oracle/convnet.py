"""Small convolutional network used as a learned CG preconditioner
(test infrastructure, FP64).

The paper's denoisers are DRUNets (Sec. 3.2, 4.2); here a 4-layer 3x3 network
(2 real channels in and out, 32 hidden, ReLU) is used inside flexible CG for
the data-consistency solve.  Definitions:

  conv(x, W, b)[n, o, y, x] = b[o] + sum_i sum_{dy,dx in 0..2} W[o, i, dy, dx] * xp[n, i, y+dy, x+dx]
  (cross-correlation with one pixel of zero padding, xp the padded input)
  net(x) = conv4(relu(conv3(relu(conv2(relu(conv1(x)))))))

Loss on a batch: mean over samples of ||net(x_n) - t_n||^2 / ||t_n||^2.
Adam: m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2; p -= lr (m/(1-b1^t)) / (sqrt(v/(1-b2^t)) + eps).
The learned preconditioner: z = zdc + s net(zdc / s), zdc the DC-preconditioned
residual, s its root-mean-square over the complex pixels; the two network
channels are the real and imaginary parts.
"""
from __future__ import annotations

import math

import numpy as np

from . import toeplitz

LAYERS = [(2, 32), (32, 32), (32, 32), (32, 2)]


def num_params(layers=LAYERS) -> int:
    return sum(co * ci * 9 + co for ci, co in layers)


def init_params(seed: int, layers=LAYERS):
    """He-normal weights, zero biases, last layer zero (the network starts as 0)."""
    rng = np.random.default_rng(seed)
    params = []
    for li, (ci, co) in enumerate(layers):
        if li == len(layers) - 1:
            W = np.zeros((co, ci, 3, 3))
        else:
            W = rng.normal(size=(co, ci, 3, 3)) * math.sqrt(2.0 / (ci * 9))
        params.append((W, np.zeros(co)))
    return params


def flatten(params) -> np.ndarray:
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params])


def unflatten(vec, layers=LAYERS):
    out, k = [], 0
    for ci, co in layers:
        W = np.asarray(vec[k:k + co * ci * 9], dtype=np.float64).reshape(co, ci, 3, 3)
        k += co * ci * 9
        b = np.asarray(vec[k:k + co], dtype=np.float64)
        k += co
        out.append((W, b))
    return out


def conv3x3(x, W, b):
    """x (N, ci, H, W) -> (N, co, H, W)."""
    N, ci, H, Wd = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    out = np.zeros((N, W.shape[0], H, Wd))
    for dy in range(3):
        for dx in range(3):
            patch = xp[:, :, dy:dy + H, dx:dx + Wd]            # (N, ci, H, W)
            out += np.einsum("oi,nihw->nohw", W[:, :, dy, dx], patch)
    return out + b[None, :, None, None]


def conv3x3_input_grad(dz, W):
    """Gradient of conv3x3 w.r.t. its input: (N, co, H, W) -> (N, ci, H, W)."""
    N, co, H, Wd = dz.shape
    dxp = np.zeros((N, W.shape[1], H + 2, Wd + 2))
    for dy in range(3):
        for dx in range(3):
            dxp[:, :, dy:dy + H, dx:dx + Wd] += np.einsum("oi,nohw->nihw", W[:, :, dy, dx], dz)
    return dxp[:, :, 1:H + 1, 1:Wd + 1]


def conv3x3_weight_grad(x, dz):
    """Gradients of conv3x3 w.r.t. W (co, ci, 3, 3) and b (co,)."""
    N, ci, H, Wd = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    dW = np.zeros((dz.shape[1], ci, 3, 3))
    for dy in range(3):
        for dx in range(3):
            dW[:, :, dy, dx] = np.einsum("nohw,nihw->oi", dz, xp[:, :, dy:dy + H, dx:dx + Wd])
    return dW, dz.sum(axis=(0, 2, 3))


def forward(params, x):
    acts = [np.asarray(x, dtype=np.float64)]
    h = acts[0]
    for li, (W, b) in enumerate(params):
        z = conv3x3(h, W, b)
        h = z if li == len(params) - 1 else np.maximum(z, 0.0)
        acts.append(h)
    return h, acts


def loss_and_grad(params, x, t):
    """Mean relative squared error and its gradient (list of (dW, db))."""
    out, acts = forward(params, x)
    t = np.asarray(t, dtype=np.float64)
    N = x.shape[0]
    tn = np.sum(t.reshape(N, -1) ** 2, axis=1)
    diff = out - t
    loss = float(np.mean(np.sum(diff.reshape(N, -1) ** 2, axis=1) / tn))
    dz = 2.0 * diff / (N * tn[:, None, None, None])
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        W, b = params[li]
        dW, db = conv3x3_weight_grad(acts[li], dz)
        grads[li] = (dW, db)
        if li > 0:
            da = conv3x3_input_grad(dz, W)
            dz = da * (acts[li] > 0.0)
    return loss, grads


def adam_step(vec, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return vec - lr * mh / (np.sqrt(vh) + eps), m, v


def learned_precond(r, lam, a, b, params):
    """z = zdc + s * net(zdc / s) for one complex (n, n) residual."""
    zdc = toeplitz.precond_apply(r, lam, a, b)
    s = math.sqrt(float(np.mean(np.abs(zdc) ** 2)))
    if s == 0.0:
        return zdc
    x = np.stack([zdc.real / s, zdc.imag / s])[None]
    out, _ = forward(params, x)
    return zdc + s * (out[0, 0] + 1j * out[0, 1])
