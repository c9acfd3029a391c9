"""FP64 CPU oracle of the learned warm start's convolutional network.

TEST INFRASTRUCTURE ONLY: like the rest of ``oracle/``, only the tests, the
package's smoke check and the benchmark's CPU legs use it; the CUDA path
never imports it, and it shares no code with the CUDA path.

The paper initialises the first frame with zero flows and names smarter
initialisation of the first frame as future work (Section 7, Limitations).
The warm start is a small convolutional network that maps the four
coarsest-level images of a quadruple to the coarsest level's six delta fields
(s, m, d, x and y each, on the warp grid), which then replace the zero
initialisation of the coarsest level (the mechanism the temporal transfer of
Section 5.3 uses for later frames). This module states the network and its
training arithmetic in plain numpy, in double precision:

  input   x0 = I - 1/2, I the four coarsest images [B, 4, 60, 80]
  layer   conv 3x3, zero padding 1, stride s, bias, then ReLU (not after the last)
          1: 4 -> 32, s 2 (60x80 -> 30x40)     4: 64 -> 64, s 1 (8x10)
          2: 32 -> 64, s 2 (30x40 -> 15x20)    5: 64 -> 32, s 1 (8x10)
          3: 64 -> 64, s 2 (15x20 -> 8x10)     6: 32 -> 6,  s 1 (8x10), linear
  output  [B, 6, 8, 10], component-major like the solver's fields
  loss    mean squared error over all B * 480 outputs
  update  Adam (Kingma and Ba, 2015) with bias correction

A convolution here is the cross-correlation
  y[b, o, i, j] = bias[o] + sum_{c, u, v} w[o, c, u, v] * xp[b, c, s*i + u, s*j + v]
with xp the input padded by one zero on every side, output size ceil(n / s).

Parity status: pinned (tests/test_oracle_net.py): the convolution against
scipy.signal.correlate2d, the backward pass and the whole loss gradient by
central finite differences, Adam by its closed form on constant gradients,
the input centring by a zero-bias network mapping mid-grey to zero.
"""

from __future__ import annotations

import numpy as np

# (in channels, out channels, stride, ReLU after)
LAYERS = ((4, 32, 2, True), (32, 64, 2, True), (64, 64, 2, True),
          (64, 64, 1, True), (64, 32, 1, True), (32, 6, 1, False))
IN_SHAPE = (4, 60, 80)
OUT_SHAPE = (6, 8, 10)


def out_size(n: int, stride: int) -> int:
    return (n + stride - 1) // stride


def conv2d(x: np.ndarray, w: np.ndarray, bias: np.ndarray, stride: int) -> np.ndarray:
    """Forward convolution (definition above); x [B, C, H, W], w [O, C, 3, 3]."""
    B, C, H, W = x.shape
    O = w.shape[0]
    Ho, Wo = out_size(H, stride), out_size(W, stride)
    xp = np.zeros((B, C, H + 2, W + 2))
    xp[:, :, 1:H + 1, 1:W + 1] = x
    y = np.zeros((B, O, Ho, Wo)) + bias[None, :, None, None]
    for u in range(3):
        for v in range(3):
            patch = xp[:, :, u:u + stride * (Ho - 1) + 1:stride, v:v + stride * (Wo - 1) + 1:stride]
            y += np.einsum("bchw,oc->bohw", patch, w[:, :, u, v])
    return y


def conv2d_backward(x: np.ndarray, w: np.ndarray, stride: int, dy: np.ndarray):
    """Gradients (dx, dw, dbias) of <dy, conv2d(x, w, bias, stride)>."""
    B, C, H, W = x.shape
    Ho, Wo = dy.shape[2], dy.shape[3]
    xp = np.zeros((B, C, H + 2, W + 2))
    xp[:, :, 1:H + 1, 1:W + 1] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for u in range(3):
        for v in range(3):
            sl = (slice(None), slice(None), slice(u, u + stride * (Ho - 1) + 1, stride),
                  slice(v, v + stride * (Wo - 1) + 1, stride))
            dw[:, :, u, v] = np.einsum("bohw,bchw->oc", dy, xp[sl])
            dxp[sl] += np.einsum("bohw,oc->bchw", dy, w[:, :, u, v])
    return dxp[:, :, 1:H + 1, 1:W + 1], dw, dy.sum(axis=(0, 2, 3))


def init_params(seed: int) -> list:
    """He-normal weights, zero biases, seeded: [(w, bias), ...] per layer."""
    rng = np.random.default_rng(seed)
    params = []
    for cin, cout, _, _ in LAYERS:
        std = np.sqrt(2.0 / (9 * cin))
        params.append((rng.standard_normal((cout, cin, 3, 3)) * std, np.zeros(cout)))
    return params


def forward(params, imgs: np.ndarray):
    """Network output [B, 6, 8, 10] and the activations the backward pass needs."""
    a = np.asarray(imgs, dtype=np.float64) - 0.5
    acts = [a]
    pre = []
    for (w, b), (_, _, stride, relu) in zip(params, LAYERS):
        z = conv2d(a, w, b, stride)
        pre.append(z)
        a = np.maximum(z, 0.0) if relu else z
        acts.append(a)
    return a, (acts, pre)


def loss_and_grads(params, imgs: np.ndarray, target: np.ndarray):
    """Mean squared error and its gradient with respect to every parameter."""
    y, (acts, pre) = forward(params, imgs)
    r = y - np.asarray(target, dtype=np.float64)
    loss = float(np.mean(r * r))
    g = 2.0 * r / r.size
    grads = [None] * len(params)
    for k in range(len(params) - 1, -1, -1):
        _, _, stride, relu = LAYERS[k]
        if relu:
            g = g * (pre[k] > 0.0)
        w, _ = params[k]
        dx, dw, db = conv2d_backward(acts[k], w, stride, g)
        grads[k] = (dw, db)
        g = dx
    return loss, grads


def adam_step(params, grads, state, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update of every tensor. state = (t, m, v) with m, v lists like
    params (zeros and t = 0 at the start); returns (new params, new state)."""
    t, m, v = state
    t += 1
    new_p, new_m, new_v = [], [], []
    for (p, gp), (mp, vp) in zip(zip(params, grads), zip(m, v)):
        out_p, out_m, out_v = [], [], []
        for x, g, mm, vv in zip(p, gp, mp, vp):
            mm = beta1 * mm + (1.0 - beta1) * g
            vv = beta2 * vv + (1.0 - beta2) * g * g
            mh = mm / (1.0 - beta1 ** t)
            vh = vv / (1.0 - beta2 ** t)
            out_p.append(x - lr * mh / (np.sqrt(vh) + eps))
            out_m.append(mm)
            out_v.append(vv)
        new_p.append(tuple(out_p))
        new_m.append(tuple(out_m))
        new_v.append(tuple(out_v))
    return new_p, (t, new_m, new_v)


def adam_state(params):
    zeros = [tuple(np.zeros_like(x) for x in p) for p in params]
    return 0, zeros, [tuple(np.zeros_like(x) for x in p) for p in params]
