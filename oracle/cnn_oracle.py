"""FP64 CPU oracle for the learned warm start (a 6-layer 3x3 CNN).

TEST INFRASTRUCTURE ONLY (see ``firls_oracle``): used by tests and the
CPU legs of bench.py, never by the CUDA library.

The network maps the zero-filled reconstruction to a correction,
x1 = A^H b + CNN([Re A^H b, Im A^H b, mask]): five 3x3 'same' convolutions
with ReLU and a last 3x3 convolution to two channels (Re, Im).  Each
convolution is the definition written out,
    z[y, x, o] = b[o] + sum_{dy, dx in -1..1} sum_i a[y+dy, x+dx, i] w[dy+1, dx+1, i, o]
with zero padding, and its gradients follow by the chain rule.  Loss:
sum |x1 - x*|^2 (the sum rather than the mean, so gradients are O(1)).
"""
from __future__ import annotations

import numpy as np


def conv3x3(a, w, b):
    """a [B][H][W][Ci], w [3][3][Ci][Co], b [Co] -> z [B][H][W][Co]."""
    B, H, W, _ = a.shape
    ap = np.pad(a, ((0, 0), (1, 1), (1, 1), (0, 0)))
    z = np.broadcast_to(b, (B, H, W, w.shape[3])).astype(np.float64).copy()
    for ky in range(3):
        for kx in range(3):
            z += np.einsum("bhwi,io->bhwo", ap[:, ky:ky + H, kx:kx + W, :], w[ky, kx])
    return z


def conv3x3_backward(a, w, dz):
    """Gradients of sum(dz * conv3x3(a, w, b)) w.r.t. a, w and b."""
    B, H, W, _ = a.shape
    ap = np.pad(a, ((0, 0), (1, 1), (1, 1), (0, 0)))
    dap = np.zeros_like(ap, dtype=np.float64)
    dw = np.zeros_like(w, dtype=np.float64)
    for ky in range(3):
        for kx in range(3):
            dap[:, ky:ky + H, kx:kx + W, :] += np.einsum("bhwo,io->bhwi", dz, w[ky, kx])
            dw[ky, kx] = np.einsum("bhwi,bhwo->io", ap[:, ky:ky + H, kx:kx + W, :], dz)
    db = dz.sum(axis=(0, 1, 2))
    return dap[:, 1:-1, 1:-1, :], dw, db


def forward(params, inp):
    """Activations [inp, y1, ..., y5, out]; ReLU on all but the last layer."""
    acts = [inp]
    a = inp
    for l, (w, b) in enumerate(params):
        z = conv3x3(a, w, b)
        a = np.maximum(z, 0.0) if l < len(params) - 1 else z
        acts.append(a)
    return acts


def loss_and_grads(params, inp, atb, target):
    """Sum-of-squares loss of x1 = atb + out against target, and its gradients."""
    acts = forward(params, inp)
    out = acts[-1]
    x1 = atb + (out[..., 0] + 1j * out[..., 1])
    res = x1 - target
    loss = float(np.sum(np.abs(res) ** 2))
    dout = np.stack([2 * res.real, 2 * res.imag], axis=-1)
    grads = [None] * len(params)
    g = dout
    for l in reversed(range(len(params))):
        w, _ = params[l]
        if l < len(params) - 1:
            g = g * (acts[l + 1] > 0)
        da, dw, db = conv3x3_backward(acts[l], w, g)
        grads[l] = (dw, db)
        g = da
    return loss, grads, x1


def adam_step(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) of every weight and bias; state is
    {'t': steps taken, 'm': [...], 'v': [...]} and is updated in place."""
    state["t"] += 1
    t = state["t"]
    out = []
    for i, ((w, b), (gw, gb)) in enumerate(zip(params, grads)):
        new = []
        for j, (p, g) in enumerate(((w, gw), (b, gb))):
            m = state["m"][2 * i + j] = beta1 * state["m"][2 * i + j] + (1 - beta1) * g
            v = state["v"][2 * i + j] = beta2 * state["v"][2 * i + j] + (1 - beta2) * g * g
            mh = m / (1 - beta1 ** t)
            vh = v / (1 - beta2 ** t)
            new.append(p - lr * mh / (np.sqrt(vh) + eps))
        out.append(tuple(new))
    return out


def adam_init(params):
    z = []
    for w, b in params:
        z += [np.zeros_like(w, dtype=np.float64), np.zeros_like(b, dtype=np.float64)]
    return {"t": 0, "m": list(z), "v": [a.copy() for a in z]}
