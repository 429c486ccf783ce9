"""Learned warm start for FIRLS: training pairs from the solver itself, CNN
training on the GPU, and the count of PCG steps it saves.

The CNN (``binding.Cnn``) maps [Re A^H b, Im A^H b, mask] to a correction,
x1 = A^H b + CNN(.).  Its targets are FIRLS solutions computed by this
library; ``firls_warm_start_guard`` keeps A^H b (plain PCG) for any slice
where F_eps(x1) > F_eps(A^H b).  Every numerical step runs in the CUDA
library; this module only orchestrates calls and moves tensors.
"""
from __future__ import annotations

import numpy as np

from . import binding as B


def workload(n, seeds, ratio=0.20, sigma=0.01, lam_tv=1e-3, lam_w=5e-4, levels=4):
    """Seeded TV + D4 slices of the 256^2 recipe (inputs only, numpy)."""
    import firls_synth as fs
    probs = [fs.make_problem(n, ratio, sigma, s, real=False, psi=fs.PSI_TV | fs.PSI_DB4, levels=levels,
                             lam=lam_w, lam_tv=lam_tv) for s in seeds]
    return (np.stack([p.mask for p in probs]), np.stack([p.b for p in probs]).astype(np.complex64),
            dict(lam=lam_w, lam_tv=lam_tv, levels=levels))


def _ctx(n, masks, meta, stream=None):
    import torch
    ctx = B.Context(n, batch=masks.shape[0], stream=stream)
    ctx.set_operator(torch.from_numpy(masks).cuda(), B.PSI_TV | B.PSI_DB4, meta["levels"])
    return ctx


def generate_pairs(n, seeds, outer, inner, chunk=128):
    """(A^H b, mask, x) on the GPU for every seed, x = FIRLS(outer x inner)."""
    import torch
    atbs, masks_all, xs = [], [], []
    for i in range(0, len(seeds), chunk):
        masks, b, meta = workload(n, seeds[i:i + chunk])
        ctx = _ctx(n, masks, meta)
        bd = torch.from_numpy(b).cuda()
        params = B.make_params(outer, inner, lam=meta["lam"], lam_tv=meta["lam_tv"])
        xs.append(ctx.solve(bd, params))
        atbs.append(ctx.adjoint(bd))
        masks_all.append(torch.from_numpy(masks).cuda())
        ctx.close()
    return torch.cat(atbs), torch.cat(masks_all), torch.cat(xs)


def train(net, atb, masks, target, epochs, lr, batch, seed=0, log=None):
    """Adam on minibatches of `batch` slices (net.batch must equal batch)."""
    import torch
    rng = np.random.default_rng(seed)
    m = atb.shape[0]
    losses = []
    for ep in range(epochs):
        order = torch.as_tensor(rng.permutation(m), device=atb.device)
        tot = 0.0
        for j in range(0, m - batch + 1, batch):
            idx = order[j:j + batch]
            tot += net.train_step(atb[idx].contiguous(), masks[idx].contiguous(), target[idx].contiguous(), lr)
        losses.append(tot)
        if log:
            log(f"epoch {ep}: loss {tot:.4e}")
    return losses


def warm_start(ctx, net, b, atb, masks, params):
    """Guarded learned start: x1 = DC(A^H b + CNN(.)), kept where
    F_eps(x1) <= F_eps(A^H b); DC restores the measured k-space entries."""
    import torch
    x1 = net.forward(atb, masks)
    x1 = ctx.data_consistency(b, x1, out=x1)
    x0 = torch.empty_like(x1)
    chosen = ctx.warm_start_guard(b, params, x1, x0)
    return x0, chosen


def steps_to_tolerance(n, masks, b, meta, x0, xstar, inner, tol=1e-4, max_outer=80):
    """Outer steps (each `inner` PCG steps) until ||x - x*|| <= tol ||x*|| per slice."""
    import torch
    ctx = _ctx(n, masks, meta)
    bd = torch.from_numpy(b).cuda()
    one = B.make_params(1, inner, lam=meta["lam"], lam_tv=meta["lam_tv"])
    x = x0.clone()
    need = np.full(masks.shape[0], -1)
    xs_norm = torch.linalg.vector_norm(xstar.reshape(xstar.shape[0], -1), dim=1)
    for k in range(1, max_outer + 1):
        x = ctx.solve(bd, one, x0=x)
        err = torch.linalg.vector_norm((x - xstar).reshape(x.shape[0], -1), dim=1) / xs_norm
        e = err.cpu().numpy()
        need[(need < 0) & (e <= tol)] = k
        if np.all(need > 0):
            break
    ctx.close()
    return need
