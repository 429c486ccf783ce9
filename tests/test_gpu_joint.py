"""Multi-contrast reconstruction on the GPU (Sec. 5.6: FIRLS_MT, FIRLS_JTV)
against the FP64 oracle's joint solver: C consecutive slices of the batch
are the contrasts of one image, with joint weights and one PCG on the stacked
unknown."""
import numpy as np
import pytest

import firls_synth as fs
from oracle import firls_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_OP = 2e-5
TOL_SOLVE = 1e-4


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1411_5057_gb300 as F
    return F


def c64(a):
    return torch.from_numpy(np.ascontiguousarray(a).astype(np.complex64)).cuda()


def host(t):
    return t.cpu().numpy().astype(np.complex128)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _ctx(F, probs, C):
    p0 = probs[0]
    ctx = F.Context(p0.n, batch=len(probs), real=False)
    ctx.set_channels(C)
    ctx.set_operator(torch.from_numpy(np.stack([p.mask for p in probs])).cuda(), p0.psi, p0.levels)
    return ctx, c64(np.stack([p.b for p in probs]))


_CASES = {
    "mt_db4": dict(n=64, psi=fs.PSI_DB4, levels=3, lam=1e-3, lam_tv=0.0),
    "jtv": dict(n=64, psi=fs.PSI_TV, levels=0, lam=0.0, lam_tv=1e-3),
    "jtv_haar": dict(n=96, psi=fs.PSI_TV | fs.PSI_HAAR, levels=2, lam=5e-4, lam_tv=1e-3),
}


@pytest.mark.parametrize("name", sorted(_CASES))
def test_joint_weights_S_Pinv_parity(F, name):
    """Joint weights from three contrasts, then S d and P^-1 r per contrast."""
    cfg = _CASES[name]
    T, n = 3, cfg["n"]
    probs = fs.multi_contrast(n, T, 0.25, 0.01, 5, psi=cfg["psi"], levels=cfg["levels"], lam=cfg["lam"],
                              lam_tv=cfg["lam_tv"])
    rng = np.random.default_rng(8)
    cr = lambda: rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    xs = [p.x0 + 0.05 * cr() for p in probs]
    ds, rs = [cr() for _ in range(T)], [cr() for _ in range(T)]
    js = O.JointSystem([p.mask for p in probs], cfg["psi"], cfg["levels"], cfg["lam"], cfg["lam_tv"])
    js.update_weights(xs)
    ctx, _ = _ctx(F, probs, T)
    p = F.make_params(1, 1, lam=cfg["lam"], lam_tv=cfg["lam_tv"])
    q = torch.empty(T, n, n, dtype=torch.complex64, device="cuda")
    z = torch.empty_like(q)
    ctx.apply_S_P(p, c64(np.stack(xs)), c64(np.stack(ds)), q, c64(np.stack(rs)), z)
    ww = torch.empty(T, n, n, dtype=torch.float32, device="cuda")
    wt = torch.empty_like(ww)
    ctx.get_weights(ww, wt)
    for t, part in enumerate(js.parts):
        # weights through the joint norms 1/w (absolute error: a few ulp of the largest)
        if part.kind:
            g_gpu, g_ref = 1.0 / ww[t].cpu().numpy().reshape(-1), 1.0 / part.w
            assert np.max(np.abs(g_gpu - g_ref)) < TOL_OP * np.max(g_ref), t
        if part.tv:
            g_gpu, g_ref = 1.0 / wt[t].cpu().numpy().reshape(-1), 1.0 / part.Wtv
            assert np.max(np.abs(g_gpu - g_ref)) < TOL_OP * np.max(g_ref), t
        assert rel(host(q)[t], part.apply_S(ds[t])) < 1e-4, t
        assert rel(host(z)[t], part.apply_Pinv(rs[t])) < 1e-4, t
    # the weights are shared: identical across the contrasts
    for t in range(1, T):
        assert torch.equal(ww[t], ww[0]) and torch.equal(wt[t], wt[0])
    ctx.close()


@pytest.mark.parametrize("name,outer,inner", [("mt_db4", 20, 20), ("jtv", 30, 20)])
def test_joint_fixed_schedule_parity(F, name, outer, inner):
    cfg = _CASES[name]
    probs = fs.multi_contrast(96, 3, 0.25, 0.01, 6, psi=cfg["psi"], levels=cfg["levels"], lam=cfg["lam"],
                              lam_tv=cfg["lam_tv"])
    x_ref, info = O.firls_joint([p.b for p in probs], [p.mask for p in probs], psi=cfg["psi"],
                                levels=cfg["levels"], lam=cfg["lam"], lam_tv=cfg["lam_tv"], outer=outer, inner=inner)
    ctx, b = _ctx(F, probs, 3)
    x = host(ctx.solve(b, F.make_params(outer, inner, lam=cfg["lam"], lam_tv=cfg["lam_tv"])))
    for t in range(3):
        assert rel(x[t], x_ref[t]) < TOL_SOLVE, (t, rel(x[t], x_ref[t]))
    ctx.close()


def test_joint_tv_db4_one_outer_step_parity(F):
    """JTV + joint D4 at 128^2: one outer step (joint weights, P, 20 PCG) from
    the oracle's own iterates x^0 and x^3."""
    probs = fs.multi_contrast(128, 3, 0.2, 0.01, 9, psi=fs.PSI_TV | fs.PSI_DB4, levels=3, lam=5e-4, lam_tv=1e-3)
    kw = dict(psi=probs[0].psi, levels=3, lam=5e-4, lam_tv=1e-3, inner=20)
    bs, ms = [p.b for p in probs], [p.mask for p in probs]
    xk = None
    for k in (0, 3):
        if k:
            xk, _ = O.firls_joint(bs, ms, outer=k, **kw)
        x_ref, _ = O.firls_joint(bs, ms, outer=1, x_init=xk, **kw)
        ctx, b = _ctx(F, probs, 3)
        x0 = None if xk is None else c64(np.stack(xk))
        x = host(ctx.solve(b, F.make_params(1, 20, lam=5e-4, lam_tv=1e-3), x0=x0))
        for t in range(3):
            assert rel(x[t], x_ref[t]) < TOL_SOLVE, (k, t, rel(x[t], x_ref[t]))
        ctx.close()


def test_images_lockstep_and_independent(F):
    """Two images of three contrasts in one batch, stopped by tolerances: the
    contrasts of an image take the same outer and PCG counts, and each image
    equals that image solved alone, bit for bit."""
    imgs = [fs.multi_contrast(64, 3, 0.2 + 0.05 * i, 0.01, 20 + i, psi=fs.PSI_TV | fs.PSI_HAAR, levels=2,
                              lam=4e-4 * (1 + i), lam_tv=1e-3) for i in range(2)]
    probs = imgs[0] + imgs[1]
    lams = [p.lam for p in probs]
    mk = lambda ls: F.make_params(40, 60, lam_per_slice=ls, lam_tv_per_slice=[1e-3] * len(ls), pcg_tol=0.05,
                                  pcg_tol_rel=True, outer_tol=1e-4)
    ctx, b = _ctx(F, probs, 3)
    xb = ctx.solve(b, mk(lams)).clone()
    _, od, _, pc = ctx.slot_status(with_pcg=True)
    assert od[0:3] == [od[0]] * 3 and od[3:6] == [od[3]] * 3, od
    assert pc[0:3] == [pc[0]] * 3 and pc[3:6] == [pc[3]] * 3, pc
    for i, img in enumerate(imgs):
        one, b1 = _ctx(F, img, 3)
        x1 = one.solve(b1, mk([p.lam for p in img]))
        _, od1, _, pc1 = one.slot_status(with_pcg=True)
        assert od1 == od[3 * i:3 * i + 3] and pc1 == pc[3 * i:3 * i + 3]
        assert torch.equal(x1, xb[3 * i:3 * i + 3]), i
        one.close()
    ctx.close()


@pytest.mark.parametrize("name", sorted(_CASES))
def test_joint_objective(F, name):
    cfg = _CASES[name]
    probs = fs.multi_contrast(cfg["n"], 3, 0.25, 0.01, 4, psi=cfg["psi"], levels=cfg["levels"], lam=cfg["lam"],
                              lam_tv=cfg["lam_tv"])
    rng = np.random.default_rng(2)
    xs = [p.x0 + 0.02 * (rng.standard_normal(p.x0.shape) + 1j * rng.standard_normal(p.x0.shape)) for p in probs]
    xs = [np.asarray(x.astype(np.complex64), np.complex128) for x in xs]
    want = O.objective_joint(xs, [np.asarray(p.b.astype(np.complex64), np.complex128) for p in probs],
                             [p.mask for p in probs], cfg["psi"], cfg["levels"], cfg["lam"], cfg["lam_tv"], O.EPS)
    ctx, b = _ctx(F, probs, 3)
    got = ctx.objective(b, F.make_params(1, 1, lam=cfg["lam"], lam_tv=cfg["lam_tv"]), c64(np.stack(xs)))
    assert got == [got[0]] * 3
    assert abs(got[0] - want) < 1e-5 * want, (got[0], want)
    ctx.close()


def test_channel_errors(F):
    probs = fs.multi_contrast(32, 3, 0.3, 0.01, 3, psi=fs.PSI_TV | fs.PSI_HAAR, levels=2, lam=1e-3, lam_tv=1e-3)
    ctx = F.Context(32, batch=3)
    with pytest.raises(F.FirlsError):
        ctx.set_channels(2)                       # does not divide the batch
    with pytest.raises(F.FirlsError):
        ctx.set_channels(0)
    ctx.set_channels(3)
    masks = torch.from_numpy(np.stack([p.mask for p in probs])).cuda()
    with pytest.raises(F.FirlsError):
        ctx.set_operator(masks, fs.PSI_TV_ANISO, 0)   # joint TV is the isotropic form
    with pytest.raises(F.FirlsError):
        ctx.set_operator(masks, fs.PSI_HAAR, 2, groups=torch.arange(32 * 32, dtype=torch.int32).reshape(-1, 2).cuda())
    ctx.set_operator(masks, fs.PSI_TV | fs.PSI_HAAR, 2)
    b = c64(np.stack([p.b for p in probs]))
    with pytest.raises(F.FirlsError):              # the contrasts share the regulariser
        ctx.solve(b, F.make_params(2, 2, lam_per_slice=[1e-3, 2e-3, 1e-3], lam_tv=1e-3))
    with pytest.raises(F.FirlsError):
        ctx.slot_load(0, masks[0], b[0], 1e-3, 1e-3)
    x = ctx.solve(b, F.make_params(2, 2, lam=1e-3, lam_tv=1e-3))
    assert torch.isfinite(torch.view_as_real(x)).all()
    ctx.close()


def test_mt_workload_matches_stored_oracle(F):
    """The multi-contrast workload (3 contrasts at 256^2, joint D4) for the
    paper's 100-iteration budget: each contrast against the FP64 oracle's
    result of the same schedule (tests/golden/make_xmt.py)."""
    import os
    d = os.path.join(os.path.dirname(__file__), "golden", "xmt_db4_256")
    seeds = [s for s in (1, 2) if os.path.exists(os.path.join(d, f"seed{s}.npz"))]
    assert seeds, "no stored multi-contrast result"
    probs = [p for s in seeds for p in fs.mt_db4_256(s)]
    z0 = np.load(os.path.join(d, f"seed{seeds[0]}.npz"))
    ctx, b = _ctx(F, probs, 3)
    x = host(ctx.solve(b, F.make_params(int(z0["outer"]), int(z0["inner"]), lam=probs[0].lam)))
    for i, s in enumerate(seeds):
        ref = np.load(os.path.join(d, f"seed{s}.npz"))["x"].astype(np.complex128)
        for t in range(3):
            assert rel(x[3 * i + t], ref[t]) < TOL_SOLVE, (s, t, rel(x[3 * i + t], ref[t]))
    ctx.close()
