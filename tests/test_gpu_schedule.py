"""Inner-solve schedules on the macro-step solver: every slice advances on its
own, so its result does not depend on the other slices of the batch, and a
schedule with more PCG steps in later outer steps equals the same outer steps
taken one by one (the outer loop of Alg. 2 / Alg. 3 is memoryless: W^k and P
come from x^k, PCG restarts at x^k)."""
import numpy as np
import pytest

import firls_synth as fs
from oracle import firls_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_SOLVE = 1e-4


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1411_5057_gb300 as F
    return F


def _ctx(F, probs):
    p0 = probs[0]
    ctx = F.Context(p0.n, batch=len(probs), real=p0.real)
    ctx.set_operator(torch.from_numpy(np.stack([p.mask for p in probs])).cuda(), p0.psi, p0.levels)
    b = torch.from_numpy(np.stack([p.b for p in probs]).astype(np.complex64)).cuda()
    return ctx, b


def test_late_inner_schedule_equals_steps_one_by_one(F):
    p = fs.haar_l1_64()
    K, J, J_late, k_late = 10, 20, 45, 4
    ctx, b = _ctx(F, [p])
    x_sched = ctx.solve(b, F.make_params(K, J, lam=p.lam, pcg_late=J_late, outer_late=k_late)).clone()
    x = None
    x_ref = None
    for k in range(K):
        jk = J_late if k >= k_late else J
        x = ctx.solve(b, F.make_params(1, jk, lam=p.lam), x0=x).clone()
        x_ref, _ = O.firls_problem(p, outer=1, inner=jk, x_init=x_ref)
    assert torch.equal(x_sched, x)
    got = x_sched[0].cpu().numpy().astype(np.complex128).real
    assert np.linalg.norm(got - x_ref) / np.linalg.norm(x_ref) < TOL_SOLVE
    ctx.close()


def test_slices_with_different_inner_counts_are_independent(F):
    """PCG stopped per slice by a tolerance (relative to each outer step's
    first residual): slices take different PCG counts per outer step, and each
    result equals the slice solved alone, bit for bit."""
    probs = [fs.make_problem(64, 0.15 + 0.05 * i, 0.01, 90 + i, real=False, psi=fs.PSI_TV | fs.PSI_DB4, levels=3,
                             lam=3e-4 * (1 + i), lam_tv=8e-4) for i in range(3)]
    params = F.make_params(6, 80, lam_per_slice=[p.lam for p in probs], lam_tv_per_slice=[p.lam_tv for p in probs],
                           pcg_tol=0.05, pcg_tol_rel=True)
    ctx, b = _ctx(F, probs)
    xb, st = ctx.solve(b, params, stats=True)
    _, od, _, pc = ctx.slot_status(with_pcg=True)
    assert od == [6, 6, 6]
    assert len(set(pc)) > 1, pc                       # the slices took different PCG counts
    for i, p in enumerate(probs):
        one, b1 = _ctx(F, [p])
        pp = F.make_params(6, 80, lam_per_slice=[p.lam], lam_tv_per_slice=[p.lam_tv], pcg_tol=0.05, pcg_tol_rel=True)
        x1 = one.solve(b1, pp)
        _, _, _, pc1 = one.slot_status(with_pcg=True)
        assert pc1[0] == pc[i]
        assert torch.equal(x1[0], xb[i]), i
        one.close()
    ctx.close()


def test_boundary_period_changes_timing_not_results(F):
    """Outer-step transitions every 4th macro step: slices wait for them, but
    every slice computes exactly what it computes with a transition in every
    macro step (same outer steps, same PCG steps, same x)."""
    probs = [fs.make_problem(64, 0.2, 0.01, 95 + i, real=False, psi=fs.PSI_TV | fs.PSI_DB4, levels=3, lam=5e-4,
                             lam_tv=1e-3) for i in range(3)]
    ctx, b = _ctx(F, probs)
    base = dict(lam=5e-4, lam_tv=1e-3, outer_tol=1e-4, stop_on_distance=False)
    x1, s1 = ctx.solve(b, F.make_params(30, 15, **base), stats=True)
    x1 = x1.clone()
    _, od1, _, pc1 = ctx.slot_status(with_pcg=True)
    x4, s4 = ctx.solve(b, F.make_params(30, 15, boundary_period=4, **base), stats=True)
    _, od4, _, pc4 = ctx.slot_status(with_pcg=True)
    assert od1 == od4 and pc1 == pc4
    assert torch.equal(x1, x4)
    ctx.close()


def _serve_probs():
    return [fs.make_problem(64, 0.15 + 0.02 * (i % 5), 0.01, 300 + i, real=False, psi=fs.PSI_TV | fs.PSI_DB4,
                            levels=3, lam=4e-4, lam_tv=1e-3) for i in range(10)]


def test_slot_move_continues_bit_for_bit(F):
    """A slice moved to another slot mid-solve continues exactly as it would
    have in its own slot (every per-slice array and its state move)."""
    p = _serve_probs()[0]
    prm = F.make_params(1, 20, lam=p.lam, lam_tv=p.lam_tv, outer_tol=1e-4, stop_on_distance=True)
    mask = torch.from_numpy(p.mask).cuda()
    b = torch.from_numpy(p.b.astype(np.complex64)).cuda()
    outs = []
    for move in (False, True):
        ctx = F.Context(64, batch=3)
        ctx.set_operator(mask[None].expand(3, 64, 64).contiguous(), p.psi, p.levels)
        for s in range(3):
            ctx.slot_retire(s)
        ctx.slot_load(0, mask, b, p.lam, p.lam_tv)
        ctx.run_steps(prm, 37)
        src = 0
        if move:
            ctx.slot_move(0, 2)
            src = 2
        ctx.run_steps(prm, 50)
        x = torch.empty(64, 64, dtype=torch.complex64, device="cuda")
        ctx.slot_get(src, x)
        _, od, rel, pc = ctx.slot_status(with_pcg=True)
        outs.append((x, od[src], rel[src], pc[src]))
        ctx.close()
    assert torch.equal(outs[0][0], outs[1][0])
    assert outs[0][1:] == outs[1][1:]


def test_serve_compaction_is_bit_exact(F):
    """The serving loop's compaction at the end of the queue (running slices
    moved to the lowest slots, fewer slots launched) changes no result."""
    probs = _serve_probs()
    masks = [torch.from_numpy(p.mask).cuda() for p in probs]
    bs = [torch.from_numpy(p.b.astype(np.complex64)).cuda() for p in probs]
    prm = F.make_params(300, 20, lam=4e-4, lam_tv=1e-3, outer_tol=3e-5, stop_on_distance=True, stall_tol=6e-7,
                        pcg_late=60, outer_late=20, boundary_period=4)
    res = []
    for compact in (False, True):
        ctx = F.Context(64, batch=4)
        ctx.set_operator(torch.stack(masks[:4]), probs[0].psi, probs[0].levels)
        outs = [torch.zeros(64, 64, dtype=torch.complex64, device="cuda") for _ in probs]
        pcg = [0] * len(probs)
        cnt = {}
        steps = F.serve(ctx, masks, bs, [p.lam for p in probs], [p.lam_tv for p in probs], prm, outs, chunk=8,
                        max_outer=300, counters=cnt, pcg_steps=pcg, compact=compact)
        res.append((outs, steps, pcg, cnt))
        ctx.close()
    (o0, s0, p0, c0), (o1, s1, p1, c1) = res
    assert c0["moves"] == 0 and c1["moves"] > 0
    assert s0 == s1 and p0 == p1
    for a, b in zip(o0, o1):
        assert torch.equal(a, b)
