"""Continuous batching: a queue of slices through fewer slots gives every
slice exactly its stand-alone result (slots are independent; a slice stops
changing once its relative change is below outer_tol)."""
import numpy as np
import pytest

import firls_synth as fs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1411_5057_gb300 as F
    return F


def test_serve_matches_standalone_solves(F):
    n = 64
    probs = [fs.make_problem(n, 0.2 + 0.02 * i, 0.01, 70 + i, real=False, psi=6, levels=3,
                             lam=3e-4 * (1 + i % 3), lam_tv=6e-4 * (1 + i % 2)) for i in range(7)]
    masks = [torch.from_numpy(p.mask).cuda() for p in probs]
    bs = [torch.from_numpy(p.b).to(torch.complex64).cuda() for p in probs]
    params = F.make_params(120, 20, outer_tol=2e-4)
    ctx = F.Context(n, batch=3)
    ctx.set_operator(torch.stack(masks[:3]), 6, 3)
    outs = [torch.empty_like(b) for b in bs]
    steps = F.serve(ctx, masks, bs, [p.lam for p in probs], [p.lam_tv for p in probs], params, outs, chunk=4,
                    max_outer=120)
    torch.cuda.synchronize()
    assert all(0 < s < 120 for s in steps)
    for i, p in enumerate(probs):
        one = F.Context(n, batch=1)
        one.set_operator(masks[i][None], 6, 3)
        pp = F.make_params(120, 20, outer_tol=2e-4, lam_per_slice=[p.lam], lam_tv_per_slice=[p.lam_tv])
        ref, st = one.solve(bs[i][None], pp, stats=True)
        torch.cuda.synchronize()
        assert st["outer_done"] == steps[i]
        assert torch.equal(outs[i], ref[0]), i


def test_slot_retire_and_reload(F):
    n = 64
    p = fs.tv_db4_256(n=n)
    ctx = F.Context(n, batch=2)
    m = torch.from_numpy(p.mask).cuda()
    b = torch.from_numpy(p.b).to(torch.complex64).cuda()
    ctx.set_operator(torch.stack([m, m]), p.psi, p.levels)
    ctx.slot_load(0, m, b, p.lam, p.lam_tv)
    ctx.slot_retire(1)
    ctx.run(F.make_params(3, 10))
    done, od, _ = ctx.slot_status()
    assert od == [3, 0] and done[1] == 1
    ctx.slot_load(1, m, b, p.lam, p.lam_tv)
    ctx.run(F.make_params(3, 10))
    done, od, _ = ctx.slot_status()
    assert od == [6, 3]
