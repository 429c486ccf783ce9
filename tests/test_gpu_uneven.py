"""Slices of uneven size (128^2 .. 320^2, TV + D4, per-slice lambdas and mask
ratios) solved together: one CUDA graph of macro steps over four contexts."""
import numpy as np
import pytest

import firls_synth as fs
from oracle import firls_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1411_5057_gb300 as F
    return F


def _groups(per_size=2):
    out = {}
    for p in fs.uneven_batch(per_size=per_size):
        out.setdefault(p.n, []).append(p)
    return [out[n] for n in sorted(out)]


def _ctx(F, probs, stream):
    ctx = F.Context(probs[0].n, batch=len(probs), stream=stream)
    ctx.set_operator(torch.from_numpy(np.stack([p.mask for p in probs])).cuda(), probs[0].psi, probs[0].levels)
    return ctx


def _params(F, probs, outer, inner):
    return F.make_params(outer, inner, lam_per_slice=[p.lam for p in probs],
                         lam_tv_per_slice=[p.lam_tv for p in probs])


def test_uneven_graph_matches_separate_solves(F):
    groups = _groups()
    ctxs = [_ctx(F, probs, torch.cuda.Stream()) for probs in groups]
    bs = [torch.from_numpy(np.stack([p.b for p in probs])).to(torch.complex64).cuda() for probs in groups]
    ps = [_params(F, probs, 3, 20) for probs in groups]
    torch.cuda.synchronize()
    ref = [c.solve(b, p) for c, b, p in zip(ctxs, bs, ps)]
    torch.cuda.synchronize()
    outs = [torch.empty_like(b) for b in bs]
    for _ in range(2):  # second call replays the cached graph
        F.solve_multi(ctxs, bs, ps, outs)
        torch.cuda.synchronize()
        for a, r in zip(outs, ref):
            assert torch.equal(a, r)


def test_uneven_graph_with_boundary_period(F):
    """Outer-step transitions every 8th macro step in the multi-context
    graph: every slice computes what it computes when each context is solved
    alone with a transition in every macro step (same x, bit for bit)."""
    groups = _groups()
    ctxs = [_ctx(F, probs, torch.cuda.Stream()) for probs in groups]
    bs = [torch.from_numpy(np.stack([p.b for p in probs])).to(torch.complex64).cuda() for probs in groups]

    def prm(probs, period):
        return F.make_params(30, 20, lam_per_slice=[p.lam for p in probs], lam_tv_per_slice=[p.lam_tv for p in probs],
                             outer_tol=1e-4, stop_on_distance=False, boundary_period=period)

    torch.cuda.synchronize()
    ref = [c.solve(b, prm(g, 1)).clone() for c, b, g in zip(ctxs, bs, groups)]
    torch.cuda.synchronize()
    outs = [torch.empty_like(b) for b in bs]
    F.solve_multi(ctxs, bs, [prm(g, 8) for g in groups], outs)
    torch.cuda.synchronize()
    for a, r in zip(outs, ref):
        assert torch.equal(a, r)


def test_uneven_batch_reaches_converged_oracle(F):
    """The first slice of each size (seeds 1000, 1016, 1032, 1048: 128^2 ..
    320^2 TV + D4 with their own lambdas and masks), solved together by
    solve_multi with the bench's schedule and per-slice stop, lands within
    1e-4 of the FP64 oracle's converged x* (tests/golden/xstar_uneven,
    written by tests/golden/make_xstar.py --uneven from the oracle alone)."""
    import os
    import bench
    golden = os.path.join(os.path.dirname(__file__), "golden", "xstar_uneven")
    seeds = (1000, 1016, 1032, 1048)
    probs = {s: p for s, p in zip(range(1000, 1064), fs.uneven_batch()) if s in seeds}
    groups = [[probs[s]] for s in seeds]
    streams = [torch.cuda.Stream() for _ in groups]
    ctxs = [_ctx(F, g, st) for g, st in zip(groups, streams)]
    bs = [torch.from_numpy(np.stack([p.b for p in g])).to(torch.complex64).cuda() for g in groups]
    ps = [F.make_params(bench.OUTER, bench.INNER, lam_per_slice=[p.lam for p in g],
                        lam_tv_per_slice=[p.lam_tv for p in g], outer_tol=bench.OUTER_TOL, stop_on_distance=True,
                        stall_tol=bench.STALL_TOL, pcg_late=bench.INNER_LATE, outer_late=bench.OUTER_LATE,
                        boundary_period=bench.BOUNDARY_PERIOD)
          for g in groups]
    outs = [torch.empty_like(b) for b in bs]
    torch.cuda.synchronize()
    F.solve_multi(ctxs, bs, ps, outs)
    torch.cuda.synchronize()
    for s, out in zip(seeds, outs):
        xs = np.load(os.path.join(golden, f"seed{s}.npz"))["x"].astype(np.complex128)
        got = out[0].cpu().numpy().astype(np.complex128)
        err = np.linalg.norm(got - xs) / np.linalg.norm(xs)
        assert err < 1e-4, (s, err)


def test_autotune_picks_candidates_and_keeps_results(F, tmp_path):
    """The autotuner picks tile shapes from its candidate sets, caches them,
    and the tuned solve reproduces the default solve bit for bit (the tile
    shapes change the grouping of the work, not the arithmetic)."""
    probs = _groups(per_size=4)[2]  # four 256^2 slices
    ctx = _ctx(F, probs, torch.cuda.current_stream())
    b = torch.from_numpy(np.stack([p.b for p in probs])).to(torch.complex64).cuda()
    pp = _params(F, probs, 2, 20)
    ref = ctx.solve(b, pp)
    torch.cuda.synchronize()
    cache = str(tmp_path / "tune.txt")
    t = ctx.autotune(cache)
    assert t["rows_per_cta"] in (1, 2, 4, 8, 16) and t["coarse_max"] in (32, 64) and t["ilu_depth"] in (42, 43, 44, 22, 23, 24)
    assert "n=256 batch=4" in open(cache).read()
    got = ctx.solve(b, pp)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)
    ctx2 = _ctx(F, probs, torch.cuda.current_stream())
    assert ctx2.autotune(cache) == t  # cache hit
