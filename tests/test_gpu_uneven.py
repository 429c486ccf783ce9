"""Slices of uneven size (128^2 .. 320^2, TV + D4, per-slice lambdas and mask
ratios) solved together: one CUDA graph per outer step over four contexts."""
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


@pytest.mark.parametrize("gi", [0, 1, 2, 3], ids=["128", "192", "256", "320"])
def test_uneven_one_step_parity(F, gi):
    """One outer step from A^H b per size.  The tolerance is 1e-4, or five
    times the error of an FP32-rounded run of the oracle on the same slice
    where that is larger (some of these slices amplify FP32 rounding to
    ~2e-3 within one PCG run; the GPU must stay within that band)."""
    from fp32_emulation import one_outer_step_fp32_error
    p = _groups()[gi][0]
    ctx = _ctx(F, [p], torch.cuda.current_stream())
    x = ctx.solve(torch.from_numpy(p.b[None]).to(torch.complex64).cuda(), _params(F, [p], 1, 20))
    torch.cuda.synchronize()
    x_ref, _ = O.firls_problem(p, outer=1, inner=20)
    got = x[0].cpu().numpy().astype(np.complex128)
    tol = max(1e-4, 5 * one_outer_step_fp32_error(p, O.op_AH(p.b, p.mask, False), 20))
    assert np.linalg.norm(got - x_ref) / np.linalg.norm(x_ref) < tol


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
