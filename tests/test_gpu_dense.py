"""Dense random-projection A on the GPU (FIRLS_L1, Sec. 5.2-5.3) against the
FP64 dense oracle: the one-pass A^T A d, abar, fixed-schedule solves per
preconditioner, the paper-size workload against the oracle's stored result,
tolerance stops with independent problems, and the error cases."""
import math
import os

import numpy as np
import pytest

import firls_synth as fs
from oracle import dense_oracle as D

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_SOLVE = 1e-4


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1411_5057_gb300 as F
    return F


def f32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _problems(P, M, N, seed=0, lam=0.05):
    rng = np.random.default_rng(seed)
    As, bs = [], []
    for _ in range(P):
        A = rng.standard_normal((M, N)) / math.sqrt(M)
        x0 = np.zeros(N)
        idx = rng.choice(N, max(1, N // 10), replace=False)
        x0[idx] = rng.standard_normal(len(idx))
        As.append(A.astype(np.float32).astype(np.float64))  # what the GPU holds
        bs.append((A @ x0 + 0.01 * rng.standard_normal(M)).astype(np.float32).astype(np.float64))
    return As, bs, lam


@pytest.mark.parametrize("M,N,shared", [(800, 4000, False), (37, 100, False), (5, 8192, True), (300, 1024, True),
                                        (1, 4, False)])
def test_AtA_parity(F, M, N, shared):
    P = 3
    rng = np.random.default_rng(M + N)
    A = rng.standard_normal((1 if shared else P, M, N)).astype(np.float32)
    d = rng.standard_normal((P, N)).astype(np.float32)
    ctx = F.DenseContext(M, N, P, shared=shared)
    ctx.set_matrix(f32(A[0] if shared else A))
    q = torch.empty(P, N, dtype=torch.float32, device="cuda")
    ctx.apply_AtA(f32(d), q)
    got = q.cpu().numpy().astype(np.float64)
    for p in range(P):
        Ap = A[0 if shared else p].astype(np.float64)
        want = Ap.T @ (Ap @ d[p].astype(np.float64))
        assert rel(got[p], want) < 2e-5, (p, rel(got[p], want))
    ab = ctx.abar()
    for m in range(len(ab)):
        want = D.DenseSystem(A[m].astype(np.float64), 0.1).abar
        assert abs(ab[m] - want) < 1e-6 * want
    ctx.close()


@pytest.mark.parametrize("precond,inner,pcg_tol", [("paper", 10, 0.0), ("jacobi", 600, 1e-7), ("none", 2000, 1e-7)])
def test_solve_parity_per_preconditioner(F, precond, inner, pcg_tol):
    """The proposed P at a fixed schedule; Jacobi and plain CG with nearly
    exact inner solves (a short fixed schedule of a weaker preconditioner
    amplifies FP32 rounding, as with the Fourier operator)."""
    P, M, N = 3, 60, 200
    As, bs, lam = _problems(P, M, N, seed=1)
    ctx = F.DenseContext(M, N, P)
    ctx.set_matrix(f32(np.stack(As)))
    x = ctx.solve(f32(np.stack(bs)), F.make_params(30, inner, lam=lam, precond=precond, pcg_tol=pcg_tol))
    x = x.cpu().numpy()
    for p in range(P):
        want, _ = D.firls_l1(As[p], bs[p], lam, outer=30, inner=inner, precond=precond, pcg_tol=pcg_tol)
        assert rel(x[p].astype(np.float64), want) < TOL_SOLVE, (p, rel(x[p], want))
    ctx.close()


def test_shared_matrix_parity(F):
    """Several signals measured by one projection: one A for all problems."""
    P, M, N = 4, 80, 400
    As, bs, lam = _problems(P, M, N, seed=2)
    A = As[0]
    rng = np.random.default_rng(3)
    bs = [(A @ np.where(rng.random(N) < 0.1, rng.standard_normal(N), 0.0)).astype(np.float32).astype(np.float64)
          for _ in range(P)]
    ctx = F.DenseContext(M, N, P, shared=True)
    ctx.set_matrix(f32(A))
    x = ctx.solve(f32(np.stack(bs)), F.make_params(40, 20, lam=lam)).cpu().numpy()
    for p in range(P):
        want, _ = D.firls_l1(A, bs[p], lam, outer=40, inner=20)
        assert rel(x[p].astype(np.float64), want) < TOL_SOLVE, p
    ctx.close()


def test_paper_workload_matches_stored_oracle(F):
    """The Sec. 5.3 workload (4000 long, 800 measurements, 10 % non-zeros)
    for 200 outer steps of 30 PCG: against the FP64 oracle's stored result of
    the same schedule (tests/golden/make_xdense.py)."""
    d = os.path.join(os.path.dirname(__file__), "golden", "xdense_l1")
    seeds = [s for s in (1, 2) if os.path.exists(os.path.join(d, f"seed{s}.npz"))]
    assert seeds, "no stored dense result"
    probs = [fs.dense_l1(s) for s in seeds]
    z0 = np.load(os.path.join(d, f"seed{seeds[0]}.npz"))
    ctx = F.DenseContext(800, 4000, len(probs))
    ctx.set_matrix(f32(np.stack([p.A for p in probs])))
    x = ctx.solve(f32(np.stack([p.b for p in probs])),
                  F.make_params(int(z0["outer"]), int(z0["inner"]), lam=probs[0].lam)).cpu().numpy()
    for i, s in enumerate(seeds):
        want = np.load(os.path.join(d, f"seed{s}.npz"))["x"]
        assert rel(x[i].astype(np.float64), want) < TOL_SOLVE, (s, rel(x[i], want))
    ctx.close()


def test_shared_paper_workload_matches_stored_oracle(F):
    """The Sec. 5.3 workload with one A shared by several signals (the GEMM
    form of S d): problem 0 of firls_synth.dense_l1_shared(1, P) is
    dense_l1(1), so after 200 x 30 it matches the FP64 oracle's stored
    result of seed 1; every problem lands near its sparse truth."""
    f = os.path.join(os.path.dirname(__file__), "golden", "xdense_l1", "seed1.npz")
    assert os.path.exists(f), "no stored dense result"
    z = np.load(f)
    A, B, X0, lam = fs.dense_l1_shared(1, 5)
    ctx = F.DenseContext(800, 4000, 5, shared=True)
    ctx.set_matrix(f32(A))
    x = ctx.solve(f32(B), F.make_params(int(z["outer"]), int(z["inner"]), lam=lam)).cpu().numpy()
    assert rel(x[0].astype(np.float64), z["x"]) < TOL_SOLVE, rel(x[0], z["x"])
    for p in range(5):
        assert np.mean((x[p] - X0[p]) ** 2) < 2 * float(z["mse"]) + 0.02, p
    ctx.close()


def test_tolerance_stops_and_independence(F):
    """Problems with different lambdas stop on their own outer tolerance and
    PCG tolerance; each equals that problem solved beside other problems
    (same batch size, so the same row chunks), bit for bit."""
    P, M, N = 3, 64, 256
    As, bs, _ = _problems(P, M, N, seed=4)
    lams = [0.02, 0.05, 0.1]
    prm = lambda ls: F.make_params(300, 40, lam_per_slice=ls, pcg_tol=1e-5, outer_tol=1e-4)
    ctx = F.DenseContext(M, N, P)
    ctx.set_matrix(f32(np.stack(As)))
    x, st = ctx.solve(f32(np.stack(bs)), prm(lams), stats=True)
    assert st["outer_done"] < 300
    # each side stops where its own relative change first falls to 1e-4 (and
    # its PCG where its own residual falls to 1e-5): FP32 and FP64 can take
    # those decisions one step apart, so the iterates agree to the stopping
    # tolerances' scale, not to the fixed-schedule 1e-4 of the tests above
    for p in range(P):
        want, info = D.firls_l1(As[p], bs[p], lams[p], outer=300, inner=40, pcg_tol=1e-5, outer_tol=1e-4)
        assert rel(x[p].cpu().numpy().astype(np.float64), want) < 1e-3, p
    # problem 1 with two different neighbours
    As2 = [As[2], As[1], As[0]]
    bs2 = [bs[2], bs[1], bs[0]]
    ctx2 = F.DenseContext(M, N, P)
    ctx2.set_matrix(f32(np.stack(As2)))
    x2 = ctx2.solve(f32(np.stack(bs2)), prm([0.1, 0.05, 0.02]))
    assert torch.equal(x2[1], x[1]) and torch.equal(x2[0], x[2]) and torch.equal(x2[2], x[0])
    ctx.close()
    ctx2.close()


def test_breakdown_is_isolated(F):
    P, M, N = 3, 40, 120
    As, bs, lam = _problems(P, M, N, seed=5)
    ctx = F.DenseContext(M, N, P)
    ctx.set_matrix(f32(np.stack(As)))
    good = ctx.solve(f32(np.stack(bs)), F.make_params(10, 10, lam=lam)).clone()
    bad = np.stack(bs)
    bad[2, 3] = np.nan
    with pytest.raises(F.FirlsError) as e:
        ctx.solve(f32(bad), F.make_params(10, 10, lam=lam))
    assert e.value.status == 6
    out = torch.empty(P, N, dtype=torch.float32, device="cuda")
    try:
        ctx.solve(f32(bad), F.make_params(10, 10, lam=lam), out=out)
    except F.FirlsError:
        pass
    assert torch.equal(out[:2], good[:2])
    ctx.close()


def test_dense_errors(F):
    for M, N in ((10, 6), (10, 8196), (0, 8)):
        with pytest.raises(F.FirlsError):
            F.DenseContext(M, N, 1)
    ctx = F.DenseContext(10, 16, 2)
    b = torch.zeros(2, 10, device="cuda")
    with pytest.raises(F.FirlsError):
        ctx.solve(b, F.make_params(1, 1, lam=0.1))            # matrix not set
    ctx.set_matrix(torch.randn(2, 10, 16, device="cuda"))
    with pytest.raises(F.FirlsError):
        ctx.solve(b, F.make_params(1, 1, lam=0.1, precond="ilu0"))
    with pytest.raises(F.FirlsError):
        ctx.solve(b, F.make_params(1, 1, lam=0.1, lam_tv=0.1))
    with pytest.raises(F.FirlsError):
        ctx.solve(b, F.make_params(1, 1, lam=-1.0))
    x = ctx.solve(b, F.make_params(2, 2, lam=0.1))                 # b = 0: x = 0 exactly
    assert torch.count_nonzero(x) == 0
    q = torch.empty(2, 16, device="cuda")
    for bad in (torch.zeros(2, 16, dtype=torch.float64, device="cuda"), torch.zeros(2, 15, device="cuda"),
                torch.zeros(16, 2, device="cuda").t()):
        with pytest.raises(F.FirlsError):                                # wrong type, size or layout
            ctx.apply_AtA(bad, q)
    with pytest.raises(F.FirlsError):
        ctx.solve(b.double(), F.make_params(1, 1, lam=0.1))
    ctx.close()


def test_shared_matrix_gemm_ragged_tiles(F):
    """A shared matrix whose sizes leave ragged tiles in every dimension of
    both products (200 problems over 128-row tiles, M = 260 and N = 1000 over
    128-column tiles, K split unevenly): A^T A d against FP64."""
    P, M, N = 200, 260, 1000
    rng = np.random.default_rng(21)
    A = (rng.standard_normal((M, N)) / math.sqrt(M)).astype(np.float32)
    d = rng.standard_normal((P, N)).astype(np.float32)
    ctx = F.DenseContext(M, N, P, shared=True)
    ctx.set_matrix(f32(A))
    q = torch.empty(P, N, dtype=torch.float32, device="cuda")
    ctx.apply_AtA(f32(d), q)
    A64 = A.astype(np.float64)
    want = (d.astype(np.float64) @ A64.T) @ A64
    got = q.cpu().numpy().astype(np.float64)
    for p in range(P):
        assert rel(got[p], want[p]) < 2e-5, (p, rel(got[p], want[p]))
    ctx.close()
