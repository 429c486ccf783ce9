"""Pins for the dense-matrix oracle (FIRLS_L1 with a random projection A,
Sec. 5.2-5.3): closed forms, a dense direct solve, the gradient identity and
Theorem 2, each independent of the oracle's own code path."""
import math

import numpy as np
import pytest

import firls_synth as fs
from oracle import dense_oracle as D


def _small(seed=0, M=30, N=80, lam=0.05, density=0.15):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((M, N)) / math.sqrt(M)
    x0 = np.zeros(N)
    idx = rng.choice(N, int(density * N), replace=False)
    x0[idx] = rng.standard_normal(len(idx))
    return A, A @ x0 + 0.01 * rng.standard_normal(M), lam


def test_abar_of_orthonormal_rows_is_M_over_N():
    """Rows of A orthonormal (A A^T = I): tr(A^T A) = tr(A A^T) = M, so the
    mean diagonal entry of A^T A is M / N (Eq. ps)."""
    rng = np.random.default_rng(1)
    M, N = 24, 96
    Q, _ = np.linalg.qr(rng.standard_normal((N, M)))
    s = D.DenseSystem(Q.T, 0.1)
    assert abs(s.abar - M / N) < 1e-14
    # a hand-computed case: squared entries 1 + 4 + 9 + 1 = 15 over N = 5 columns
    A = np.zeros((3, 5))
    A[0, 0], A[0, 1], A[1, 2], A[2, 4] = 1.0, 2.0, 3.0, -1.0
    assert D.DenseSystem(A, 0.1).abar == 3.0


def _smoothed_soft(c, lam, eps):
    """Per coordinate, the root of x - c + lam x / sqrt(x^2 + eps) = 0 (the
    stationarity condition of 1/2 (x - c)^2 + lam sqrt(x^2 + eps), strictly
    increasing in x), by bisection."""
    lo, hi = np.minimum(c, 0.0) - 1.0, np.maximum(c, 0.0) + 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        f = mid - c + lam * mid / np.sqrt(mid * mid + eps)
        lo, hi = np.where(f < 0, mid, lo), np.where(f < 0, hi, mid)
    return 0.5 * (lo + hi)


def test_orthogonal_A_reaches_the_smoothed_soft_threshold():
    """A square and orthogonal: ||Ax - b|| = ||x - A^T b||, so the problem
    separates and its F_eps minimiser is the smoothed soft threshold of
    c = A^T b, coordinate by coordinate (and the soft threshold itself,
    sign(c) max(|c| - lam, 0), up to O(sqrt(eps)))."""
    rng = np.random.default_rng(2)
    N, lam = 64, 0.1
    Q, _ = np.linalg.qr(rng.standard_normal((N, N)))
    mag = np.concatenate([rng.uniform(0.0, 0.8 * lam, N // 2), rng.uniform(1.2 * lam, 3 * lam, N - N // 2)])
    c = mag * rng.choice([-1.0, 1.0], N)
    b = Q @ c
    x, info = D.firls_l1(Q, b, lam, outer=300, inner=5)
    xs = _smoothed_soft(c, lam, D.EPS)
    assert np.max(np.abs(x - xs)) < 1e-9
    soft = np.sign(c) * np.maximum(np.abs(c) - lam, 0.0)
    assert np.max(np.abs(x - soft)) < 1e-4


@pytest.mark.parametrize("precond", D.PRECONDS)
def test_pcg_matches_dense_direct_solve(precond):
    A, b, lam = _small(3)
    s = D.DenseSystem(A, lam, precond)
    rng = np.random.default_rng(4)
    s.update_weights(rng.standard_normal(A.shape[1]))
    S = A.T @ A + lam * np.diag(s.w)
    rhs = rng.standard_normal(A.shape[1])
    x, _ = D.pcg(s, rhs, np.zeros_like(rhs), 8 * len(rhs), 1e-15, float(np.linalg.norm(rhs)))
    want = np.linalg.solve(S, rhs)
    assert np.linalg.norm(x - want) <= 1e-9 * np.linalg.norm(want)


def test_jacobi_diagonal_is_diag_of_dense_S():
    A, _, lam = _small(5)
    s = D.DenseSystem(A, lam, "jacobi")
    rng = np.random.default_rng(6)
    s.update_weights(rng.standard_normal(A.shape[1]))
    cols = [s.apply_S(np.eye(A.shape[1])[:, j])[j] for j in range(A.shape[1])]
    assert np.allclose(s.p_diag(), cols, rtol=1e-13, atol=0)


def test_system_is_gradient_of_F_eps():
    """S(W(x)) x - A^T b equals the gradient of F_eps (central differences of
    the objective alone)."""
    A, b, lam = _small(7, M=12, N=20)
    eps = 1e-4
    rng = np.random.default_rng(8)
    x = rng.standard_normal(20)
    s = D.DenseSystem(A, lam, eps=eps)
    s.update_weights(x)
    g = s.apply_S(x) - A.T @ b
    h = 1e-6
    for i in range(20):
        e = np.zeros(20)
        e[i] = h
        fd = (D.objective(x + e, A, b, lam, eps) - D.objective(x - e, A, b, lam, eps)) / (2 * h)
        assert abs(fd - g[i]) < 1e-6 * (1 + abs(fd))


@pytest.mark.parametrize("inner", [1, 3, 30])
def test_theorem2_monotone(inner):
    A, b, lam = _small(9, M=60, N=200)
    _, info = D.firls_l1(A, b, lam, outer=25, inner=inner, record=True)
    F = info["F_eps"]
    for k in range(len(F) - 1):
        assert F[k + 1] <= F[k] * (1 + 1e-12)
    assert F[-1] < F[0]


def test_dense_generator_shapes():
    p = fs.dense_l1(3, N=500, M=100)
    assert p.A.shape == (100, 500) and p.b.shape == (100,)
    assert np.count_nonzero(p.x0) == 50
    q = fs.dense_l1(3, N=500, M=100)
    assert np.array_equal(p.A, q.A) and np.array_equal(p.b, q.b)


def test_dense_shared_generator():
    """One projection for every signal; problem p takes the signal and noise
    of dense_l1(seed + p), so problem 0 is dense_l1(seed) bit for bit."""
    A, B, X0, lam = fs.dense_l1_shared(3, 3, N=500, M=100)
    assert A.shape == (100, 500) and B.shape == (3, 100) and X0.shape == (3, 500)
    for p in range(3):
        one = fs.dense_l1(3 + p, N=500, M=100)
        assert np.array_equal(X0[p], one.x0)
        assert np.count_nonzero(X0[p]) == 50
        if p == 0:
            assert np.array_equal(A, one.A) and np.array_equal(B[0], one.b) and lam == one.lam
        else:
            assert not np.array_equal(A, one.A)
            assert np.allclose(B[p], A @ X0[p], atol=0.1)
