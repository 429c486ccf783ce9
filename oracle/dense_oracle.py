"""FP64 CPU oracle for FIRLS with a dense sensing matrix (arXiv 1411.5057,
Sec. 5.2-5.3: random projections instead of a partial Fourier operator).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import this module.  It
shares no code with the CUDA library; both sides read the same seeded inputs
from ``firls_synth``, which holds none of the method's arithmetic.

Problem (Eq. anapro with Phi = I and singleton groups, real x):
    min_x  1/2 ||A x - b||^2 + lam ||x||_1,   A a dense M x N real matrix.
FIRLS_L1 (Alg. 2 with Phi = I):
  * weights (Eq. gw, singleton groups): W = diag((x_i^2 + eps)^(-1/2));
  * inner system (Eq. subprob): S = A^T A + lam W, right-hand side A^T b;
  * the proposed preconditioner (Eq. pog with Phi = I): P = abar I + lam W,
    abar = tr(A^T A) / N, the mean diagonal entry of A^T A (Eq. ps);
  * Jacobi PCG (Sec. 5.2): P = diag(S) = diag(A^T A) + lam W; plain CG: P = I.
PCG restarts every outer step (d = z), warm-started at x^k from x^1 = A^T b,
and stops when ||r|| / ||A^T b|| <= pcg_tol or after ``inner`` steps; the
outer loop stops when ||x^{k+1} - x^k|| / ||x^k|| <= outer_tol.
Plain numpy: dense products, no blocking or fusion.
"""
from __future__ import annotations

import math

import numpy as np

from .firls_oracle import EPS, pcg, rdot

PRECONDS = ("paper", "jacobi", "none")


class DenseSystem:
    """S = A^T A + lam W and its preconditioner for one weight vector."""

    def __init__(self, A, lam, precond="paper", eps=EPS):
        if precond not in PRECONDS:
            raise ValueError(precond)
        self.A = np.asarray(A, dtype=np.float64)
        self.N = self.A.shape[1]
        self.lam = float(lam)
        self.eps = float(eps)
        self.precond = precond
        AtA = self.A.T @ self.A
        self.abar = float(np.trace(AtA)) / self.N
        self.diag_AtA = np.diag(AtA).copy()
        self.w = np.ones(self.N)

    def update_weights(self, x):
        self.w = (np.asarray(x, dtype=np.float64) ** 2 + self.eps) ** -0.5

    def apply_S(self, d):
        return self.A.T @ (self.A @ d) + self.lam * self.w * d

    def p_diag(self):
        if self.precond == "paper":
            return self.abar + self.lam * self.w
        if self.precond == "jacobi":
            return self.diag_AtA + self.lam * self.w
        return np.ones(self.N)

    def apply_Pinv(self, r):
        return r / self.p_diag()


def objective(x, A, b, lam, eps=0.0):
    """F(x) (eps = 0) or F_eps(x): 1/2 ||Ax - b||^2 + lam sum_i sqrt(x_i^2 + eps)."""
    x = np.asarray(x, dtype=np.float64)
    res = np.asarray(A, dtype=np.float64) @ x - np.asarray(b, dtype=np.float64)
    return 0.5 * float(res @ res) + lam * float(np.sum(np.sqrt(x * x + eps)))


def firls_l1(A, b, lam, *, outer=200, inner=30, pcg_tol=0.0, outer_tol=0.0, precond="paper", x_init=None,
             record=False, eps=EPS):
    """FIRLS_L1 on a dense A.  Returns (x, info)."""
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    system = DenseSystem(A, lam, precond, eps)
    rhs = A.T @ b
    rhs_norm = math.sqrt(rdot(rhs, rhs))
    x = rhs.copy() if x_init is None else np.array(x_init, dtype=np.float64)
    info = dict(pcg_steps=[], rel_change=[], F_eps=[], outer_done=0)
    if record:
        info["F_eps"].append(objective(x, A, b, lam, eps))
    for k in range(outer):
        system.update_weights(x)
        x_new, steps = pcg(system, rhs, x, inner, pcg_tol, rhs_norm)
        nx = math.sqrt(rdot(x, x))
        rel = math.sqrt(rdot(x_new - x, x_new - x)) / nx if nx > 0 else float("inf")
        x = x_new
        info["pcg_steps"].append(steps)
        info["rel_change"].append(rel)
        info["outer_done"] = k + 1
        if record:
            info["F_eps"].append(objective(x, A, b, lam, eps))
        if outer_tol > 0 and rel <= outer_tol:
            break
    return x, info
