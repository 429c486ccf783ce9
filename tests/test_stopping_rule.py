"""The outer-loop stop on the estimated distance to the limit (outer_tol_kind 1).

FIRLS converges linearly near x* (Theorem 3 gives convergence; the rate is
observed): ||x^{k+1} - x^k|| shrinks by a near-constant factor mu per outer
step.  Summing the remaining steps gives the distance estimate
relchg_k * mu / (1 - mu), with mu the mean contraction over the last W = 24
steps, (relchg_k / relchg_{k-W})^(1/W), at most 0.999 (the same definition
as the library's outer_tol_kind 1).  This test measures the estimate against
the true distance to the converged point on the FP64 oracle's own trajectory
for the 64x64 TV + D4 workload: the estimate must not understate the
distance by more than the margin the 256^2 stop (3e-5 for a 1e-4 target)
leaves.
"""
import math

import numpy as np
import pytest

import firls_synth as fs
from oracle import firls_oracle as O


W = 24


def distance_estimate(rels, k):
    mu = min((rels[k] / rels[k - W]) ** (1.0 / W), 0.999)
    return rels[k] * mu / (1.0 - mu)


@pytest.fixture(scope="module")
def trajectory():
    p = fs.tv_db4_256(n=64)
    xs = [O.op_AH(p.b, p.mask, False)]
    rels = []
    for _ in range(160):
        x, info = O.firls_problem(p, outer=1, inner=30, x_init=xs[-1])
        xs.append(x)
        rels.append(info["rel_change"][0])
    return xs, rels


def test_distance_estimate_tracks_true_distance(trajectory):
    xs, rels = trajectory
    # the last iterate stands in for x*; its own remaining distance is about
    # the final estimate, so only distances well above it are compared
    xstar = xs[-1]
    floor = 10 * distance_estimate(rels, len(rels) - 1)
    checked = 0
    ratios = []
    for k in range(W, len(rels) - 1):
        true = np.linalg.norm(xs[k + 1] - xstar) / np.linalg.norm(xs[k + 1])
        if not floor <= true <= 2e-3:
            continue
        ratios.append(distance_estimate(rels, k) / true)
        checked += 1
    assert checked >= 20
    assert 0.33 <= min(ratios) and max(ratios) <= 4.0, (min(ratios), max(ratios))


def test_estimate_is_exact_for_a_geometric_sequence():
    """x^k = x* + mu^k e: the estimate reproduces ||x^k - x*|| / ||x^k|| up to
    the change of ||x^k|| between steps."""
    rng = np.random.default_rng(0)
    xstar = rng.standard_normal(500)
    e = rng.standard_normal(500) * 1e-2
    mu = 0.9
    xs = [xstar + mu ** k * e for k in range(60)]
    rels = [np.linalg.norm(xs[k + 1] - xs[k]) / np.linalg.norm(xs[k]) for k in range(59)]
    for k in range(W, 59):
        true = np.linalg.norm(xs[k + 1] - xstar) / np.linalg.norm(xs[k])
        assert abs(distance_estimate(rels, k) / true - 1) < 1e-3
