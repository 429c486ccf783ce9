"""Pins for the multi-contrast oracle (Sec. 5.6: FIRLS_MT, FIRLS_JTV): joint
weights across contrasts, one PCG on the stacked block system."""
import math

import numpy as np
import pytest

import firls_synth as fs
from oracle import firls_oracle as O


def _contrasts(n=16, T=3, psi=O.PSI_DB4, levels=2, lam=1e-3, lam_tv=0.0, seed=7, ratio=0.3):
    return fs.multi_contrast(n, T, ratio, 0.01, seed, psi=psi, levels=levels, lam=lam, lam_tv=lam_tv)


@pytest.mark.parametrize("psi,lam,lam_tv", [(O.PSI_DB4, 2e-3, 0.0), (O.PSI_TV, 0.0, 2e-3),
                                            (O.PSI_TV | O.PSI_HAAR, 1e-3, 2e-3)])
def test_identical_contrasts_reduce_to_one_with_scaled_lambda(psi, lam, lam_tv):
    """T copies of one contrast: sqrt(sum_t |c|^2 + eps) = sqrt(T) sqrt(|c|^2 +
    eps/T), so the joint weights are T^-1/2 times the single-contrast weights
    with eps/T, every block of S is the single-contrast S with lam/sqrt(T),
    and the stacked inner products are T times the single ones: the joint
    trajectory equals single-contrast FIRLS with lam/sqrt(T) and eps/T."""
    T = 3
    p = fs.make_problem(16, 0.3, 0.01, 5, real=False, psi=psi, levels=2, lam=lam, lam_tv=lam_tv)
    xs, _ = O.firls_joint([p.b] * T, [p.mask] * T, psi=psi, levels=2, lam=lam, lam_tv=lam_tv, outer=6, inner=8)
    r = math.sqrt(T)
    x1, _ = O.firls(p.b, p.mask, real=False, psi=psi, levels=2, lam=lam / r, lam_tv=lam_tv / r, outer=6, inner=8,
                    eps=O.EPS / T)
    for x in xs:
        assert np.linalg.norm(x - x1) <= 1e-10 * np.linalg.norm(x1)


def test_one_contrast_is_plain_firls():
    p = fs.make_problem(16, 0.3, 0.01, 6, real=False, psi=O.PSI_TV | O.PSI_DB4, levels=2, lam=1e-3, lam_tv=1e-3)
    xs, ij = O.firls_joint([p.b], [p.mask], psi=p.psi, levels=2, lam=p.lam, lam_tv=p.lam_tv, outer=5, inner=10)
    x1, i1 = O.firls(p.b, p.mask, real=False, psi=p.psi, levels=2, lam=p.lam, lam_tv=p.lam_tv, outer=5, inner=10)
    assert np.allclose(xs[0], x1, rtol=0, atol=1e-13 * np.abs(x1).max())
    assert ij["pcg_steps"] == i1["pcg_steps"]


@pytest.mark.parametrize("psi,lam,lam_tv", [(O.PSI_HAAR, 5e-3, 0.0), (O.PSI_TV, 0.0, 1e-2)])
def test_joint_system_is_the_gradient_of_joint_F_eps(psi, lam, lam_tv):
    """S(W(x)) x - A^H b of every contrast equals the gradient of the joint
    F_eps (central differences of the objective alone)."""
    n, T, eps = 6, 2, 1e-4
    probs = _contrasts(n=n, T=T, psi=psi, levels=1, lam=lam, lam_tv=lam_tv, seed=3, ratio=0.4)
    bs, masks = [p.b for p in probs], [p.mask for p in probs]
    rng = np.random.default_rng(4)
    xs = [p.x0 + 0.05 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) for p in probs]
    js = O.JointSystem(masks, psi, 1, lam, lam_tv, eps)
    js.update_weights(xs)
    g = [s - O.op_AH(m * b, m.astype(float), False) for s, b, m in zip(js.apply_S(xs), bs, masks)]
    F = lambda zs: O.objective_joint(zs, bs, masks, psi, 1, lam, lam_tv, eps)
    h = 1e-6
    for t in range(T):
        for i in range(n * n):
            for e in (1.0, 1j):
                zp = [x.copy() for x in xs]
                zm = [x.copy() for x in xs]
                zp[t].reshape(-1)[i] += h * e
                zm[t].reshape(-1)[i] -= h * e
                fd = (F(zp) - F(zm)) / (2 * h)
                got = g[t].reshape(-1)[i]
                got = got.real if e == 1.0 else got.imag
                assert abs(fd - got) < 1e-5 * (1 + abs(fd)), (t, i, e, fd, got)


@pytest.mark.parametrize("psi,lam,lam_tv", [(O.PSI_DB4, 1e-3, 0.0), (O.PSI_TV, 0.0, 1e-3),
                                            (O.PSI_TV | O.PSI_DB4, 5e-4, 1e-3)])
def test_theorem2_monotone_joint(psi, lam, lam_tv):
    probs = _contrasts(n=32, T=3, psi=psi, levels=2, lam=lam, lam_tv=lam_tv, seed=11, ratio=0.25)
    _, info = O.firls_joint([p.b for p in probs], [p.mask for p in probs], psi=psi, levels=2, lam=lam,
                            lam_tv=lam_tv, outer=8, inner=5, record=True)
    F = info["F_eps"]
    for k in range(len(F) - 1):
        assert F[k + 1] <= F[k] * (1 + 1e-12)
    assert F[-1] < F[0]


def test_joint_pcg_matches_dense_block_solve():
    n, T = 8, 2
    probs = _contrasts(n=n, T=T, psi=O.PSI_TV | O.PSI_HAAR, levels=1, lam=0.05, lam_tv=0.02, seed=12)
    js = O.JointSystem([p.mask for p in probs], probs[0].psi, 1, 0.05, 0.02)
    rng = np.random.default_rng(13)
    js.update_weights([rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) for _ in range(T)])
    N = n * n
    dense = np.zeros((T * N, T * N), complex)
    for t in range(T):
        for j in range(N):
            e = np.zeros(N, complex)
            e[j] = 1
            dense[t * N:(t + 1) * N, t * N + j] = js.parts[t].apply_S(e.reshape(n, n)).reshape(-1)
    rhs = [rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) for _ in range(T)]
    x_direct = np.linalg.solve(dense, np.concatenate([r.reshape(-1) for r in rhs]))
    xs, _ = O.pcg_joint(js, rhs, [np.zeros((n, n), complex)] * T, 4 * T * N, 1e-14,
                        math.sqrt(O.rdot_joint(rhs, rhs)))
    got = np.concatenate([x.reshape(-1) for x in xs])
    assert np.linalg.norm(got - x_direct) <= 1e-9 * np.linalg.norm(x_direct)
