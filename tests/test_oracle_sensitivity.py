"""Why parity for the TV + Daubechies-4 workloads is taken at the converged
minimiser x* rather than at a fixed schedule's iterate (pure FP64, CPU).

For the combined TV + wavelet regulariser (workloads 2, 4, 5) the reweighting
map of Alg. 3 is locally expanding along some directions during the first
outer steps: a relative perturbation of 1e-9 in x^1 (far below FP32 rounding)
grows to more than 1e-4 within the 50 x 20 schedule, so no implementation whose
rounding differs from the oracle's can reproduce that iterate to 1e-4.  Both
runs nevertheless converge to the same point, the unique minimiser of the
strictly convex F_eps (Theorem 2: monotone; Theorem 3: its stationary point),
where a 1e-4 comparison is meaningful.
"""
import numpy as np

import firls_synth as fs
from oracle import firls_oracle as O


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_tv_db4_iterates_separate_then_converge_together():
    p = fs.make_problem(64, 0.20, 0.01, 2, real=False, psi=fs.PSI_TV | fs.PSI_DB4, levels=4, lam=5e-4,
                        lam_tv=1e-3)
    rhs = O.op_AH(p.mask * p.b, p.mask.astype(np.float64), False)
    r = np.random.default_rng(7)
    pert = r.standard_normal(rhs.shape) + 1j * r.standard_normal(rhs.shape)
    pert *= 1e-9 * np.linalg.norm(rhs) / np.linalg.norm(pert)
    xa, xb = rhs.copy(), rhs + pert

    def run(x, outer):
        return O.firls_problem(p, outer=outer, inner=20, x_init=x)[0]

    xa, xb = run(xa, 10), run(xb, 10)
    assert _rel(xb, xa) > 1e-4            # 1e-9 -> ~1e-3 after ten outer steps
    xa, xb = run(xa, 40), run(xb, 40)
    assert _rel(xb, xa) > 1e-4            # still apart at the end of the 50 x 20 schedule
    xa, xb = run(xa, 110), run(xb, 110)
    assert _rel(xb, xa) < 1e-5            # 160 outer steps: both near the same x*
