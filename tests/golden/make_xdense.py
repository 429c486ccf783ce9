"""Write the FP64 oracle's result of the dense random-projection workload.

Calls only the FP64 oracle and the seeded input generator.  For each seed:
the 1-D problem of Sec. 5.3 (firls_synth.dense_l1: length 4000, 10 %
non-zeros, 800 Gaussian measurements, lambda 0.05), FIRLS_L1 with the
proposed preconditioner from A^T b for OUTER outer steps of INNER PCG steps
(the paper runs 30 PCG steps per outer step and sees convergence within 200
iterations).  One file per seed, ``xdense_l1/seed<S>.npz``: x (float64), the
relative changes and the MSE against the sparse ground truth.  The dense GPU
test and the bench compare with these.

    python tests/golden/make_xdense.py [--procs P] [seed ...]
"""
import argparse
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "xdense_l1")
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

OUTER = 200
INNER = 30
DEFAULT_SEEDS = [1, 2]


def solve(seed):
    import firls_synth as fs
    from oracle import dense_oracle as D
    p = fs.dense_l1(seed)
    t0 = time.time()
    x, info = D.firls_l1(p.A, p.b, p.lam, outer=OUTER, inner=INNER)
    mse = float(np.mean((x - p.x0) ** 2))
    np.savez(os.path.join(OUT, f"seed{seed}.npz"), x=x, outer=OUTER, inner=INNER,
             rel_change=np.asarray(info["rel_change"]), mse=mse)
    return seed, mse, info["rel_change"][-1], time.time() - t0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=2)
    ap.add_argument("seeds", type=int, nargs="*")
    a = ap.parse_args()
    os.makedirs(OUT, exist_ok=True)
    with mp.get_context("spawn").Pool(a.procs) as pool:
        for seed, mse, rel, sec in pool.imap_unordered(solve, a.seeds or DEFAULT_SEEDS):
            print(f"seed {seed}: MSE {mse:.4f}, last relative change {rel:.3e}, {sec:.0f} s", flush=True)


if __name__ == "__main__":
    main()
