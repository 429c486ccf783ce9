"""Write the FP64 oracle's result of the 512^2 overlapping-group workload.

Calls only the FP64 oracle and the seeded input generator.  For each seed:
the 512x512 slice with 5-level D4 parent-child tree groups (firls_synth.
tree_db4_512: 15 % mask, sigma 0.005, lambda 2e-4), FIRLS_OG (Alg. 2) from
A^H b for OUTER outer steps of INNER PCG steps, the paper's budget of 100
iterations for the tree-sparsity comparison with 20 PCG steps each (within
the 10 to 30 it finds sufficient).  One file per seed,
``xtree_db4_512/seed<S>.npz``: x (complex64), the relative changes and the
SNR against the phantom.  The GPU test and the bench compare with these.

    python tests/golden/make_xtree.py [--procs P] [seed ...]
"""
import argparse
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "xtree_db4_512")
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

OUTER = 100
INNER = 20
DEFAULT_SEEDS = [3, 4]


def solve(seed):
    import firls_synth as fs
    from oracle import firls_oracle as O
    p = fs.tree_db4_512(seed=seed)
    t0 = time.time()
    x, info = O.firls_problem(p, outer=OUTER, inner=INNER)
    snr = 20 * np.log10(np.linalg.norm(p.x0) / np.linalg.norm(x - p.x0))
    np.savez(os.path.join(OUT, f"seed{seed}.npz"), x=np.asarray(x).astype(np.complex64), outer=OUTER, inner=INNER,
             rel_change=np.asarray(info["rel_change"]), snr_db=snr)
    return seed, snr, info["rel_change"][-1], time.time() - t0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=2)
    ap.add_argument("seeds", type=int, nargs="*")
    a = ap.parse_args()
    os.makedirs(OUT, exist_ok=True)
    with mp.get_context("spawn").Pool(a.procs) as pool:
        for seed, snr, rel, sec in pool.imap_unordered(solve, a.seeds or DEFAULT_SEEDS):
            print(f"seed {seed}: SNR {snr:.2f} dB, last relative change {rel:.3e}, {sec:.0f} s", flush=True)


if __name__ == "__main__":
    main()
