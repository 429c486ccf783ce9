"""Write the FP64 oracle's result of the multi-contrast workload's schedule.

Calls only the FP64 oracle and the seeded input generator.  For each seed:
the 3-contrast 256^2 cross section with joint 4-level D4 sparsity
(firls_synth.mt_db4_256), FIRLS_MT (Sec. 5.6: Alg. 2 on the stacked
contrasts with joint weights) from A^H b for OUTER outer steps of INNER PCG
steps, the budget of 100 iterations the paper gives every method in its
multi-contrast comparison, with INNER in the 10 to 30 PCG steps it finds
sufficient.  One file per seed, ``xmt_db4_256/seed<S>.npz``: x (complex64
[3][256][256]), the relative changes and the SNR of each contrast against
its phantom.  The multi-contrast GPU test and the bench compare with these.

    python tests/golden/make_xmt.py [--procs P] [seed ...]
"""
import argparse
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "xmt_db4_256")
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

OUTER = 100
INNER = 20
DEFAULT_SEEDS = [1, 2]


def out_path(seed):
    return os.path.join(OUT, f"seed{seed}.npz")


def solve(seed):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import firls_synth as fs
    from oracle import firls_oracle as O
    probs = fs.mt_db4_256(seed)
    p0 = probs[0]
    t0 = time.time()
    xs, info = O.firls_joint([p.b for p in probs], [p.mask for p in probs], psi=p0.psi, levels=p0.levels,
                             lam=p0.lam, lam_tv=p0.lam_tv, outer=OUTER, inner=INNER)
    snr = [20 * np.log10(np.linalg.norm(p.x0) / np.linalg.norm(x - p.x0)) for p, x in zip(probs, xs)]
    np.savez(out_path(seed), x=np.stack(xs).astype(np.complex64), outer=OUTER, inner=INNER,
             rel_change=np.asarray(info["rel_change"]), snr_db=np.asarray(snr))
    return seed, snr, info["rel_change"][-1], time.time() - t0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=2)
    ap.add_argument("seeds", type=int, nargs="*")
    a = ap.parse_args()
    os.makedirs(OUT, exist_ok=True)
    with mp.get_context("spawn").Pool(a.procs) as pool:
        for seed, snr, rel, sec in pool.imap_unordered(solve, a.seeds or DEFAULT_SEEDS):
            print(f"seed {seed}: SNR {', '.join(f'{s:.2f}' for s in snr)} dB, last relative change {rel:.3e}, "
                  f"{sec:.0f} s", flush=True)


if __name__ == "__main__":
    main()
