"""Write the stored converged solution x* used by the 256^2 TV + D4 parity test.

Calls only the FP64 oracle and the seeded input generator.  x* is the unique
minimiser of F_eps for the 256x256 TV + 4-level D4 workload (seed 2); it is
reached by running FIRLS (Alg. 3 with the wavelet term added, 60 PCG steps
per outer step so that each outer step is nearly exact) until the relative
change falls below 1e-9.  A strided sample x*[::4, ::4] (64 x 64 complex
values) is stored; the GPU test compares its result on the same pixels.

    python tests/golden/make_xstar.py [seed ...]     (default: 2)
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import firls_synth as fs  # noqa: E402
from oracle import firls_oracle as O  # noqa: E402

def out_path(seed):
    return os.path.join(HERE, f"xstar_tv_db4_256_seed{seed}_stride4.npy")


def main(seeds):
    for seed in seeds:
        p = fs.tv_db4_256(seed=seed)
        x, info = O.firls_problem(p, outer=1500, inner=60, outer_tol=1e-9)
        print("seed", seed, "outer steps", info["outer_done"], "last relative change", info["rel_change"][-1])
        np.save(out_path(seed), np.asarray(x)[::4, ::4].astype(np.complex128))
        print("wrote", out_path(seed))


if __name__ == "__main__":
    main([int(a) for a in sys.argv[1:]] or [2])
