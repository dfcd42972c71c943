"""Write the oracle's end state of the headline run, for full-run parity tests.

Workload: two-level MLSDC, fine T170 on 512 x 256, coarse T85 on 256 x 128,
5/3 Gauss-Lobatto nodes, 4 iterations with 1 fine + 2 coarse sweeps, dt 150 s,
400 steps, from the seeded n^-3/2 state (seed 1805).  Calls only oracle/ and
the seeded input generator.  Output: headline_T170_T85_400.npy (complex128
[3][N_c]) and a checkpoint every 50 steps so a long run can resume.

Usage: python tests/golden/make_headline_reference.py [n_steps]
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import sdc  # noqa: E402
from oracle.swe import SWE, Params  # noqa: E402
from paper_1805_07923_gb300 import inputs  # noqa: E402


def main(n_steps=400):
    out = os.path.join(HERE, f"headline_T170_T85_{n_steps}.npy")
    ckpt = os.path.join(HERE, f".headline_ckpt_{n_steps}.npz")
    fine = sdc.Level(SWE(170, 512, 256, Params()), 5)
    coarse = sdc.Level(SWE(85, 256, 128, Params()), 3)
    u = inputs.initial_state(170, seed=1805)
    start = 0
    if os.path.exists(ckpt):
        d = np.load(ckpt)
        u, start = d["u"], int(d["step"])
    t0 = time.time()
    for step in range(start, n_steps):
        u = sdc.mlsdc_step(fine, coarse, u, 150.0, 4, 2)
        if (step + 1) % 50 == 0:
            np.savez(ckpt, u=u, step=step + 1)
            print(f"step {step + 1}  {time.time() - t0:.0f} s", flush=True)
    np.save(out, u)
    if os.path.exists(ckpt):
        os.remove(ckpt)
    print("wrote", out)


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 400)
