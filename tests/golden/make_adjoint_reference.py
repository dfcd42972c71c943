"""Write the oracle's gradient of the geopotential misfit, for adjoint parity tests.

Workload: two-level MLSDC, fine T85 on 256 x 128 (5 Gauss-Lobatto nodes),
coarse T42 on 128 x 64 (3 nodes), 4 iterations of 1 fine + 2 coarse sweeps,
dt 300 s, 48 steps from the seeded n^-3/2 state (seed 1805).  Objective
J = 1/2 ||Phi'(T) - Phi_t||^2 (Parseval norm) with Phi_t the geopotential of
the seeded state with seed 1806.  Calls only oracle/ and the seeded input
generator.  Output: adjoint_T85_T42_48.npz with J, the gradient dJ/dTheta^0
(complex128 [3][N_c], (Re, Im) convention, Im of m = 0 zero) and the end state.

Usage: python tests/golden/make_adjoint_reference.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import adjoint, sdc  # noqa: E402
from oracle.swe import SWE, Params  # noqa: E402
from paper_1805_07923_gb300 import inputs  # noqa: E402


def main(n_steps=48):
    fine = sdc.Level(SWE(85, 256, 128, Params()), 5)
    coarse = sdc.Level(SWE(42, 128, 64, Params()), 3)
    u0 = inputs.initial_state(85, seed=1805)
    target = inputs.initial_state(85, seed=1806)[0]
    t0 = time.time()
    J, g, uT = adjoint.gradient(fine, coarse, u0, target, 300.0, n_steps, 4, 2)
    out = os.path.join(HERE, f"adjoint_T85_T42_{n_steps}.npz")
    np.savez(out, J=J, grad=g, end_state=uT)
    print(f"J = {J:.16e}, |g| = {np.sqrt(np.sum(np.abs(g) ** 2)):.6e}, {time.time() - t0:.0f} s -> {out}")


if __name__ == "__main__":
    main(*(int(a) for a in sys.argv[1:]))
