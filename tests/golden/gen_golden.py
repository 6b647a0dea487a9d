"""Write the stored expected values of the full-size parity tests.

Calls only the FP64 CPU oracle (oracle/) on seeded synthetic inputs from the workloads
module; nothing here touches the CUDA path.  Run from the repository root:

    python tests/golden/gen_golden.py

Outputs (NumPy .npz, one per case):
  spin1_c1_sys0.npz   spin-1 two-mode system, amplitude pair 0 of the 64-pair set (seed 1),
                      N = (10, 10), n = 1323: all quasienergies, U(t_k, 0) on 64 uniform times
                      over 2 pi / omega_1, Pbar, and the oracle's Jacobi sweep count.
"""

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
from paper_2005_03426_gb300 import workloads as W  # noqa: E402


def spin1_c1_sys0():
    p = W.spin1_amplitude_set(64, seed=1)[0]
    t = W.time_grid(p, 64)
    t0 = time.time()
    r = O.solve(p, t=t, t0=0.0)
    np.savez_compressed(os.path.join(HERE, "spin1_c1_sys0.npz"), E=r["E"], U=r["U"], P=r["P"],
                        t=t, status=r["status"], sweeps=r["sweeps"])
    print(f"spin1_c1_sys0: n={p.n} status={r['status']} sweeps={r['sweeps']} "
          f"{time.time() - t0:.1f}s")


if __name__ == "__main__":
    spin1_c1_sys0()
