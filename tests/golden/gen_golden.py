"""Write the stored expected values of the full-size parity tests.

Calls only the FP64 CPU oracle (oracle/) on seeded synthetic inputs from the workloads
module; nothing here touches the CUDA path.  Run from the repository root:

    python tests/golden/gen_golden.py [c1] [c2]

Outputs (NumPy .npz):
  spin1_c1_sys0.npz     spin-1 two-mode system, amplitude pair 0 of the 64-pair set (seed 1),
                        N = (10, 10), n = 1323: all quasienergies, U(t_k, 0) on 64 uniform times
                        over 2 pi / omega_1, Pbar, and the oracle's Jacobi sweep count.
  spin1_c1_sys1_6.npz   the same for amplitude pairs 1..6 of that set (keys E_i, U_i, P_i,
                        sweeps_i; `indices` lists i).
  uneven_c2_sample.npz  20 systems of the 4096-system uneven batch (seed 0), chosen at the
                        0, 1/19, ..., 1 quantiles of n (18 ... 1998): E, U on 64 times, Pbar
                        (keys as above; `indices` are positions in the batch).
The solves run in parallel worker processes (one system per process).
"""

import os
import sys
import time
from concurrent.futures import ProcessPoolExecutor
import multiprocessing as mp

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
from paper_2005_03426_gb300 import workloads as W  # noqa: E402

NT = 64


def c2_sample_indices(ps, k: int = 20):
    """Positions of k systems of the uneven batch at evenly spaced quantiles of n (stable order)."""
    ns = np.array([p.n for p in ps])
    order = np.argsort(ns, kind="stable")
    q = np.linspace(0, len(ns) - 1, k).round().astype(int)
    return [int(i) for i in order[q]]


def _solve(args):
    kind, i = args
    if kind == "c1":
        p = W.spin1_amplitude_set(64, seed=1)[i]
    else:
        p = W.uneven_batch(4096, seed=0)[i]
    t = W.time_grid(p, NT)
    t0 = time.time()
    r = O.solve(p, t=t, t0=0.0)
    return kind, i, p.n, r["E"], r["U"], r["P"], r["status"], r["sweeps"], time.time() - t0


def spin1_c1_sys0():
    p = W.spin1_amplitude_set(64, seed=1)[0]
    t = W.time_grid(p, NT)
    t0 = time.time()
    r = O.solve(p, t=t, t0=0.0)
    np.savez_compressed(os.path.join(HERE, "spin1_c1_sys0.npz"), E=r["E"], U=r["U"], P=r["P"],
                        t=t, status=r["status"], sweeps=r["sweeps"])
    print(f"spin1_c1_sys0: n={p.n} status={r['status']} sweeps={r['sweeps']} "
          f"{time.time() - t0:.1f}s")


def _write(name, results):
    out = {"indices": np.array([r[1] for r in results], dtype=np.int64)}
    for kind, i, n, E, U, P, st, sw, dt in results:
        assert st == 0, (kind, i, st)
        out[f"E_{i}"], out[f"U_{i}"], out[f"P_{i}"], out[f"sweeps_{i}"] = E, U, P, np.int64(sw)
        print(f"{name}: system {i} n={n} sweeps={sw} {dt:.1f}s")
    np.savez_compressed(os.path.join(HERE, name), **out)


def main(which):
    O.build()
    jobs = []
    if "c1" in which:
        jobs += [("c1", i) for i in range(1, 7)]
    if "c2" in which:
        jobs += [("c2", i) for i in c2_sample_indices(W.uneven_batch(4096, seed=0))]
    # largest first so the long solves start at once
    sizes = {("c1", i): 1323 for i in range(64)}
    if "c2" in which:
        ps = W.uneven_batch(4096, seed=0)
        sizes.update({("c2", i): ps[i].n for _, i in jobs if _ == "c2"})
    jobs.sort(key=lambda j: -sizes[j])
    with ProcessPoolExecutor(max_workers=os.cpu_count(), mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_solve, jobs))
    c1 = sorted([r for r in res if r[0] == "c1"], key=lambda r: r[1])
    c2 = [r for r in res if r[0] == "c2"]
    if c1:
        _write("spin1_c1_sys1_6.npz", c1)
    if c2:
        _write("uneven_c2_sample.npz", c2)


if __name__ == "__main__":
    args = sys.argv[1:] or ["c1", "c2"]
    if "c1sys0" in args:
        spin1_c1_sys0()
    main([a for a in args if a in ("c1", "c2")])
