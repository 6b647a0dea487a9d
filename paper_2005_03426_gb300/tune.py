"""Autotuner of the solver-path choices: for each size bucket and band class of a set of sample
systems, time the candidate paths on the device and write a tuning table that
``Context.load_tuning`` (``mmf_ctx_load_tuning``) reads.

Candidates per bucket (only those the bucket allows):
  - the shared-memory Jacobi kernel (n within its maximum) or the Householder paths;
  - for the Householder paths, the band path (bulge chase on H_F's band, half-bandwidth <= 64)
    or the dense reduction;
  - for the mixed path's dense reduction, the back-transform on the tensor cores or on the FP32
    units.
A rule depends only on a system's n and half-bandwidth, so a system takes the same path whatever
else is in its batch.  Timing: one warm-up run, then the mean of ``reps`` runs of a batch of up to
``sample`` systems spread evenly over the bucket (host clock around device-synchronised runs), per system.

    python -m paper_2005_03426_gb300.tune --out paper_2005_03426_gb300/tuning_gb300.txt
"""

from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_2005_03426_gb300 import mmf as M  # noqa: E402
from paper_2005_03426_gb300 import workloads as W  # noqa: E402

N_EDGES = [1, 33, 65, 85, 119, 192, 256, 384, 512, 768, 1024, 1400, 2048, 3072, 2 ** 31 - 1]
BAND_CLASSES = [(0, 8), (9, 16), (17, 32), (33, 48), (49, 64), (65, 2 ** 31 - 1)]
JACOBI_MAX = {M.MMF_FP64: 84, M.MMF_MIXED: 118}
NAMES = {M.MMF_FP64: "fp64", M.MMF_MIXED: "mixed"}


def bucket_of(n: int, band: int):
    for a, bnd in zip(N_EDGES[:-1], N_EDGES[1:]):
        if a <= n < bnd:
            nb = (a, bnd - 1)
            break
    for lo, hi in BAND_CLASSES:
        if lo <= band <= hi:
            return nb, (lo, hi)
    raise ValueError(band)


def default_samples():
    """The workloads' system types: the uneven batch (seed 0), the spin-1 benchmark set, the qubit
    sweep and the driven lattice."""
    ps = list(W.uneven_batch(4096, seed=0))
    ps += W.spin1_amplitude_set(64, seed=1)
    ps += W.qubit_sweep(64)
    ps += W.lattice_sweep(16)
    return ps


def spread(items, sample):
    """Up to ``sample`` items evenly spaced over the list (so that every source workload in a
    bucket is represented)."""
    if len(items) <= sample:
        return list(items)
    return [items[int(k * len(items) / sample)] for k in range(sample)]


def candidates(precision, nb, band_cls, any_band_ok):
    out = []
    if nb[0] <= JACOBI_MAX[precision]:
        out.append((1, -1, -1))
    if nb[1] > 4:
        bands = [0, 1] if any_band_ok else [0]
        for bd in bands:
            if precision == M.MMF_MIXED and bd == 0 and nb[1] >= 128:
                out += [(0, 0, 1), (0, 0, 0)]
            else:
                out.append((0, bd, -1))
    return out


def time_config(precision, rule, problems, nt, reps):
    ctx = M.Context(0)
    ctx.add_rule(precision, *rule)
    systems = [M.System(ctx, p) for p in problems]
    b = M.Batch(ctx, systems, precision, nt)
    if nt:
        b.set_times(0.0, np.stack([W.time_grid(p, nt) for p in problems]))
    b.run()
    st = b.sync()
    t0 = time.perf_counter()
    for _ in range(reps):
        b.run()
    b.sync()
    dt = (time.perf_counter() - t0) / reps
    paths = sorted({b.path(i)[0] for i in range(b.count)})
    b.close()
    for s in systems:
        s.close()
    ctx.close()
    return dt / len(problems), int(st.max()), paths


def tune(precisions, problems, sample=64, reps=2, nt=64, log=print):
    groups = {}
    ctx = M.Context(0)
    for p in problems:
        s = M.System(ctx, p)  # the library's own half-bandwidth of H_F
        band = s.bandwidth()
        s.close()
        groups.setdefault(bucket_of(p.n, band), []).append((p, band))
    ctx.close()
    lines = []
    for precision in precisions:
        for (nb, bc) in sorted(groups):
            items = spread(groups[(nb, bc)], sample)
            ps = [p for p, _ in items]
            band_ok = any(band <= 64 and p.n >= 2 * band + 2 for p, band in items)
            cands = candidates(precision, nb, bc, band_ok)
            if len(cands) < 2:
                continue
            res = []
            for cand in cands:
                rule = (nb[0], nb[1], bc[0], bc[1]) + cand
                ms, st, paths = time_config(precision, rule, ps, nt, reps)
                res.append((ms * 1e3, cand, st, paths))
                log(f"{NAMES[precision]} n {nb} band {bc} x{len(ps)}: {cand} -> {ms * 1e3:.3f} ms/system"
                    f" (paths {paths}, status {st})")
            ok = [r for r in res if r[2] == 0] or res
            best = min(ok, key=lambda r: r[0])
            note = " | ".join(f"{c}:{t:.3f}" for t, c, _, _ in res)
            lines.append(f"{NAMES[precision]} {nb[0]} {nb[1]} {bc[0]} {bc[1]} {best[1][0]} {best[1][1]} {best[1][2]}"
                         f"   # ms/system (jacobi,band,bt_tc): {note}; {len(ps)} systems")
    return lines


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_gb300.txt"))
    ap.add_argument("--precision", nargs="+", default=["mixed", "fp64"], choices=["mixed", "fp64"])
    ap.add_argument("--sample", type=int, default=64)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--nt", type=int, default=64)
    args = ap.parse_args()
    precs = [M.MMF_MIXED if x == "mixed" else M.MMF_FP64 for x in args.precision]
    t0 = time.time()
    lines = tune(precs, default_samples(), sample=args.sample, reps=args.reps, nt=args.nt)
    try:
        import torch

        dev = torch.cuda.get_device_name(0)
    except Exception:
        dev = "unknown device"
    with open(args.out, "w") as f:
        f.write(f"# tuning table of the solver paths, measured on {dev} by paper_2005_03426_gb300/tune.py\n")
        f.write(f"# ({time.time() - t0:.0f} s; samples: uneven batch seed 0, spin-1 set, qubit sweep, lattice)\n")
        f.write("# precision n_lo n_hi band_lo band_hi jacobi band bt_tc\n")
        for ln in lines:
            f.write(ln + "\n")
    print(f"wrote {len(lines)} rules to {args.out}")


if __name__ == "__main__":
    main()
