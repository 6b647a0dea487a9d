"""Benchmark: multimode Floquet eigensolves per second on one GB300 (or N, weak scaling).

Workload (one step): the spin-1 two-mode system H = w0 Fz + O1 cos(w1 t) Fx + O2 cos(w2 t) Fz,
w = (1, (sqrt5-1)/2), N = (10, 10) -> n = 1323, for 64 seeded amplitude pairs (O1, O2) ~
U[0.05, 0.5]^2 (seed 1); per system: H_F assembly, full eigendecomposition, U(t, 0) at 64 times
over 2 pi / w1 and Pbar.  Synthetic inputs; the per-step working set (about 13 GB on the mixed
path, 7 GB on the FP64 path) exceeds L2, so no flush is needed between steps.  With N ranks each
rank solves its own 64 systems (seed 1 + rank).

The headline line times the mixed-precision path; the same process then times the plain FP64
path on the same systems (fp64_value, mixed_over_fp64) and compares both with stored oracle
results (accuracy_vs_oracle).  The CPU baseline runs complete oracle solves, one system per host
core.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
    python bench.py --impl reference      # the FP64 CPU oracle, one system per host core
"""

from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import multiprocessing as mp
import threading
import time
from concurrent.futures import ProcessPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "spin1_bichromatic_n1323_x64"
METRIC = "floquet_eigensolves_per_s"
COUNT, NT = 64, 64

# peaks: measured copy bandwidth / bf16 GEMM (generated file); FP64 / FP32 ALU peaks from
# the nominal 1.25 TFLOP/s FP64 and 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz.
FP64_ALU_PEAK = 1.25e12
FP32_ALU_PEAK = 152 * 128 * 2 * 2.07e9


# DRAM traffic per launch of a dominant kernel (dram__bytes_read.sum + dram__bytes_write.sum) from one
# single-pass ncu capture of the default workload, keyed by (kernel, workload, precision) and
# recorded with the SHA-256 of the kernel's source file at capture time: once that source changes,
# the figure no longer describes the kernel and the roofline reports traffic as null.
MEASURED_TRAFFIC = {
    ("k_sbr_chase", WORKLOAD, "mixed"): (393.52e6 + 6.69e9, "paper_2005_03426_gb300/csrc/k_sbr.cu",
                                         "90700a66c9d8e0cfd3747f6a40de2c21465d75286f9022633e100d741071de0c"),
    ("k_hetrd", WORKLOAD, "mixed"): (194.41e9 + 7.87e9, "paper_2005_03426_gb300/csrc/k_hetrd.cu",
                                     "21b0e78d37918c74e12f76b80e16cc7b1133f64906c9d06ab25408de54e30116"),
}


def _measured_traffic(kernel: str, workload: str, precision: str):
    rec = MEASURED_TRAFFIC.get((kernel, workload, precision))
    if rec is None:
        return None
    import hashlib
    try:
        with open(os.path.join(ROOT, rec[1]), "rb") as f:
            digest = hashlib.sha256(f.read()).hexdigest()
    except OSError:
        return None
    return rec[0] if digest == rec[2] else None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "fallback": True}


class Clocks:
    """nvidia-smi sampling (SM clock, throttle reasons) during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[3 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}



def stage_model(stage: str, n: int, nt: int, mixed: bool, band: int = 0):
    """The bounds of a stage's main kernel for one system on its path (band > 0: the band path
    with half-bandwidth band): a list of (bound, algorithmic work, peak per second, unit, peak
    description, kernel).  The roofline reports the bound whose work / peak is largest (the one
    that limits the kernel).
    - hetrd, dense path: (16/3) n^3 real flops (LAPACK count); the hemv of every column streams
      the trailing lower triangle, sum_m m^2/2 = n^3/6 complex entries (8 bytes FP32, 16 FP64).
    - hetrd, band path (the bulge chase): about 6 b^2 complex multiply-adds per step (the
      one-sided update of the bulge block, the two-sided update of the diagonal block) over
      n^2 / (2 b) steps = 24 b n^2 real flops.
    - backtransform: 8 n^3 real flops (LAPACK count), on either path; in the mixed path from
      n = 256 on (band path: half-bandwidths 33..64, the library's default thresholds) on the
      tensor cores in split TF32, against the TF32 rate (the measured sustained bf16 rate x the
      nominal TF32 / BF16 ratio 1.1 / 2.25).
    - refine_gram: the first refinement step's G on the band |i - j| <= 16 in double-FP32,
      33 n^2 complex multiply-adds = 264 n^2 real flops (FP64-equivalent) against the FP32 rate.
    - outputs: 8 nt n^2 flops (the Phi contraction)."""
    pk = _peaks()
    hbm = pk["hbm_gbs"] * 1e9
    bf16 = pk.get("bf16_tflops_sustained", pk["bf16_tflops"]) * 1e12
    src = "of fallback" if pk.get("fallback") else "of measured"
    alu = (FP32_ALU_PEAK, "FP32 SIMT: 152 SMs x 128 lanes x 2 x 2.07 GHz (derived from unit counts and clock)") \
        if mixed else (FP64_ALU_PEAK, "FP64: nominal 1.25 TFLOP/s")
    if stage == "hetrd":
        if band:
            return [("alu", 24.0 * band * n ** 2, alu[0], "TFLOP/s", alu[1], "k_sbr_chase")]
        esz = 8.0 if mixed else 16.0
        return [("alu", 16.0 / 3.0 * n ** 3, alu[0], "TFLOP/s", alu[1], "k_hetrd"),
                ("hbm", esz * n ** 3 / 6.0, hbm, "GB/s", f"copy bandwidth {pk['hbm_gbs']} GB/s {src}", "k_hetrd")]
    if stage == "backtransform":
        tf32 = bf16 * 1.1 / 2.25
        tc = (f"TF32: cuBLAS bf16 sustained {bf16 / 1e12:.1f} TFLOP/s {src} x 1.1 / 2.25 (nominal ratio)")
        if band:
            if mixed and n >= 256 and 33 <= band <= 64:
                return [("tensor", 8.0 * n ** 3, tf32, "TFLOP/s", tc, "k_sbr_bt_tc")]
            return [("alu", 8.0 * n ** 3, alu[0], "TFLOP/s", alu[1], "k_sbr_bt_f32" if mixed else "k_sbr_bt_f64")]
        if mixed and n >= 256:
            return [("tensor", 8.0 * n ** 3, tf32, "TFLOP/s", tc, "k_tf3_gemm")]
        return [("alu", 8.0 * n ** 3, alu[0], "TFLOP/s", alu[1],
                 "k_backtransform_f32" if mixed else "k_backtransform")]
    if stage == "refine_gram" and mixed:
        return [("alu", 264.0 * n ** 2, alu[0], "TFLOP/s", alu[1], "k_gram_band_df32")]
    if stage == "outputs":
        return [("alu", 8.0 * nt * n * n, alu[0], "TFLOP/s", alu[1], "k_time_evolution")]
    return None


# ------------------------------------------------------------------ CPU baseline (the oracle)
def _oracle_solve_c1(i: int):
    """One complete oracle solve of system i of the benchmark workload (worker process)."""
    from oracle import oracle as O
    from paper_2005_03426_gb300 import workloads as W

    p = W.spin1_amplitude_set(COUNT, seed=1)[i]
    t = W.time_grid(p, NT)
    t0 = time.perf_counter()
    r = O.solve(p, t=t, t0=0.0)
    return time.perf_counter() - t0, int(r["status"])


def _noop(_):
    return os.getpid()


def cpu_baseline_oracle(nsys: int = 0, cores: int = 0):
    """The FP64 oracle as it stands, timed on complete solves (H_F build, cyclic Jacobi to
    convergence, U at the 64 times, Pbar) of the benchmark's systems, one system per host core in
    separate processes (the oracle itself is single-threaded).  nsys systems (default: one per
    core) are solved in one wave; value = nsys / wall time of the wave."""
    cores = cores or os.cpu_count() or 1
    nsys = nsys or cores
    workers = min(cores, nsys)
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        list(ex.map(_noop, range(workers)))  # start the workers before the clock
        t0 = time.perf_counter()
        res = list(ex.map(_oracle_solve_c1, [i % COUNT for i in range(nsys)]))
        wall = time.perf_counter() - t0
    per = [r[0] for r in res]
    return {"value": nsys / wall, "unit": "solves/s", "cores": workers, "kind": "oracle",
            "sample": (f"{nsys} complete oracle solves (systems 0..{nsys - 1} of the workload, n = 1323, "
                       f"U at {NT} times, Pbar) in {workers} processes, one system each; wave {wall:.1f}s, "
                       f"per solve {min(per):.1f}..{max(per):.1f}s"),
            "status_max": max(r[1] for r in res)}


# ------------------------------------------------------------------ serving
def run_serving(M, W, ctx, precision, rate_fracs, n_requests, slots=4, max_batch=16, seed=40,
                max_seconds=None):
    """Poisson request streams through the continuous-batching server.  Saturation throughput is
    measured first with a burst; each rate is a fraction of it.  Latency = submit -> results on host.
    max_seconds bounds the arrival span of one rate (fewer requests at low rates)."""
    problems = W.serving_stream(n_requests, seed=seed)
    systems = [M.System(ctx, p) for p in problems]
    times = [W.time_grid(p, NT) for p in problems]
    srv = M.Server(ctx, slots=slots, max_batch=max_batch, precision=precision)
    # saturation: a burst of everything at once
    burst = min(len(problems), 96)
    t0 = time.perf_counter()
    tk = [srv.submit(systems[i], times[i]) for i in range(burst)]
    for k in tk:
        srv.wait(k)
    sat = burst / (time.perf_counter() - t0)
    out = {"saturation_solves_per_s": sat, "rates": []}
    for r, frac in enumerate(rate_fracs):
        srv.reset_stats()
        rate = frac * sat
        arr = W.poisson_arrivals(len(problems), rate, seed + 1 + r)
        if max_seconds:
            arr = arr[arr <= max_seconds] if (arr <= max_seconds).sum() >= 8 else arr[:8]
        tickets = []
        start = time.perf_counter()
        for i, ta in enumerate(arr):
            now = time.perf_counter() - start
            if ta > now:
                time.sleep(ta - now)
            tickets.append(srv.submit(systems[i], times[i]))
        for k in tickets:
            srv.wait(k)
        wall = time.perf_counter() - start
        st = srv.stats()
        out["rates"].append({"rate_frac": frac, "offered_per_s": rate, "requests": len(tickets),
                             "solves_per_s": len(tickets) / wall, "p50_ms": st["p50_ms"],
                             "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"]})
    srv.close()
    return out


# ------------------------------------------------------------------ multi-rank workload split
def balanced_partition(costs, world: int):
    """Split items with the given costs over `world` ranks: largest cost first, each to the rank
    with the least total so far (ties to the lower rank).  Returns one sorted index list per rank;
    together they cover every item exactly once."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def rank_workload(W, workload: str, count: int, rank: int, world: int):
    """The systems rank `rank` of `world` solves, the systems-per-step count and the length of
    their time grid.  The systems are independent parameter points, so nothing crosses ranks on
    the data path:
    - spin1: each rank takes its own seeded set of `count` systems (weak scaling);
    - uneven: the one 4096-system batch (seed 0) is split over the ranks, balanced by the sum of
      n^3 (the eigensolver's cost), so the ranks share a fixed job (strong scaling);
    - lattice: consecutive slices of one frequency grid of count x world points;
    - large: the single large instance runs as a replica on every rank."""
    nt = NT
    if workload == "uneven":
        total = 4096 if count == COUNT else count
        allp = W.uneven_batch(total, seed=0)
        part = balanced_partition([float(p.n) ** 3 for p in allp], world)[rank]
        problems = [allp[i] for i in part]
        count = len(problems)
    elif workload == "large":
        count, nt = 1, 256
        problems = [W.large_instance(seed=3)]
    elif workload == "lattice":
        # spectrum versus frequency: quasienergies, eigenvectors and Pbar at every frequency of
        # one grid over all ranks (no time grid)
        nt = 0
        problems = W.lattice_sweep(count * world)[rank * count:(rank + 1) * count]
    else:
        problems = W.spin1_amplitude_set(count, seed=1 + rank)
    return problems, count, nt


def scaling_kind(workload: str) -> str:
    return "strong" if workload == "uneven" else "weak"


def max_over_ranks(x: float, world: int, dist, device) -> float:
    """Largest x over the ranks: the job's step time is set by its slowest rank."""
    if world <= 1:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int, dist, device) -> float:
    if world <= 1:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------------ accuracy against the oracle
def golden_c1():
    """Stored oracle results of systems of the benchmark workload: {index: (E, U, P)}."""
    g = {}
    d = os.path.join(ROOT, "tests", "golden")
    f0 = os.path.join(d, "spin1_c1_sys0.npz")
    if os.path.exists(f0):
        z = np.load(f0)
        g[0] = (z["E"], z["U"], z["P"])
    f1 = os.path.join(d, "spin1_c1_sys1_6.npz")
    if os.path.exists(f1):
        z = np.load(f1)
        for i in z["indices"]:
            g[int(i)] = (z[f"E_{i}"], z[f"U_{i}"], z[f"P_{i}"])
    return g


def accuracy(batch, E, U, P, gold):
    """Largest errors of the systems with stored oracle results: quasienergies relative to
    max|E| (= ||H_F||_2), U and Pbar absolute."""
    if not gold:
        return None
    e_rel = u_abs = p_abs = 0.0
    for i, (ge, gu, gp) in gold.items():
        if i >= batch.count:
            continue
        e, u, pp = batch.unpack(E, U, P, i)
        e_rel = max(e_rel, float(np.abs(e - ge).max() / np.abs(ge).max()))
        if u.size:
            u_abs = max(u_abs, float(np.abs(u - gu).max()))
        p_abs = max(p_abs, float(np.abs(pp - gp).max()))
    return {"E_rel_to_normH": e_rel, "U_abs": u_abs, "P_abs": p_abs,
            "systems": sorted(i for i in gold if i < batch.count)}


# ------------------------------------------------------------------ timing
def time_steps(batch, stream, steps: int, barrier, local: int):
    """CUDA-event time of `steps` runs of the batch on its stream (after a synchronize and
    barrier on both sides), per-stage event times, launches and SM clocks sampled meanwhile."""
    import torch

    batch.timing(steps)
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(steps):
            launches += batch.run()
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1) / steps
    stage, runs = batch.stage_ms()
    batch.timing(0)
    per = {k: v / max(runs, 1) for k, v in stage.items()}
    return ms, per, launches, clk.summary()


def run_reference(args):
    """The oracle as it stands on the host cores, on the benchmark workload: each step is one
    wave of complete solves, one system per core.  The number of steps is capped so the run ends
    within a few minutes (a wave takes about as long as one solve, ~40 s)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    steps = max(1, min(args.steps, args.ref_max_steps))
    warm = min(args.warmup, max(0, args.ref_max_steps - steps))
    vals = []
    for s in range(warm + steps):
        cb = cpu_baseline_oracle(nsys=args.ref_systems)
        if s >= warm:
            vals.append(cb["value"])
    value = float(np.mean(vals))
    nsys = args.ref_systems or cb["cores"]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
            "n_gpus": args.gpus, "steps": steps, "warmup": warm,
            "steps_requested": args.steps, "warmup_requested": args.warmup,
            "ms_per_step": nsys / value * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "systems_per_step": nsys, "n": 1323, "nt": NT,
                       "note": "a step is one wave of complete oracle solves, one system per host core"},
            "cpu_baseline": {**cb, "value": value},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--fp64-steps", type=int, default=3,
                    help="timed steps of the FP64 comparison arm (0: skip it)")
    ap.add_argument("--serve", action="store_true", help="only the serving rate sweep")
    ap.add_argument("--workload", default="spin1", choices=["spin1", "uneven", "large", "lattice"],
                    help="spin1: 64 spin-1 systems n=1323 (default); uneven: 4096 systems n=18..2000; "
                         "large: one D=8 three-mode system n=17576 with U at 256 times; "
                         "lattice: 64 frequencies of the D=256 driven lattice, n=1792, spectrum and Pbar")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-seconds", type=float, default=6.0,
                    help="arrival span per rate in the default run's serving sweep")
    ap.add_argument("--count", type=int, default=COUNT,
                    help="systems per step (64 = the benchmark workload; smaller for profiler captures)")
    ap.add_argument("--ref-systems", type=int, default=0,
                    help="reference arm / CPU baseline: systems per wave (default: one per host core)")
    ap.add_argument("--ref-max-steps", type=int, default=2)
    ap.add_argument("--tuning", default=os.path.join(ROOT, "paper_2005_03426_gb300", "tuning_gb300.txt"),
                    help="tuning table of the solver paths (written by paper_2005_03426_gb300/tune.py)")
    ap.add_argument("--no-tuning", action="store_true")
    ap.add_argument("--band-max", type=int, default=-1,
                    help="widest band reduced by the bulge chase (library option; 0: dense reduction only)")
    ap.add_argument("--hetrd-simt", action="store_true",
                    help="mixed path: the dense reduction's trailing update on the FP32 units instead of the tensor cores")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    from paper_2005_03426_gb300 import mmf as M
    from paper_2005_03426_gb300 import workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    # a dedicated stream shared by the library and the timing events (the legacy default
    # stream has handle 0, which the library would read as "make your own")
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)

    def barrier():
        if world > 1:
            dist.barrier()

    prec = M.MMF_MIXED if args.precision == "mixed" else M.MMF_FP64
    if args.serve:
        ctx = M.Context(local, stream=stream.cuda_stream)
        # mixed: the full request count at every rate; FP64 (about 10x slower): arrivals bounded
        # to a minute per rate so that the sweep ends in minutes
        for pname, pp, cap in (("mixed", M.MMF_MIXED, None), ("fp64", M.MMF_FP64, 60.0)):
            res = run_serving(M, W, ctx, pp, [0.1, 0.25, 0.5, 0.75, 0.9], args.serve_requests, max_seconds=cap)
            if rank == 0:
                for rr in res["rates"]:
                    print(json.dumps({"metric": "serving_latency_p50_ms", "value": rr["p50_ms"], "unit": "ms",
                                      "higher_is_better": False, "p99_ms": rr["p99_ms"], "n_gpus": world,
                                      "precision": pname, "data": "synthetic",
                                      "config": {"workload": "poisson_mix_qubit_spin1_uneven_nt64",
                                                 "saturation_solves_per_s": res["saturation_solves_per_s"],
                                                 **rr}}), flush=True)
        return
    problems, count, nt = rank_workload(W, args.workload, args.count, rank, world)
    total_count = int(round(sum_over_ranks(float(count), world, dist, "cuda")))
    ctx = M.Context(local, stream=stream.cuda_stream)
    ctx.set_option(M.MMF_OPT_BAND_MAX, args.band_max)
    ctx.set_option(M.MMF_OPT_HETRD_TC, 0 if args.hetrd_simt else 1)
    tuning = None
    if not args.no_tuning and args.tuning and os.path.exists(args.tuning):
        tuning = {"table": os.path.relpath(args.tuning, ROOT), "rules": ctx.load_tuning(args.tuning)}
    systems = [M.System(ctx, p) for p in problems]
    batch = M.Batch(ctx, systems, prec, nt)
    paths = {}
    sys_band, sys_path = [], []  # each system's path, and its half-bandwidth on the band path (else 0)
    for i in range(batch.count):
        pth, bnd_i = batch.path(i)
        k = ("jacobi", "dense", "whole_gpu", "band")[pth]
        paths[k] = paths.get(k, 0) + 1
        sys_path.append(k)
        sys_band.append(bnd_i if k == "band" else 0)
    ts = np.stack([W.time_grid(p, nt) for p in problems])
    batch.set_times(0.0, ts)

    for _ in range(max(args.warmup, 3 if args.workload != "large" else 1)):
        batch.run()
    st = batch.sync()

    # device-resident timed region
    ms, per, launches, clocks = time_steps(batch, stream, args.steps, barrier, local)
    ms = max_over_ranks(ms, world, dist, "cuda")
    value = total_count / (ms / 1e3)

    # end to end through the public API: H2D of inputs, run, D2H of E, U, Pbar every step
    hE = torch.empty(batch.nE, dtype=torch.float64).pin_memory().numpy()
    hU = torch.empty(max(batch.nU, 1), dtype=torch.complex128).pin_memory().numpy()
    hP = torch.empty(batch.nP, dtype=torch.float64).pin_memory().numpy()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        batch.upload()
        batch.run()
        batch.results(hE, hU, hP)
    e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    e2e_s = max_over_ranks(e2e_s, world, dist, "cuda")
    h2d = 16 * sum(p.D * p.D * (1 + sum(len(c) for c in p.couplings)) for p in problems) + 8 * ts.size
    d2h = hE.nbytes + 16 * batch.nU + hP.nbytes

    # accuracy of the systems with stored oracle results
    is_c1 = args.workload == "spin1" and count == COUNT
    gold = golden_c1() if (rank == 0 and is_c1) else {}
    acc = accuracy(batch, hE, hU, hP, gold)

    # roofline of the dominant kernel (the stage holding it is timed on the library's stream)
    n = problems[0].n
    mixed = prec == M.MMF_MIXED
    modelled = {k: v for k, v in per.items() if stage_model(k, n, nt, mixed) is not None}
    dom = max(modelled, key=modelled.get)
    # the reduction and back-transform stages run the kernels of the systems' own paths; the
    # roofline follows the path most of the batch takes (all systems at the benchmark sizes)
    hh = [i for i in range(len(problems)) if sys_path[i] != "jacobi"]
    if dom in ("hetrd", "backtransform"):
        nband = sum(1 for i in hh if sys_band[i])
        use_band = nband * 2 > len(hh)
        members = [i for i in hh if bool(sys_band[i]) == use_band]
    else:
        members = list(range(len(problems)))
    ref_i = members[0] if members else 0
    bounds = []
    for j, (bnd, _, peak, unit, src, kern) in enumerate(stage_model(dom, problems[ref_i].n, nt, mixed, sys_band[ref_i])):
        work = sum(stage_model(dom, problems[i].n, nt, mixed, sys_band[i])[j][1] for i in members)
        bounds.append((work / peak, bnd, work, peak, unit, src, kern))
    _, bnd, work, peak, unit, src, kern = max(bounds)
    achieved = work / (per[dom] / 1e3) if per[dom] > 0 else 0.0
    scale = 1e9 if unit == "GB/s" else 1e12
    wname = WORKLOAD if is_c1 else None
    roof = {"kernel": kern, "bound": bnd, "achieved": achieved / scale, "peak": peak / scale,
            "unit": unit, "frac": achieved / peak,
            "traffic": _measured_traffic(kern, wname, args.precision) if wname else None,
            "peak_source": src, "work_per_launch": work}

    # the plain FP64 path on the same systems (the metric's comparison arm)
    fp64 = None
    if mixed and args.fp64_steps > 0 and args.workload in ("spin1", "uneven"):
        batch.close()  # the mixed plan's memory goes back before the FP64 plan is made
        b64 = M.Batch(ctx, systems, M.MMF_FP64, nt)
        b64.set_times(0.0, ts)
        b64.run()
        st64 = b64.sync()
        ms64, per64, _, clk64 = time_steps(b64, stream, args.fp64_steps, barrier, local)
        ms64 = max_over_ranks(ms64, world, dist, "cuda")
        E64, U64, P64 = b64.results()
        v64 = total_count / (ms64 / 1e3)
        fp64 = {"value": v64, "ms_per_step": ms64, "steps": args.fp64_steps, "warmup": 1,
                "stage_ms": {k: round(v, 3) for k, v in per64.items()},
                "accuracy_vs_oracle": accuracy(b64, E64, U64, P64, gold),
                "status_max": int(st64.max()), "clocks": clk64}
        b64.close()

    serving = None
    if rank == 0 and world == 1 and args.serve_requests > 0 and is_c1:
        sv = run_serving(M, W, ctx, prec, [0.1, 0.25, 0.5, 0.75, 0.9], args.serve_requests,
                         max_seconds=args.serve_seconds)
        serving = {"saturation_solves_per_s": sv["saturation_solves_per_s"], "rates": sv["rates"],
                   "mix": "1/3 qubit n=82, 1/3 spin-1 n=1323, 1/3 uneven n<=2000; nt=64",
                   "arrival_span_s": args.serve_seconds}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "spin1":
        cpu = cpu_baseline_oracle()

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": scaling_kind(args.workload), "vs_baseline": None,
                "dtype": "f64" if prec == M.MMF_FP64 else "f32+f64",
                "data": "synthetic",
                "config": {"workload": ("uneven_batch_n18_2000_x4096" if args.workload == "uneven" else
                                        "large_D8_three_mode_n17576" if args.workload == "large" else
                                        f"driven_lattice_D256_N3_n1792_x{count}" if args.workload == "lattice" else
                                        WORKLOAD if count == COUNT else f"{WORKLOAD}[:{count}]"),
                           "systems_per_step": total_count, "n": n, "nt": nt,
                           "precision": args.precision, "l2": "working set > L2 (no flush)",
                           "tuning": tuning,
                           "parallelism": f"replicas x{world}" if args.workload != "uneven"
                           else f"instances split by sum n^3 over {world} rank(s)"},
                "stage_ms": {k: round(v, 3) for k, v in per.items()},
                "paths": paths,
                "roofline": roof, "clocks": clocks, "gpu_launches": launches,
                "e2e": {"value": total_count / e2e_s, "unit": "solves/s",
                        "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
                "accuracy_vs_oracle": acc, "status_max": int(st.max()),
                "status_counts": {str(k): int(v) for k, v in zip(*np.unique(st, return_counts=True))},
                "fp64_value": fp64["value"] if fp64 else None,
                "fp64_ms_per_step": fp64["ms_per_step"] if fp64 else None,
                "mixed_over_fp64": value / fp64["value"] if fp64 else None,
                "fp64": fp64,
                "serving": serving,
                "cpu_baseline": cpu}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
