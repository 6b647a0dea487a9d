"""Multi-rank path of bench.py on CPU: world size 2 over gloo (no GPU).

With N ranks, each rank solves its own systems and only the step time crosses ranks (the max
over ranks). These tests check three things:
- the sharding gives disjoint system sets that together make up the intended workload;
- the reduction returns the slowest rank's time on every rank;
- a rank's problems do not depend on anything but (rank, world).
"""

import importlib.util
import os
import socket

import numpy as np
import pytest

from paper_2005_03426_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_lattice_sweep_shards_partition_the_grid():
    B = _bench()
    world, count = 3, 5
    shards = [B.rank_workload(W, "lattice", count, r, world) for r in range(world)]
    ws = np.concatenate([[p.omegas[0] for p in probs] for probs, _, _ in shards])
    np.testing.assert_array_equal(ws, np.linspace(0.2, 1.0, world * count))
    assert all(c == count and nt == 0 for _, c, nt in shards)
    # one rank alone is the single-GPU benchmark grid
    probs, _, _ = B.rank_workload(W, "lattice", 64, 0, 1)
    np.testing.assert_array_equal([p.omegas[0] for p in probs], np.linspace(0.2, 1.0, 64))


def test_random_workloads_differ_between_ranks():
    B = _bench()
    a, _, _ = B.rank_workload(W, "spin1", 3, 0, 2)
    b, _, _ = B.rank_workload(W, "spin1", 3, 1, 2)
    assert not np.array_equal(a[0].couplings[0][0], b[0].couplings[0][0])
    a2, _, _ = B.rank_workload(W, "spin1", 3, 0, 2)
    assert np.array_equal(a[0].couplings[0][0], a2[0].couplings[0][0])  # seeded: reproducible


def test_uneven_batch_split_covers_it_once_and_balances_n_cubed():
    B = _bench()
    allp = W.uneven_batch(4096, seed=0)
    cost = np.array([float(p.n) ** 3 for p in allp])
    for world in (2, 3, 8):
        shards = [B.rank_workload(W, "uneven", 64, r, world) for r in range(world)]
        assert sum(c for _, c, _ in shards) == 4096
        parts = B.balanced_partition(list(cost), world)
        idx = np.sort(np.concatenate(parts))
        np.testing.assert_array_equal(idx, np.arange(4096))  # every system exactly once
        # the shards are the batch's own systems (same bytes), in batch order
        for (probs, _, _), part in zip(shards, parts):
            assert [p.n for p in probs] == [allp[i].n for i in part]
            assert np.array_equal(probs[0].H0, allp[part[0]].H0)
        loads = np.array([cost[p].sum() for p in parts])
        # greedy largest-first: no rank exceeds the mean by more than the largest single system
        assert loads.max() - loads.mean() <= cost.max()
        assert loads.max() / loads.mean() < 1.01
    assert B.scaling_kind("uneven") == "strong" and B.scaling_kind("spin1") == "weak"


def test_balanced_partition_small_cases():
    B = _bench()
    assert B.balanced_partition([5.0, 1.0, 1.0, 3.0], 2) == [[0], [1, 2, 3]]
    assert B.balanced_partition([1.0], 3) == [[0], [], []]
    assert B.balanced_partition([], 2) == [[], []]


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        B = _bench()
        # each rank reports a different step time; every rank must see the largest
        ms = B.max_over_ranks(10.0 + 7.0 * rank, world, dist, "cpu")
        probs, count, _ = B.rank_workload(W, "lattice", 4, rank, world)
        np.save(os.path.join(out_dir, f"rank{rank}.npy"),
                np.array([ms, count] + [p.omegas[0] for p in probs]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_and_shards(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [np.load(tmp_path / f"rank{r}.npy") for r in range(world)]
    for r in res:
        assert r[0] == 17.0  # max over ranks, seen by every rank
        assert r[1] == 4
    ws = np.concatenate([r[2:] for r in res])
    np.testing.assert_array_equal(ws, np.linspace(0.2, 1.0, 8))
    # value = systems over all ranks / slowest rank's time
    assert world * res[0][1] / (res[0][0] / 1e3) == pytest.approx(8 / 0.017)
