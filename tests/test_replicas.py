"""The N-GPU path of bench.py runs independent replicas (no collective on the data path): the
whole-job numbers are the slowest rank's time and the work summed over ranks, and every rank
draws its own seeded workload.  Checked here with world_size-2 gloo process groups on CPU."""
import os
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, u, e = bench.reduce_over_ranks(dist, 10.0 + 5.0 * rank, 1000.0 * (rank + 1), 3.0 + rank, "cpu")
    out[rank] = (t, u, e)
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_ranks_gloo_world_size_2():
    port = 29500 + (os.getpid() % 2000)
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        assert res[r] == (15.0, 3000.0, 7.0)


def test_single_process_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(None, 4.5, 12.0, 3.0, "cpu") == (4.5, 12.0, 3.0)


def test_replicas_draw_distinct_workloads():
    from paper_2402_08404_gb300 import synth
    cfg = dict(synth.CONFIGS["small"])
    a = synth.plasma(cfg, seed=cfg["seed"] + 0)
    b = synth.plasma(cfg, seed=cfg["seed"] + 1)
    assert not np.array_equal(a["e"]["x"], b["e"]["x"])
    assert len(a["e"]["x"]) == len(b["e"]["x"])      # the same work per rank: weak scaling


def test_reference_arm_runs_on_rank_0_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(config="small", cpu_sample=2000, steps=1, warmup=0)
    assert bench.run_reference(args) is None


def _ens_rank(rank, world, port, n, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    idx = bench.ensemble_share(n, world, rank)
    rows = [[float(i), float(i * i) + 0.5, float(rank)] for i in idx]     # stands in for an instance's diagnostics
    out[rank] = (idx, bench.gather_instances(dist, idx, rows, n, "cpu"))
    dist.barrier()
    dist.destroy_process_group()


def test_ensemble_partition_gloo_world_size_2():
    """The ensemble is split over the ranks: every instance is stepped by exactly one rank, and
    the gathered per-instance table equals the one a single process writes for all instances."""
    sys.path.insert(0, ROOT)
    import bench
    n = 13
    port = 31500 + (os.getpid() % 2000)
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_ens_rank, args=(2, port, n, out), nprocs=2, join=True)
        res = dict(out)
    shares = [res[r][0] for r in (0, 1)]
    assert sorted(shares[0] + shares[1]) == list(range(n)) and not set(shares[0]) & set(shares[1])
    one = bench.gather_instances(None, list(range(n)), [[float(i), float(i * i) + 0.5, 0.0] for i in range(n)], n, "cpu")
    for r in (0, 1):
        table = res[r][1]
        assert not np.isnan(table).any()
        assert np.array_equal(table[:, :2], one[:, :2])
        assert np.array_equal(table[:, 2], np.array([i % 2 for i in range(n)], dtype=float))   # the rank that stepped it
