"""The multi-process host logic of the benchmark on CPU (gloo, world size 2):
the whole-job reduction (slowest rank's time, sum of the units) and the
sharding of independent boxes over ranks (each box on exactly one rank, the
same assignment on every rank, balanced loads).  No GPU is used."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402
import synth  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        secs, units = bench.job_totals(1.5 + rank, 1000.0 * (rank + 1))
        specs = synth.batched_systems(count=64, seed=7)
        mine = bench.shard_systems(specs, rank, world)
        ids = [s["seed"] for s in mine]
        gathered = [None] * world
        dist.all_gather_object(gathered, ids)
        out[rank] = (secs, units, gathered, sum(s["n"] for s in mine))
    finally:
        dist.destroy_process_group()


def test_job_totals_and_sharding_over_two_gloo_ranks():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world,
                           start_method="spawn")
        res = dict(out)
    specs = synth.batched_systems(count=64, seed=7)
    all_ids = sorted(s["seed"] for s in specs)
    loads = []
    for rank in range(world):
        secs, units, gathered, load = res[rank]
        assert secs == 2.5                    # the slowest rank
        assert units == 3000.0                # 1000 + 2000
        # the same assignment seen from both ranks, a partition of the boxes
        assert gathered == res[0][2]
        assert sorted(gathered[0] + gathered[1]) == all_ids
        assert not set(gathered[0]) & set(gathered[1])
        loads.append(load)
    biggest = max(s["n"] for s in specs)
    assert max(loads) - min(loads) <= biggest


def test_without_a_process_group_totals_are_the_rank_values():
    assert bench.job_totals(2.0, 7.0) == (2.0, 7.0)
    specs = synth.batched_systems(count=10, seed=3)
    assert bench.shard_systems(specs, 0, 1) == specs
