"""The multi-GPU form of the bench is N independent replicas (the path has no
exchange step): each rank localizes its own queries and the job's throughput
is every rank's work over the slowest rank's time.  Its host logic runs here
as two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        hidden, seeds = bench.rank_queries(rank)
        shards = [None] * world
        dist.all_gather_object(shards, [tuple(map(float, h)) for h in hidden])
        my_time = 2.0 + 1.5 * rank                       # rank 1 is the slowest replica
        slowest = bench.max_over_ranks(dist, my_time, torch.device("cpu"))
        value = bench.job_throughput(world, 64 * 20, slowest)
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            f.write(repr({"shards": shards, "n": len(hidden), "n_seeds": len(seeds),
                          "slowest": slowest, "value": value}))
    finally:
        dist.destroy_process_group()


def test_two_replicas_gloo(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    res = [eval(open(tmp_path / f"rank{r}.txt").read()) for r in range(world)]
    sys.path.insert(0, ROOT)
    import bench
    for r in res:
        assert r["n"] == r["n_seeds"] == bench.N_QUERIES
        assert r["slowest"] == 3.5                       # max over ranks, seen by every rank
        assert r["value"] == pytest.approx(2 * 64 * 20 / 3.5)
        assert r["shards"] == res[0]["shards"]
    a, b = res[0]["shards"]
    assert not set(a) & set(b)                           # disjoint queries per replica
    # rank 0 holds the single-GPU workload's queries
    h0, _ = bench.rank_queries(0)
    assert a == [tuple(map(float, h)) for h in h0]


def test_single_process_has_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, 1.25, None) == 1.25
    assert bench.job_throughput(1, 1280, 0.5) == 2560
