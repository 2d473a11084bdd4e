"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

The path shards into independent instances (weak scaling, no collective on
the data path): each rank reconstructs its own seeded instance, the timed
region ends with the maximum of the ranks' times, and the reported value is
the iterations of all ranks divided by that time.  The reference arm runs on
rank 0 only.  These tests run the same functions bench.py calls, in two gloo
processes.
"""
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


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import synth
        wl = synth.get_config(bench.WORKLOAD)
        inst = bench.instance_workload(wl, rank)
        ms = bench.max_over_ranks(10.0 * (rank + 1), world, device="cpu")
        ref = bench.run_reference(type("A", (), dict(warmup=0, steps=0, gpus=world, config=wl.name))(),
                                  rank, world) if rank == 1 else "skipped"
        q.put((rank, inst.seed, ms, ref))
    finally:
        dist.destroy_process_group()


def test_two_ranks_weak_scaling_host_logic():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(world):
        rank, seed, ms, ref = q.get(timeout=120)
        out[rank] = (seed, ms, ref)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sys.path.insert(0, ROOT)
    import bench
    # distinct seeded instances per rank, the same workload otherwise
    assert out[0][0] != out[1][0]
    # every rank sees the slowest rank's time
    assert out[0][1] == out[1][1] == 20.0
    # the reference arm does no work on rank > 0
    assert out[1][2] is None
    # whole-job aggregate: all ranks' iterations over the slowest time
    assert bench.whole_job_value(2, 30, 20.0) == pytest.approx(3000.0)
    assert bench.whole_job_value(1, 30, 20.0) == pytest.approx(1500.0)
