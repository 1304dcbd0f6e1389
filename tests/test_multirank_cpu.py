"""The multi-replica path of bench.py on CPU: two gloo ranks (127.0.0.1).
Each rank draws its own batch (distinct seeds, weak scaling) and the job
time is the maximum over ranks; nothing else is exchanged."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2509_12086_gb300 import synth
    seed = bench.replica_seed(rank)
    X = synth.power_law(64, 16, 1.0, seed=seed)
    t = bench.max_over_ranks(world, 1.0 + rank, device="cpu")
    bench.barrier(world)
    q.put((rank, seed, float(X[0, 0]), t))
    dist.destroy_process_group()


def test_two_gloo_replicas():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert out[0][1] != out[1][1]          # distinct seeds
    assert out[0][2] != out[1][2]          # distinct batches
    assert out[0][3] == out[1][3] == 2.0   # max over ranks
