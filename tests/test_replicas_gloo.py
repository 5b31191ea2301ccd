"""The N > 1 host path of bench.py on CPU: two gloo ranks (world size 2)
run as independent replicas (different seeds, scenes and weights) and agree
on the slowest rank's time, the only cross-rank operation."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import argparse

    import bench
    args = argparse.Namespace(width=32, height=18, prims=64)
    seed = bench.replica_seed(rank)
    _, params, frames = bench.build_workload(args, seed_offset=seed - 1)
    slowest = bench.max_over_ranks(10.0 + rank, torch.device("cpu"))
    out[rank] = (seed, float(params[:1000].sum()), int(frames[0].blob().sum()), slowest)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_with_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = [out[r] for r in range(world)]
    seeds, psums, bsums, slowest = zip(*res)
    assert len(set(seeds)) == world             # independent replicas
    assert psums[0] != psums[1] and bsums[0] != bsums[1]
    assert all(np.isclose(s, 10.0 + world - 1) for s in slowest)  # max over ranks
