"""The multi-GPU path of bench.py is independent replicas (one core hole per
rank, no data-path collective): the timing is the maximum over ranks and the
whole-job throughput is world * steps / that maximum.  Checked here with two
gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    elapsed = 1.5 + rank          # rank 1 is the slower replica
    mx = bench.max_over_ranks(elapsed, world)
    out[rank] = (mx, bench.replica_throughput(10, mx, world))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        mx, value = res[r]
        assert mx == pytest.approx(2.5)
        assert value == pytest.approx(2 * 10 / 2.5)


def test_single_rank_needs_no_group():
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.replica_throughput(10, 2.0, 1) == 5.0
