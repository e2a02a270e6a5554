"""The multi-GPU path is replicas only (independent trajectories, no data-path
collective): bench.py's max-over-ranks timing and whole-job value, run as two gloo
ranks on the CPU, and the reference arm's rank > 0 behaviour."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    import bench
    ms_local = 0.10 if rank == 0 else 0.25          # rank 1 is the slow replica
    ms, value = bench.replica_timing(ms_local, world, dist)
    out[rank] = (ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_timing_takes_the_slowest_rank():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world,
                           start_method="spawn", join=True)
        res = dict(out)
    assert res[0] == res[1]
    ms, value = res[0]
    assert ms == pytest.approx(0.25)
    assert value == pytest.approx(world * 1000.0 / 0.25)


def test_single_rank_timing_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_timing(0.5, 1) == (0.5, 2000.0)


def test_reference_arm_prints_nothing_on_other_ranks(capsys):
    sys.path.insert(0, ROOT)
    import bench
    from paper_1912_03174_gb300 import inputs as I
    sysm, run = I.chain_c1()

    class Args:
        steps, gpus = 2, 2
    assert bench.reference_arm(Args(), sysm, run, rank=1) is None
    assert capsys.readouterr().out == ""
