"""The multi-GPU pump-probe scan as two gloo ranks on the CPU, with a stand-in binding:
every probe runs on exactly one rank, the shares follow the longest-processing-time
partition, and the whole-job rate is all probe steps over the slowest rank's time."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TESTS = os.path.dirname(os.path.abspath(__file__))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class _NoCuda:
    class cuda:
        @staticmethod
        def synchronize():
            pass


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, TESTS)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    import bench
    from paper_1912_03174_gb300 import scan
    from test_scan_host import _FakeB
    fake = _FakeB()
    seen = []
    real = scan.run_shard

    def spy(B, systems, run, which, tau, mine, post_steps, form="fp16x6", sync=None):
        seen.extend(mine)
        return real(B, systems, run, which, tau, mine, post_steps, form, sync)

    scan.run_shard = spy
    r = bench.c4_sharded(fake, _NoCuda, dist, rank, world, n_traj=12, post_steps=5)
    u, t, rate = bench.shard_throughput(10.0 * (rank + 1), 0.5 + rank, dist)
    out[rank] = (sorted(seen), r["probes"], r["probes_this_rank"], (u, t, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_scan_shares_every_probe_once_over_two_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world,
                           start_method="spawn", join=True)
        res = dict(out)
    sys.path.insert(0, ROOT)
    from paper_1912_03174_gb300 import inputs as I, scan
    systems, run, which, tau = I.pump_probe_c4(n_traj=12)
    parts = scan.lpt_partition(scan.probe_costs(systems, which, 5), world)
    assert res[0][0] == parts[0] and res[1][0] == parts[1]
    assert sorted(res[0][0] + res[1][0]) == list(range(12))
    assert res[0][1] == res[1][1] == 12
    assert res[0][2] + res[1][2] == 12
    u, t, rate = res[0][3]
    assert res[0][3] == res[1][3]
    assert u == 30.0 and t == 1.5 and rate == pytest.approx(20.0)


def test_shard_throughput_on_one_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.shard_throughput(100.0, 2.0) == (100.0, 2.0, 50.0)
    assert bench.shard_throughput(0.0, 0.0)[2] == 0.0
