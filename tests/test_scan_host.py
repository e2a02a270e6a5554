"""Host logic of the multi-GPU pump-probe scan (no GPU): the longest-processing-time
partition of the probe runs and one rank's branching and stepping of its share, with a
stand-in binding."""
import itertools

import numpy as np
import pytest

from paper_1912_03174_gb300 import inputs as I
from paper_1912_03174_gb300 import scan


def test_lpt_partition_worked_example():
    parts = scan.lpt_partition([5, 4, 3, 3, 2, 2, 1], 2)
    assert parts == [[0, 3, 5], [1, 2, 4, 6]]


@pytest.mark.parametrize("m", [2, 3])
def test_lpt_partition_within_grahams_bound_of_the_optimum(m):
    rng = np.random.default_rng(m)
    for _ in range(20):
        costs = rng.integers(1, 50, size=7).astype(float)
        parts = scan.lpt_partition(costs, m)
        assert sorted(i for p in parts for i in p) == list(range(7))
        span = max(costs[p].sum() for p in parts)
        best = min(max(costs[[i for i in range(7) if a[i] == q]].sum() for q in range(m))
                   for a in itertools.product(range(m), repeat=7))
        assert span <= (4.0 / 3.0 - 1.0 / (3 * m)) * best + 1e-9


def test_lpt_partition_more_parts_than_jobs():
    assert scan.lpt_partition([3.0, 1.0], 4) == [[0], [1], [], []]
    with pytest.raises(ValueError):
        scan.lpt_partition([1.0], 0)


class _Sys:
    def __init__(self, n_orb):
        self.n_orb = n_orb


def test_probe_costs_are_n_cubed_times_steps():
    c = scan.probe_costs([_Sys(128), _Sys(1024)], [1, 0, 1], 10)
    np.testing.assert_allclose(c, [10 * 1024.0 ** 3, 10 * 128.0 ** 3, 10 * 1024.0 ** 3])


class _Ctx:
    def __init__(self, sysm, t=0):
        self.sysm, self.t, self.kicked = sysm, t, False


class _Prop:
    def __init__(self, fake, sysm, run, form):
        self.ctx = _Ctx(sysm)
        fake.pumps.append((sysm, run.kick, form))

    def setup(self):
        pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        pass


class _FakeB:
    def __init__(self):
        self.pumps, self.clones, self.destroyed, self.batches = [], [], 0, []

    def Propagator(self, sysm, run, form):
        return _Prop(self, sysm, run, form)

    def tdb_step(self, ctx, n):
        assert n >= 0
        ctx.t += n

    def tdb_clone(self, ctx):
        c = _Ctx(ctx.sysm, ctx.t)
        self.clones.append(c)
        return c

    def tdb_kick(self, ctx, strength, direction):
        ctx.kicked = True

    def tdb_step_batch(self, ctxs, n):
        assert all(c.kicked for c in ctxs)
        self.batches.append((len(ctxs), n))
        for c in ctxs:
            c.t += n

    def tdb_dipole_history(self, ctx, cap):
        return np.full((cap, 3), float(ctx.t))

    def tdb_destroy(self, ctx):
        self.destroyed += 1


def test_run_shard_branches_each_probe_at_its_delay():
    run = I.Run(dt=0.5, n_steps=0, scc=True, kick=1e-3)
    systems = ["small", "big"]
    which = np.array([0, 1, 0, 1, 1])
    tau = np.array([2.0, 10.0, 1.0, 4.0, 3.0])           # steps 4, 20, 2, 8, 6
    fake = _FakeB()
    calls = []
    n, pump_steps, t, hist = scan.run_shard(fake, systems, run, which, tau, [0, 1, 2, 3], 7,
                                            sync=lambda: calls.append(1))
    assert n == 4 and pump_steps == 4 + 20 and len(calls) == 2 and t >= 0
    assert [p[1] for p in fake.pumps] == [0.0, 0.0]                  # pump runs not kicked
    assert fake.batches == [(4, 2), (4, 7)] and fake.destroyed == 4
    # probe i was cloned at its own delay, then took 2 + 7 steps
    for i, steps in {0: 4, 1: 20, 2: 2, 3: 8}.items():
        assert hist[i][0, 0] == steps + 9
    assert 4 not in hist


def test_run_shard_with_no_probes():
    fake = _FakeB()
    run = I.Run(dt=0.5, n_steps=0, scc=True, kick=1e-3)
    calls = []
    assert scan.run_shard(fake, ["a"], run, np.array([0]), np.array([1.0]), [], 5,
                          sync=lambda: calls.append(1)) == (0, 0, 0.0, {})
    assert len(calls) == 2          # a rank without probes still meets the others' barriers
