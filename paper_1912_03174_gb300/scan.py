"""Pump-probe scans over several GPUs (Sec. 3.2: the probe runs of a scan are
independent of one another): the probes are shared out among the ranks by greedy
longest-processing-time on their cost N^3 x steps, with no data-path collective.  Each
rank branches its own probes from its own pump runs (`tdb_clone` at the probe's
delay, then the probe kick) and advances them together (`tdb_step_batch`); the host
gathers what each rank wrote.

Host orchestration only: every step runs in the library.
"""
from __future__ import annotations

import heapq
import time

import numpy as np


def lpt_partition(costs, n_parts: int):
    """Greedy longest-processing-time: jobs by decreasing cost (ties: lower index
    first), each to the part with the least load so far (ties: lower part).  Returns
    n_parts sorted index lists."""
    if n_parts < 1:
        raise ValueError("n_parts must be >= 1")
    costs = np.asarray(costs, dtype=np.float64)
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, p) for p in range(n_parts)]
    parts = [[] for _ in range(n_parts)]
    for i in order:
        load, p = heapq.heappop(heap)
        parts[p].append(i)
        heapq.heappush(heap, (load + costs[i], p))
    return [sorted(p) for p in parts]


def probe_costs(systems, which, post_steps: int):
    """Cost of each probe run: N^3 of its system times its timed steps."""
    n_orb = np.array([s.n_orb for s in systems], dtype=np.float64)
    return n_orb[np.asarray(which)] ** 3 * post_steps


def run_shard(B, systems, run, which, tau, mine, post_steps: int, form="fp16x6", sync=None):
    """Pump runs, branching and the timed batched stepping of the probes `mine` (indices
    into which / tau).  Returns (probes run, pump steps, seconds of the timed stepping,
    dipole histories of the probes' timed steps by probe index).  sync() is called
    before the timer starts and after it stops (a device-wide synchronisation, and a
    barrier across ranks), also by a rank with no probes."""
    import dataclasses
    pump_run = dataclasses.replace(run, kick=0.0)
    mine = list(mine)
    probes, index = [], []
    pump_steps = 0
    try:
        for s_idx, sysm in enumerate(systems):
            idx = [i for i in mine if which[i] == s_idx]
            if not idx:
                continue
            steps = {i: int(np.rint(tau[i] / run.dt)) for i in idx}
            with B.Propagator(sysm, pump_run, form) as p:
                p.setup()
                at = 0
                for i in sorted(idx, key=lambda j: (steps[j], j)):
                    B.tdb_step(p.ctx, steps[i] - at)
                    at = steps[i]
                    c = B.tdb_clone(p.ctx)
                    B.tdb_kick(c, run.kick, run.kick_dir)
                    probes.append(c)
                    index.append(i)
                pump_steps += at
        if not probes:
            if sync:                                  # the other ranks wait at both points
                sync()
                sync()
            return 0, pump_steps, 0.0, {}
        B.tdb_step_batch(probes, 2)                   # Euler step and graph capture
        if sync:
            sync()
        t0 = time.perf_counter()
        B.tdb_step_batch(probes, post_steps)
        if sync:
            sync()
        t = time.perf_counter() - t0
        hist = {i: B.tdb_dipole_history(c, post_steps) for i, c in zip(index, probes)}
        return len(probes), pump_steps, t, hist
    finally:
        for c in probes:
            B.tdb_destroy(c)
