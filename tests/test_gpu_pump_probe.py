"""Pump-probe branching (Sec. 3.2: probe runs start from snapshots of a pump run and
are independent of one another): tdb_clone, tdb_step_batch, and a branched probe run
against the oracle."""
import numpy as np
import pytest

from oracle import tdb_oracle as O
from paper_1912_03174_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import __graft_entry__ as g
    g.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1912_03174_gb300 import binding
    return binding


@pytest.mark.parametrize("form", ["fp64", "fp16x6", "fp64s"])
def test_clone_continues_bit_for_bit(B, form):
    sysm = I.small_flake(33, seed=6)
    run = I.Run(dt=0.2, n_steps=0, scc=True, kick=1e-3, kT=I.SCC_KT)
    with B.Propagator(sysm, run, form) as p:
        p.setup()
        p.step(25)
        c = B.tdb_clone(p.ctx)
        try:
            p.step(40)
            B.tdb_step(c, 40)
            assert np.array_equal(B.tdb_get_rho(p.ctx), B.tdb_get_rho(c))
            assert B.tdb_get_state(p.ctx) == B.tdb_get_state(c)
            assert np.array_equal(B.tdb_dipole_history(p.ctx, 40), B.tdb_dipole_history(c, 40))
        finally:
            B.tdb_destroy(c)


def test_batch_stepping_equals_separate_stepping(B):
    # three sizes, three forms: interleaving the contexts' steps changes nothing
    cases = [(I.small_flake(10, seed=1), "fp16x6"), (I.small_flake(33, seed=2), "fp64"),
             (I.small_flake(64, seed=3), "fp64s")]
    run = I.Run(dt=0.2, n_steps=0, scc=True, kick=1e-3, kT=I.SCC_KT)
    a = [B.Propagator(s, run, f) for s, f in cases]
    b = [B.Propagator(s, run, f) for s, f in cases]
    try:
        for p in a + b:
            p.setup()
        for p in a:
            p.step(57)
        B.tdb_step_batch([p.ctx for p in b], 57)
        for pa, pb in zip(a, b):
            assert B.tdb_get_state(pa.ctx) == B.tdb_get_state(pb.ctx)
    finally:
        for p in a + b:
            p.close()


def test_branched_probe_run_matches_oracle(B):
    # pump with a laser for k steps, branch, kick 1e-3 along x, probe m steps; the oracle
    # does the same: propagate k steps, kick rho_k, Euler step, leapfrog on at t = k dt
    sysm = I.small_flake(12, seed=5)
    fld = I.Field(E0=0.01, omega=0.1, phase=0.0, t_center=40.0, fwhm=40.0, envelope=1)
    run = I.Run(dt=0.2, n_steps=0, scc=True, kick=0.0, field=fld, kT=I.SCC_KT)
    k, m, e0 = 150, 100, 1e-3
    with B.Propagator(sysm, run, "fp64") as p:
        p.setup()
        p.step(k)
        c = B.tdb_clone(p.ctx)
        try:
            B.tdb_kick(c, e0, np.array([1.0, 0.0, 0.0]))
            B.tdb_step(c, m)
            hist = B.tdb_dipole_history(c, m)
            obs = B.tdb_observables(c)
        finally:
            B.tdb_destroy(c)
    rho0, gs, S, Sinv = O.setup(sysm, run)
    tr1 = O.propagate(sysm, run, rho0, k)
    R = np.asarray(sysm.R, dtype=np.float64)
    kicked = O.kick(sysm, tr1.rho, S, Sinv, R, e0, np.array([1.0, 0.0, 0.0]))
    tr2 = O.propagate(sysm, run, kicked, m, step0=k, t0=k * run.dt)
    mu = np.vstack([hist, obs["dipole"][None, :]])
    assert np.max(np.abs(mu - tr2.dipole)) < 1e-10
    assert obs["step"] == k + m and abs(obs["t"] - (k + m) * run.dt) < 1e-10


def test_grouped_batch_equals_separate_stepping(B):
    # four FP16X6 contexts of uneven size (N = 40, 132, 256, 520), two of them one leapfrog
    # parity off the others, all kicked: a grouped batch (one launch per phase over all of
    # them) and the same contexts stepped one by one end in the same state bit for bit
    run = I.Run(dt=0.2, n_steps=0, scc=True, kick=0.0, kT=I.SCC_KT)
    a, b = [], []
    try:
        for (nat, seed), extra in zip([(10, 1), (33, 2), (64, 3), (130, 4)], [0, 1, 0, 1]):
            s = I.small_flake(nat, seed=seed)
            for lst in (a, b):
                p = B.Propagator(s, run, "fp16x6")
                p.setup()
                p.step(3 + extra)
                B.tdb_kick(p.ctx, 1e-3, np.array([1.0, 0.0, 0.0]))
                lst.append(p)
        with B.Batch([p.ctx for p in b]) as bt:
            bt.step(1)                         # the Euler step, context by context
            bt.step(40)
            tn = bt.tuning()
            with pytest.raises(B.TdbError) as e:   # a context stepped on its own
                B.tdb_step(b[0].ctx, 1)
                bt.step(1)
            assert e.value.status == 2
        a[0].step(1)
        for p in a:
            p.step(41)
        for pa, pb in zip(a, b):
            assert B.tdb_get_state(pa.ctx) == B.tdb_get_state(pb.ctx)
            assert np.array_equal(B.tdb_dipole_history(pa.ctx, 41), B.tdb_dipole_history(pb.ctx, 41))
        assert tn["x_bn"] in (128, 176, 256) and tn["schedule"] in (0, 1) and tn["x_ms"] > 0
    finally:
        for p in a + b:
            p.close()


def test_grouped_batch_rejects_mixed_forms(B):
    run = I.Run(dt=0.2, n_steps=0, scc=True, kick=1e-3, kT=I.SCC_KT)
    s = I.small_flake(10, seed=1)
    with B.Propagator(s, run, "fp16x6") as p, B.Propagator(s, run, "fp64") as q, \
            B.Propagator(s, run, "bf16x3") as r:
        for x in (p, q, r):
            x.setup()
        with pytest.raises(B.TdbError) as e:
            B.Batch([p.ctx, q.ctx])
        assert e.value.status == 10
        with pytest.raises(B.TdbError) as e:
            B.Batch([p.ctx, r.ctx])
        assert e.value.status == 1
        with pytest.raises(B.TdbError) as e:
            B.Batch([p.ctx, p.ctx])
        assert e.value.status == 1
