"""Spectra on the GPU against the oracle: the damped-transform kernel (tdb_damped_transform),
the absorption cross section of kicked runs (eq:alpha, eq:sigma) and the transient absorption
of a pump-probe scan with branched probes (eq:chieff, eq:alphaeff, eq:sigmaeff, Sec. 3.2),
each compared with oracle/tdb_spectra.py on the oracle's own propagation."""
import math

import numpy as np
import pytest

from oracle import tdb_oracle as O
from oracle import tdb_spectra as SP
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


@pytest.mark.parametrize("nsig,K,nw", [(1, 1, 1), (3, 31, 129), (13, 257, 300), (9, 1000, 64)])
@pytest.mark.parametrize("t_damp", [math.inf, 50.0])
def test_damped_transform_kernel_matches_the_oracle(B, nsig, K, nw, t_damp):
    # ragged sizes: signals not a multiple of 8, samples not a multiple of 32 or 256,
    # frequencies not a multiple of 128
    rng = np.random.default_rng(nsig * 1000 + K)
    x = rng.normal(size=(nsig, K))
    om = rng.uniform(0.0, 5.0, size=nw)
    dt = 0.2
    got = B.tdb_damped_transform(x, dt, t_damp, om)
    ref = SP.damped_transform(x, dt, t_damp, om)
    scale = dt * np.sum(np.abs(x), axis=1, keepdims=True)
    assert got.shape == ref.shape
    assert np.max(np.abs(got - ref) / scale) < 1e-13


def test_absorption_spectrum_of_the_c1_chain_matches_the_oracle(B):
    # three kicked runs (x, y, z) of the non-SCC chain, FP64 form, 1000 steps each
    import dataclasses
    from paper_1912_03174_gb300 import spectra as GS
    sysm, run = I.chain_c1()
    K = run.n_steps
    om = np.linspace(0.01, 3.0, 700)
    mu_g = np.zeros((3, K + 1, 3))
    mu_o = np.zeros((3, K + 1, 3))
    mu0_g, mu0_o = np.zeros((3, 3)), np.zeros((3, 3))
    for ax in range(3):
        d = np.zeros(3)
        d[ax] = 1.0
        r = dataclasses.replace(run, kick=0.0)
        with B.Propagator(sysm, r, "fp64") as p:
            p.setup()
            mu0_g[ax] = p.observables(charges=False)["dipole"]
            B.tdb_kick(p.ctx, run.kick, d)
            p.step(K)
            mu_g[ax] = np.vstack([B.tdb_dipole_history(p.ctx, K), p.observables()["dipole"][None]])
        rho, gs, S, Sinv = O.setup(sysm, r)
        mu0_o[ax] = O.propagate(sysm, r, rho, 0).dipole[0]
        kicked = O.kick(sysm, rho, S, Sinv, np.asarray(sysm.R, dtype=np.float64), run.kick, d)
        mu_o[ax] = O.propagate(sysm, r, kicked, K).dipole
    assert np.max(np.abs(mu_g - mu_o)) < 1e-10
    sig_g = GS.absorption(mu_g, mu0_g, run.kick, run.dt, 200.0, om)
    sig_o = SP.absorption(mu_o, mu0_o, run.kick, run.dt, 200.0, om)
    assert np.max(np.abs(sig_g - sig_o)) < 1e-6 * np.max(np.abs(sig_o))
    assert np.max(sig_g) > 0


def test_pump_probe_transient_absorption_matches_the_oracle(B):
    # Sec. 3.2 on a 12-atom SCC flake: a Gaussian laser pump, probes branched at two delays
    # (three kicked clones and an unkicked one each), 120 probe steps; the oracle runs the same
    # protocol; phase average over two pump phases, delay filter and Delta A on both sides
    from paper_1912_03174_gb300 import spectra as GS
    sysm = I.small_flake(12, seed=5)
    delays, m, e0 = [40, 90], 120, 1e-3
    om = np.linspace(0.05, 2.5, 300)
    dt, t_damp = 0.2, 30.0
    sig_g_ph, sig_o_ph = [], []
    for phase in (0.0, math.pi):
        fld = I.Field(E0=0.01, omega=0.1, phase=phase, t_center=20.0, fwhm=20.0, envelope=1)
        run = I.Run(dt=dt, n_steps=0, scc=True, kick=0.0, field=fld, kT=I.SCC_KT)
        with B.Propagator(sysm, run, "fp64") as p:
            p.setup()
            mp_g, mb_g = GS.probe_dipoles(p, delays, e0, m)
        _, sig_g = GS.transient_absorption(mp_g, mb_g, e0, dt, t_damp, om)
        rho0, gs, S, Sinv = O.setup(sysm, run)
        R = np.asarray(sysm.R, dtype=np.float64)
        mp_o = np.zeros_like(mp_g)
        mb_o = np.zeros_like(mb_g)
        at, tr = 0, None
        rho, prev = rho0, None
        for k, d_k in enumerate(delays):
            tr = O.propagate(sysm, run, rho, d_k - at, rho_prev=prev, step0=at, t0=at * dt)
            rho, prev, at = tr.rho, tr.rho_prev, d_k
            for ax in range(3):
                d = np.zeros(3)
                d[ax] = 1.0
                kicked = O.kick(sysm, rho, S, Sinv, R, e0, d)
                mp_o[k, ax] = O.propagate(sysm, run, kicked, m, step0=at, t0=at * dt).dipole
            mb_o[k] = O.propagate(sysm, run, rho, m, rho_prev=prev, step0=at, t0=at * dt).dipole
        assert np.max(np.abs(mp_g - mp_o)) < 1e-10 and np.max(np.abs(mb_g - mb_o)) < 1e-10
        al_o = np.stack([SP.effective_polarizability(mp_o[k], mb_o[k], e0, dt, t_damp, om)
                         for k in range(len(delays))])
        sig_o = np.stack([SP.transient_cross_section(al_o[k], om) for k in range(len(delays))])
        assert np.max(np.abs(sig_g - sig_o)) < 1e-6 * np.max(np.abs(sig_o))
        sig_g_ph.append(sig_g)
        sig_o_ph.append(sig_o)
    avg_g, avg_o = GS.phase_average(sig_g_ph), SP.phase_average(sig_o_ph)
    assert np.max(np.abs(avg_g - avg_o)) < 1e-6 * np.max(np.abs(avg_o))
    f_g = GS.filter_delays(avg_g, 50 * dt, 0.05)
    f_o = SP.gaussian_filter_delay(avg_o, 50 * dt, 0.05)
    assert np.max(np.abs(f_g - f_o)) < 1e-6 * np.max(np.abs(f_o))
    assert np.max(np.abs(GS.delta_absorbance(f_g, 0) - SP.delta_absorbance(f_o, 0))) < \
        1e-6 * np.max(np.abs(f_o))
