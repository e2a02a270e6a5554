"""Pins of the spectra oracle (oracle/tdb_spectra.py) against closed forms and exact
identities: eq:alpha, eq:sigma (Sec. 2.2), eq:chieff/eq:alphaeff/eq:sigmaeff, the pump-phase
average and the Gaussian delay filter (Sec. 3.2), eq:deltaa (Sec. 3.3)."""
import dataclasses
import math

import numpy as np
import pytest

from oracle import tdb_oracle as O
from oracle import tdb_spectra as SP
from paper_1912_03174_gb300 import inputs as I


def _geometric(dt, K, r, ph):
    """dt sum_{n<K} (r e^{i ph})^n in closed form."""
    z = r * np.exp(1j * ph)
    return dt * (1.0 - z ** K) / (1.0 - z)


def test_damped_transform_of_a_sampled_cosine_is_the_geometric_series():
    rng = np.random.default_rng(11)
    K, dt = 777, 0.13
    for t_damp in (35.0, 400.0, math.inf):
        th = rng.uniform(0.05, 1.5)
        a, b = rng.normal(size=2)
        n = np.arange(K)
        x = a * np.cos(th * n) + b * np.sin(th * n)
        om = np.linspace(0.0, 4.0, 301)
        r = math.exp(-dt / t_damp) if math.isfinite(t_damp) else 1.0
        ep, em = _geometric(dt, K, r, om * dt + th), _geometric(dt, K, r, om * dt - th)
        ref = a * (ep + em) / 2 + b * (ep - em) / 2j
        got = SP.damped_transform(x, dt, t_damp, om)
        assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_absorption_of_the_c1_chain_is_a_sum_of_leapfrog_modes():
    # eq:alpha / eq:sigma on the kicked non-SCC chain: alpha(w) is matched by the closed-form
    # damped transforms of modes at arcsin(w_ai dt) per step (plus the leapfrog's parasitic
    # branch at pi - arcsin(w_ai dt)) with fitted amplitudes; modes 0.1% off, or at the plain
    # w_ai dt, leave far more unexplained.  Im alpha > 0 at the strongest absorption (sign).
    s, run = I.chain_c1()
    run = dataclasses.replace(run, kick=1e-6)
    rho, gs, S, Sinv = O.setup(s, run)
    K = 20000
    tr = O.propagate(s, run, rho, K)
    mu = tr.dipole[:, 0] - tr.dipole[0, 0]
    i, j = np.triu_indices(gs.eps.size, 1)
    keep = np.abs(gs.f[i] - gs.f[j]) > 1e-12
    w = gs.eps[j[keep]] - gs.eps[i[keep]]
    dt, t_damp = run.dt, 4000.0
    om = np.linspace(0.0, 3.2, 4000)
    alpha = SP.damped_transform(mu, dt, t_damp, om) / run.kick
    r = math.exp(-dt / t_damp)

    def residual(theta):
        cols = [_geometric(dt, K + 1, r, om * dt)]
        for th in theta:
            for base in (th, math.pi - th):
                ep, em = _geometric(dt, K + 1, r, om * dt + base), _geometric(dt, K + 1, r, om * dt - base)
                cols += [(ep + em) / 2, (ep - em) / 2j]
        C = np.array(cols).T
        A = np.vstack([C.real, C.imag])
        y = np.concatenate([alpha.real, alpha.imag])
        assert A.shape[0] > 5 * A.shape[1]
        coef, *_ = np.linalg.lstsq(A, y, rcond=None)
        return np.max(np.abs(A @ coef - y)) / np.max(np.abs(y))

    r_true = residual(np.arcsin(w * dt))
    assert r_true < 1e-6, r_true
    assert residual(np.arcsin(1.001 * w * dt)) > 1e-3
    assert residual(w * dt) > 30 * r_true
    sig = SP.cross_section(alpha / 3.0, om)
    k = int(np.argmax(np.abs(sig)))
    assert sig[k] > 0 and alpha[k].imag > 0


def test_cross_section_is_the_trace_of_the_polarizability():
    # eq:sigma with alpha_bar = Tr(alpha) / 3 from three kicked runs (eq:alpha)
    rng = np.random.default_rng(3)
    K, dt, E0 = 300, 0.2, 1e-3
    mu = rng.normal(size=(3, K, 3))
    mu0 = rng.normal(size=(3, 3))
    om = np.linspace(0.1, 2.0, 50)
    a = SP.polarizability(mu, mu0, E0, dt, 50.0, om)
    for i in range(3):
        for jj in range(3):
            ref = SP.damped_transform(mu[i, :, jj] - mu0[i, jj], dt, 50.0, om) / E0
            assert np.allclose(a[i, jj], ref, rtol=0, atol=1e-13 * np.max(np.abs(ref)))
    sig = SP.absorption(mu, mu0, E0, dt, 50.0, om)
    ref = 4 * math.pi * om / 137.035999084 * np.imag(a[0, 0] + a[1, 1] + a[2, 2]) / 3
    assert np.max(np.abs(sig - ref)) < 1e-13 * np.max(np.abs(ref))


def test_phase_average_cancels_the_pump_phase_terms():
    # Sec. 3.2: the probe-minus-pump signal carries terms in the pump phase phi (the relative
    # phase of pump and probe); averaging four phase shifts 0, pi/2, pi, 3 pi/2 removes every
    # term of order 1, 2 and 3 in e^{i phi} exactly, through the whole transform chain
    rng = np.random.default_rng(5)
    K, dt = 500, 0.2
    t = dt * np.arange(K)
    a = rng.normal(size=(3, K, 3)) * 1e-3
    b = rng.normal(size=(3, K, 3)) * 1e-3
    Om = 0.37
    phases = [0.0, math.pi / 2, math.pi, 3 * math.pi / 2]
    pump = np.zeros((K, 3))
    om = np.linspace(0.1, 2.0, 64)
    alphas, sigmas = [], []
    for ph in phases:
        probe = a + b * (np.cos(Om * t + ph) + 0.5 * np.cos(2 * Om * t + 2 * ph)
                         + 0.25 * np.sin(3 * Om * t + 3 * ph))[None, :, None]
        al = SP.effective_polarizability(probe, pump, 1e-3, dt, 30.0, om)
        alphas.append(al)
        sigmas.append(SP.transient_cross_section(al, om))
    ref = SP.effective_polarizability(a, pump, 1e-3, dt, 30.0, om)
    avg = SP.phase_average(alphas)
    assert np.max(np.abs(avg - ref)) < 1e-12 * np.max(np.abs(ref))
    assert np.max(np.abs(SP.phase_average(sigmas) - SP.transient_cross_section(ref, om))) < \
        1e-12 * np.max(np.abs(SP.transient_cross_section(ref, om)))
    # a single phase keeps the oscillating term
    assert np.max(np.abs(alphas[0] - ref)) > 1e-2 * np.max(np.abs(ref))


def test_no_probe_kick_gives_no_transient_response():
    # eq:chieff: the reference subtracted is the pump-only dipole
    rng = np.random.default_rng(2)
    pump = rng.normal(size=(200, 3))
    al = SP.effective_polarizability(np.broadcast_to(pump, (3, 200, 3)), pump, 1e-3, 0.2, 40.0,
                                     np.linspace(0.1, 1.0, 10))
    assert np.all(al == 0)


def test_gaussian_delay_filter_attenuates_each_delay_mode_by_the_gaussian():
    m, d_tau, width = 96, 0.7, 0.9
    tau = d_tau * np.arange(m)
    rng = np.random.default_rng(9)
    c = rng.normal(size=(4, 5))
    ks = [0, 1, 7, 23]
    a = sum(c[q][None, :] * np.cos(2 * math.pi * k * tau / (m * d_tau))[:, None]
            for q, k in enumerate(ks))
    ref = sum(c[q][None, :] * math.exp(-(2 * math.pi * k / (m * d_tau)) ** 2 / (2 * width ** 2))
              * np.cos(2 * math.pi * k * tau / (m * d_tau))[:, None] for q, k in enumerate(ks))
    got = SP.gaussian_filter_delay(a, d_tau, width)
    assert np.max(np.abs(got - ref)) < 1e-12
    # a constant along the delay axis passes unchanged; a complex input stays complex
    assert np.allclose(SP.gaussian_filter_delay(np.ones((m, 3)) * 2.5, d_tau, width), 2.5,
                       rtol=0, atol=1e-13)
    z = a + 1j * a
    assert np.max(np.abs(SP.gaussian_filter_delay(z, d_tau, width) - (ref + 1j * ref))) < 1e-12


def test_delta_absorbance_vanishes_at_the_end_of_the_pump():
    rng = np.random.default_rng(4)
    A = rng.normal(size=(40, 12))
    dA = SP.delta_absorbance(A, 7)
    assert np.all(dA[7] == 0)
    assert np.allclose(SP.delta_absorbance(A + rng.normal(size=(1, 12)), 7), dA, rtol=0, atol=1e-14)
