"""Absorption and transient-absorption spectra from the propagator's dipole signals.

* Sec. 2.2, eq:alpha / eq:sigma: after a delta kick E0 along each axis, alpha_ij(w) is the
  damped transform of mu_j(t) - mu_0j divided by E0, and sigma(w) = 4 pi w / c Im Tr(alpha)/3.
* Sec. 3.2, eq:chieff / eq:alphaeff / eq:sigmaeff: a probe kicked at delay tau on a pumped
  run responds by mu(t) - mu_b(t), the pump-only dipole on the same steps; damped by
  exp(-t / tau_damp) from the probe time on and transformed like eq:alpha.  Probes branch
  from the pump run (tdb_clone), so one pump run serves every delay.
* Sec. 3.2: the average over pump phases and a Gaussian filter of the effective
  polarizability along the delay axis (in its Fourier space).
* Sec. 3.3, eq:deltaa: Delta A(tau) = A(tau) - A(t_p).

The transforms (the O(K n_w) part) run in the library's FP64 kernel
(tdb_damped_transform); what remains are O(n_tau n_w) array operations on their results.
The propagation is the library's (binding.Propagator / tdb_clone / tdb_step_batch).
"""
from __future__ import annotations

import math
from typing import Sequence

import numpy as np

from . import binding as B

SPEED_OF_LIGHT_AU = 137.035999084


def transform(x, dt: float, t_damp: float, omega) -> np.ndarray:
    """dt sum_n x[..., n] exp(-n dt / t_damp) exp(i w n dt) (GPU, FP64)."""
    return B.tdb_damped_transform(x, dt, t_damp, omega)


def sigma_from_alpha_bar(alpha_bar: np.ndarray, omega) -> np.ndarray:
    """eq:sigma: 4 pi w / c Im(alpha_bar)."""
    return 4.0 * math.pi * np.asarray(omega, dtype=np.float64) / SPEED_OF_LIGHT_AU * alpha_bar.imag


def polarizability(mu, mu0, E0: float, dt: float, t_damp: float, omega) -> np.ndarray:
    """eq:alpha from kicked runs: mu[i, n, j] (kick along axis i, component j), mu0[i, j] the
    dipole before the kick.  Returns alpha[i, j, w]."""
    resp = np.asarray(mu, dtype=np.float64) - np.asarray(mu0, dtype=np.float64)[:, None, :]
    return transform(np.ascontiguousarray(resp.transpose(0, 2, 1)), dt, t_damp, omega) / E0


def absorption(mu, mu0, E0: float, dt: float, t_damp: float, omega) -> np.ndarray:
    """sigma(w) of eq:sigma from the three kicked runs."""
    a = polarizability(mu, mu0, E0, dt, t_damp, omega)
    return sigma_from_alpha_bar(np.trace(a, axis1=0, axis2=1) / 3.0, omega)


def effective_polarizability(mu_probe, mu_pump, E0: float, dt: float, t_damp: float,
                             omega) -> np.ndarray:
    """eq:alphaeff for one delay: mu_probe[i, n, j] after a probe kick E0 along i (n = 0 at
    the kick), mu_pump[n, j] the pump-only dipole on the same steps.  Returns alpha[i, j, w]."""
    d = np.asarray(mu_probe, dtype=np.float64) - np.asarray(mu_pump, dtype=np.float64)[None]
    return transform(np.ascontiguousarray(d.transpose(0, 2, 1)), dt, t_damp, omega) / E0


def transient_sigma(alpha_eff: np.ndarray, omega) -> np.ndarray:
    """eq:sigmaeff from alpha_eff[..., i, j, w] (one or many delays)."""
    return sigma_from_alpha_bar(np.trace(alpha_eff, axis1=-3, axis2=-2) / 3.0, omega)


def phase_average(per_phase: Sequence[np.ndarray]) -> np.ndarray:
    """Mean over the pump phases (Sec. 3.2)."""
    return np.mean(np.stack([np.asarray(v) for v in per_phase]), axis=0)


def filter_delays(a: np.ndarray, d_tau: float, width: float) -> np.ndarray:
    """Gaussian filter along the delay axis (axis 0): FFT over the delays, times
    exp(-nu^2 / (2 width^2)) at each delay mode's angular frequency nu, inverse FFT."""
    a = np.asarray(a)
    m = a.shape[0]
    nu = 2.0 * math.pi * np.fft.fftfreq(m, d=d_tau)
    g = np.exp(-nu ** 2 / (2.0 * width ** 2)).reshape((m,) + (1,) * (a.ndim - 1))
    out = np.fft.ifft(np.fft.fft(a, axis=0) * g, axis=0)
    return out if np.iscomplexobj(a) else out.real


def delta_absorbance(A: np.ndarray, i_tp: int) -> np.ndarray:
    """eq:deltaa: A(tau) - A(t_p), A[n_tau, n_w]."""
    A = np.asarray(A)
    return A - A[i_tp:i_tp + 1]


def probe_dipoles(pump: "B.Propagator", delay_steps: Sequence[int], kick: float, n_steps: int,
                  axes=(0, 1, 2)):
    """Sec. 3.2 protocol on the GPU for one pump run: the pump is stepped to each delay (in
    increasing order); there three probes branch from it (tdb_clone) and are kicked along the
    axes, and a fourth clone continues unkicked as the pump-only reference; the four advance
    n_steps together (tdb_step_batch).  Returns mu_probe[tau, i, n, j] and mu_pump[tau, n, j]
    for n = 0..n_steps (n = 0 at the kick), the pump left at the last delay."""
    order = np.argsort(delay_steps)
    at = 0
    nt = len(delay_steps)
    mu_probe = np.zeros((nt, len(axes), n_steps + 1, 3))
    mu_pump = np.zeros((nt, n_steps + 1, 3))
    for k in order:
        B.tdb_step(pump.ctx, int(delay_steps[k]) - at)
        at = int(delay_steps[k])
        clones = [B.tdb_clone(pump.ctx) for _ in range(len(axes) + 1)]
        try:
            for c, ax in zip(clones, axes):
                d = np.zeros(3)
                d[ax] = 1.0
                B.tdb_kick(c, kick, d)
            B.tdb_step_batch(clones, n_steps)
            for q, c in enumerate(clones):
                h = B.tdb_dipole_history(c, n_steps)
                mu = np.vstack([h, B.tdb_observables(c, charges=False)["dipole"][None]])
                if q < len(axes):
                    mu_probe[k, q] = mu
                else:
                    mu_pump[k] = mu
        finally:
            for c in clones:
                B.tdb_destroy(c)
    return mu_probe, mu_pump


def transient_absorption(mu_probe, mu_pump, kick: float, dt: float, t_damp: float, omega):
    """sigma(w, tau) of eq:sigmaeff for every delay: mu_probe[tau, i, n, j], mu_pump[tau, n, j].
    Returns (alpha_eff[tau, i, j, w], sigma[tau, w])."""
    alpha = np.stack([effective_polarizability(mu_probe[t], mu_pump[t], kick, dt, t_damp, omega)
                      for t in range(mu_probe.shape[0])])
    return alpha, transient_sigma(alpha, omega)
