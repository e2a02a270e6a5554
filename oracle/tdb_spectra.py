"""Plain FP64 CPU oracle of the spectra post-processing (absorption and transient absorption).

TEST INFRASTRUCTURE ONLY.  Only ``tests/`` may import or run this module.  The CUDA
library and ``paper_1912_03174_gb300.spectra`` never call it and share no code with it.

What it computes, following the paper (Bonafe et al., arXiv 1912.03174):

* Sec. 2.2, eq:alpha   alpha_ij(w) = (mu_j(w) - mu_0j) / E0 for a kick along i: the Fourier
                       transform of the dipole response, here the damped one-sided sum on
                       the step grid (readings below)
* Sec. 2.2, eq:sigma   sigma(w) = 4 pi w / c Im(alpha_bar(w)), alpha_bar = Tr(alpha) / 3
* Sec. 3.2, eq:chieff / eq:alphaeff / eq:sigmaeff
                       transient absorption: the probe's response is its dipole minus the
                       pump-only dipole, Delta mu(t, tau) = mu(t) - mu_b(t), damped by
                       exp(-t / tau_damp) from the probe time on, transformed as above
* Sec. 3.2             the average over pump phases (four phase shifts of the pump pulse's
                       phase) and the Gaussian Fourier filter of the effective
                       polarizability along the delay axis
* Sec. 3.3, eq:deltaa  Delta A(tau) = A(tau) - A(t_p)

Readings where the paper leaves the discrete form open:

* The Fourier transform of a sampled signal x_n = x(n dt), n = 0..K-1, is the rectangle
  rule with the damping inside: F(w) = dt sum_n x_n exp(-n dt / tau_damp) exp(+i w n dt).
  The sign e^{+i w t} makes Im alpha >= 0 at an absorption peak for a positive kick.
* The Gaussian filter along the delay axis multiplies the discrete Fourier transform over
  the delay samples (periodic grid of n_tau points, spacing d_tau) by
  exp(-nu^2 / (2 w_f^2)), nu the angular frequency of each delay mode, and transforms back.
* A(tau) in eq:deltaa is the cross section sigma(w, tau) of eq:sigmaeff.

Every function here is plain: explicit sums written as numpy broadcasts (no FFT), in the
order the paper states the steps.
"""
from __future__ import annotations

import math

import numpy as np

C_LIGHT = 137.035999084   # speed of light, atomic units


def damped_transform(x: np.ndarray, dt: float, t_damp: float, omega: np.ndarray) -> np.ndarray:
    """F(w) = dt sum_n x_n exp(-n dt / t_damp) exp(i w n dt) for each w (x: [..., K] real).
    t_damp = inf: no damping.  Returns complex [..., n_w]."""
    x = np.asarray(x, dtype=np.float64)
    K = x.shape[-1]
    t = dt * np.arange(K)
    damp = np.exp(-t / t_damp) if math.isfinite(t_damp) else np.ones(K)
    phase = np.exp(1j * np.outer(t, np.asarray(omega, dtype=np.float64)))   # [K, n_w]
    return dt * ((x * damp) @ phase)


def polarizability(mu: np.ndarray, mu0: np.ndarray, E0: float, dt: float, t_damp: float,
                   omega: np.ndarray) -> np.ndarray:
    """eq:alpha: mu[i, n, j] = dipole component j at step n after a kick E0 along i;
    mu0[i, j] its value before the kick.  Returns alpha[i, j, w]."""
    mu = np.asarray(mu, dtype=np.float64)
    resp = mu - np.asarray(mu0, dtype=np.float64)[:, None, :]          # [i, n, j]
    return damped_transform(np.transpose(resp, (0, 2, 1)), dt, t_damp, omega) / E0


def cross_section(alpha_bar: np.ndarray, omega: np.ndarray) -> np.ndarray:
    """eq:sigma: sigma(w) = 4 pi w / c Im(alpha_bar(w))."""
    return 4.0 * math.pi * np.asarray(omega) / C_LIGHT * np.imag(alpha_bar)


def absorption(mu: np.ndarray, mu0: np.ndarray, E0: float, dt: float, t_damp: float,
               omega: np.ndarray) -> np.ndarray:
    """sigma(w) of eq:sigma from the three kicked runs of eq:alpha (alpha_bar = Tr / 3)."""
    a = polarizability(mu, mu0, E0, dt, t_damp, omega)
    alpha_bar = (a[0, 0] + a[1, 1] + a[2, 2]) / 3.0
    return cross_section(alpha_bar, omega)


def effective_polarizability(mu_probe: np.ndarray, mu_pump: np.ndarray, E0: float, dt: float,
                             t_damp: float, omega: np.ndarray) -> np.ndarray:
    """eq:chieff / eq:alphaeff for one delay: mu_probe[i, n, j] after a probe kick E0 along i
    at the delay, mu_pump[n, j] the pump-only dipole on the same steps (n = 0 at the kick).
    Delta mu = mu_probe - mu_pump, damped from the probe time on.  Returns alpha[i, j, w]."""
    d = np.asarray(mu_probe, dtype=np.float64) - np.asarray(mu_pump, dtype=np.float64)[None]
    return damped_transform(np.transpose(d, (0, 2, 1)), dt, t_damp, omega) / E0


def transient_cross_section(alpha_eff: np.ndarray, omega: np.ndarray) -> np.ndarray:
    """eq:sigmaeff: sigma(w, tau) from alpha_eff[i, j, w] of one delay (trace / 3)."""
    return cross_section((alpha_eff[0, 0] + alpha_eff[1, 1] + alpha_eff[2, 2]) / 3.0, omega)


def phase_average(values: list) -> np.ndarray:
    """The average over the pump phases of Sec. 3.2 (one entry per phase shift)."""
    return sum(np.asarray(v) for v in values) / len(values)


def gaussian_filter_delay(a: np.ndarray, d_tau: float, width: float) -> np.ndarray:
    """Gaussian Fourier filter along the delay axis (axis 0 of a[n_tau, ...]): the discrete
    Fourier transform over the n_tau delays (explicit sums), times exp(-nu^2 / (2 width^2)),
    and back."""
    a = np.asarray(a)
    m = a.shape[0]
    k = np.arange(m)
    W = np.exp(-2j * math.pi * np.outer(k, k) / m)                     # forward DFT matrix
    kk = np.where(k <= m // 2, k, k - m)                                # signed mode index
    nu = 2.0 * math.pi * kk / (m * d_tau)
    g = np.exp(-nu ** 2 / (2.0 * width ** 2))
    spec = np.tensordot(W, a, axes=(1, 0))
    spec = spec * g.reshape((m,) + (1,) * (a.ndim - 1))
    back = np.tensordot(W.conj(), spec, axes=(1, 0)) / m
    return back.real if np.isrealobj(a) else back


def delta_absorbance(A: np.ndarray, i_tp: int) -> np.ndarray:
    """eq:deltaa: Delta A(tau) = A(tau) - A(t_p) with A[n_tau, n_w] and t_p at delay index i_tp."""
    A = np.asarray(A)
    return A - A[i_tp][None]
