"""Plain FP64 CPU oracle of real-time (Ehrenfest) TD-DFTB propagation.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run
this module.  The CUDA library never calls it and shares no code with it; the
only thing both sides share is the seeded input generator
(``paper_1912_03174_gb300.inputs``), which holds none of the method's
arithmetic.

Everything here follows the paper (Bonafe et al., real-time Ehrenfest
TD-DFTB, arXiv 1912.03174) in its own order and notation, in float64/complex128,
with numpy/scipy primitives (matrix products, Cholesky, generalised symmetric
eigensolver) as the only library steps:

* Sec. 2.1, eq:hscc / eq:hsccvext   SCC Hamiltonian with external potential
* Sec. 2.1, eq:coul                  gamma_AB (its short-range form is a reading:
                                      the Elstner closed form, see ``gamma_matrix``)
* Sec. 2.1, eq:qmulik                Mulliken populations (real part, a reading)
* Sec. 2.1, eq:eomrho                density-matrix equation of motion
* Sec. 2.1, eq:nac, eq:onsite        non-adiabatic coupling matrix D
* Sec. 2.1, eq:forces                Ehrenfest forces (velocity terms dropped,
                                      S-derivative terms in energy-weighted form)
* Sec. 2.2, eq:rhokick               delta kick in a non-orthogonal basis
* Sec. 2.3, eq:leapfrog              leapfrog with an Euler first step
* Sec. 2.3                           velocity Verlet for the nuclei
* Sec. 3.1, eq:pumpf                 laser pulse
* (learned form)                     closed-form leapfrog windows with a frozen
                                      Hamiltonian; the per-atom shift network

Parity pins: every function here is pinned by a test in
``tests/test_oracle_pins.py`` against something other than itself (closed
forms, quadrature, finite differences, special cases, invariants).  The
absolute physics of the synthetic model is ours by construction and is the
one thing that is "parity unpinned" (there is no published value for it).
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Optional

import numpy as np
import scipy.linalg as sla

AMU = 1822.888486     # electron masses per atomic mass unit
GAMMA_EQUAL_REL = 3e-4  # relative exponent gap below which gamma uses its equal-exponent form


# ---------------------------------------------------------------------------
# Synthetic two-centre model: stands in for the Slater-Koster tables of
# Sec. 2.1 (H0 and S "parameterized as a function of the inter-atomic
# distance ... in a minimal basis of valence orbitals").
# ---------------------------------------------------------------------------

def radial_integrals(sysm, r):
    """Hopping and overlap integrals (ss-sigma, sp-sigma, pp-sigma, pp-pi) at distance r.

    Returns (V, dV/dr, S, dS/dr), each of shape r.shape + (4,).
    V_k = eta_k t0 exp(-r/lam_H),  S_k = -eta_k s0 exp(-r/lam_S).
    """
    r = np.asarray(r, dtype=np.float64)[..., None]
    eta = np.asarray(sysm.eta, dtype=np.float64)
    V = eta * sysm.t0 * np.exp(-r / sysm.lam_H)
    dV = -V / sysm.lam_H
    S = -eta * sysm.s0 * np.exp(-r / sysm.lam_S)
    dS = -S / sysm.lam_S
    return V, dV, S, dS


def sk_block(c, k, n_orb):
    """Two-centre block <phi_mu(A)|O|phi_nu(B)> for direction cosines c (A->B).

    Slater-Koster s/p table: ss = K_ss; s-alpha = c_alpha K_sp;
    alpha-s = -c_alpha K_sp; alpha-beta = c_alpha c_beta (K_ppsig - K_pppi)
    + delta_alpha_beta K_pppi.  Shapes: c (..., 3), k (..., 4) -> (..., n, n).
    """
    out = np.zeros(c.shape[:-1] + (n_orb, n_orb))
    out[..., 0, 0] = k[..., 0]
    if n_orb == 4:
        out[..., 0, 1:] = c * k[..., 1:2]
        out[..., 1:, 0] = -c * k[..., 1:2]
        cc = c[..., :, None] * c[..., None, :]
        eye = np.eye(3)
        out[..., 1:, 1:] = cc * (k[..., 2] - k[..., 3])[..., None, None] + eye * k[..., 3][..., None, None]
    return out


def sk_block_grad(c, r, k, dk, n_orb):
    """d(block)/d(R_B) (= d/d(R_B - R_A)) of ``sk_block``: shape (..., 3, n, n)."""
    # dr/dd_g = c_g ; dc_a/dd_g = (delta_ag - c_a c_g)/r
    eye = np.eye(3)
    dc = (eye - c[..., :, None] * c[..., None, :]) / r[..., None, None]   # [..., a, g]
    out = np.zeros(c.shape[:-1] + (3, n_orb, n_orb))
    cg = c
    out[..., :, 0, 0] = dk[..., 0:1] * cg
    if n_orb == 4:
        # s-alpha: dc_a/dd_g K_sp + c_a dK_sp c_g
        sa = np.swapaxes(dc, -1, -2) * k[..., 1][..., None, None] \
            + cg[..., :, None] * c[..., None, :] * dk[..., 1][..., None, None]      # [..., g, a]
        out[..., :, 0, 1:] = sa
        out[..., :, 1:, 0] = -sa
        dsp = k[..., 2] - k[..., 3]
        ddsp = dk[..., 2] - dk[..., 3]
        dcT = np.swapaxes(dc, -1, -2)                                           # [..., g, a]
        term1 = (dcT[..., :, :, None] * c[..., None, None, :]
                 + c[..., None, :, None] * dcT[..., :, None, :]) * dsp[..., None, None, None]
        term2 = (c[..., :, None] * c[..., None, :])[..., None, :, :] * cg[..., :, None, None] \
            * ddsp[..., None, None, None]
        term3 = eye[None, :, :] * cg[..., :, None, None] * dk[..., 3][..., None, None, None]
        out[..., :, 1:, 1:] = term1 + term2 + term3
    return out


def pair_list(n_atoms):
    """All unordered atom pairs A < B."""
    iA, iB = np.triu_indices(n_atoms, k=1)
    return iA, iB


def model_matrices(sysm, R):
    """S and H0 (N x N, atom-major orbital order) for geometry R.

    On-site blocks: S_AA = 1, H0_AA = diag(eps_s, eps_p, eps_p, eps_p) of A's species.
    Off-site blocks: the two-centre table above (block_BA = block_AB^T).
    Dense, no distance cut-off.
    """
    n = sysm.orbs_per_atom
    nat = R.shape[0]
    S4 = np.zeros((nat, n, nat, n))
    H4 = np.zeros((nat, n, nat, n))
    for A in range(nat):
        sp = sysm.species[A]
        onsite = [sysm.eps_s[sp]] + [sysm.eps_p[sp]] * (n - 1)
        H4[A, :, A, :] = np.diag(onsite)
        S4[A, :, A, :] = np.eye(n)
    iA, iB = pair_list(nat)
    if iA.size:
        d = R[iB] - R[iA]
        r = np.linalg.norm(d, axis=1)
        c = d / r[:, None]
        V, _, Sk, _ = radial_integrals(sysm, r)
        hb = sk_block(c, V, n)
        sb = sk_block(c, Sk, n)
        H4[iA, :, iB, :] = hb
        H4[iB, :, iA, :] = np.swapaxes(hb, 1, 2)
        S4[iA, :, iB, :] = sb
        S4[iB, :, iA, :] = np.swapaxes(sb, 1, 2)
    N = n * nat
    return S4.reshape(N, N), H4.reshape(N, N)


def model_pair_gradients(sysm, R):
    """Per pair (A<B): d(H0 block)/dR_B and d(S block)/dR_B, shape (npairs, 3, n, n).

    d/dR_A of the same block is the negative (the blocks depend on R_B - R_A only).
    """
    n = sysm.orbs_per_atom
    iA, iB = pair_list(R.shape[0])
    d = R[iB] - R[iA]
    r = np.linalg.norm(d, axis=1)
    c = d / r[:, None]
    V, dV, Sk, dSk = radial_integrals(sysm, r)
    return iA, iB, sk_block_grad(c, r, V, dV, n), sk_block_grad(c, r, Sk, dSk, n)


# ---------------------------------------------------------------------------
# gamma (eq:coul).  The paper defers the short-range function zeta(R) to
# first-principles fits; the reading taken here is the standard DFTB form:
# the Coulomb interaction of two normalised exponential densities
# n(r) = tau^3/(8 pi) exp(-tau r) with tau = 16 U / 5, so that gamma_AA = U_A.
# ---------------------------------------------------------------------------

def _short_range(ta, tb, R):
    """zeta(R) for exponents ta, tb (closed form of the Coulomb integral of two
    exponential densities minus 1/R).  Arrays broadcast.  The equal-exponent
    form is used where |ta - tb| < 3e-4 max(ta, tb): below that the
    unequal form loses digits to cancellation (both forms agree to ~1e-8 at
    the switch, checked in high precision)."""
    ta, tb, R = np.broadcast_arrays(np.asarray(ta, float), np.asarray(tb, float), np.asarray(R, float))
    same = np.abs(ta - tb) < GAMMA_EQUAL_REL * np.maximum(ta, tb)
    t = 0.5 * (ta + tb)
    eq = np.exp(-t * R) * (1.0 / R + 11.0 * t / 16.0 + 3.0 * t * t * R / 16.0 + t ** 3 * R * R / 48.0)
    a = np.where(same, 1.0, ta)
    b = np.where(same, 2.0, tb)

    def part(a, b):
        return np.exp(-a * R) * (b ** 4 * a / (2.0 * (a * a - b * b) ** 2)
                                 - (b ** 6 - 3.0 * a * a * b ** 4) / ((a * a - b * b) ** 3 * R))
    return np.where(same, eq, part(a, b) + part(b, a))


def _short_range_dR(ta, tb, R):
    """d zeta / dR of ``_short_range``."""
    ta, tb, R = np.broadcast_arrays(np.asarray(ta, float), np.asarray(tb, float), np.asarray(R, float))
    same = np.abs(ta - tb) < GAMMA_EQUAL_REL * np.maximum(ta, tb)
    t = 0.5 * (ta + tb)
    e = np.exp(-t * R)
    poly = 1.0 / R + 11.0 * t / 16.0 + 3.0 * t * t * R / 16.0 + t ** 3 * R * R / 48.0
    dpoly = -1.0 / (R * R) + 3.0 * t * t / 16.0 + t ** 3 * R / 24.0
    eq = e * (dpoly - t * poly)
    a = np.where(same, 1.0, ta)
    b = np.where(same, 2.0, tb)

    def part(a, b):
        ea = np.exp(-a * R)
        c1 = b ** 4 * a / (2.0 * (a * a - b * b) ** 2)
        c2 = (b ** 6 - 3.0 * a * a * b ** 4) / (a * a - b * b) ** 3
        return ea * (-a * (c1 - c2 / R) + c2 / (R * R))
    return np.where(same, eq, part(a, b) + part(b, a))


def gamma_pair(UA, UB, R):
    """gamma_AB of eq:coul off-site: 1/R - zeta(R), with tau = 16 U / 5."""
    return 1.0 / np.asarray(R, float) - _short_range(3.2 * np.asarray(UA), 3.2 * np.asarray(UB), R)


def gamma_pair_dR(UA, UB, R):
    R = np.asarray(R, float)
    return -1.0 / (R * R) - _short_range_dR(3.2 * np.asarray(UA), 3.2 * np.asarray(UB), R)


def gamma_matrix(sysm, R):
    """gamma (n_atoms x n_atoms): U_A on the diagonal, gamma_pair off it."""
    nat = R.shape[0]
    U = sysm.hubbard_U[sysm.species]
    G = np.diag(U.astype(np.float64))
    iA, iB = pair_list(nat)
    if iA.size:
        r = np.linalg.norm(R[iB] - R[iA], axis=1)
        g = gamma_pair(U[iA], U[iB], r)
        G[iA, iB] = g
        G[iB, iA] = g
    return G


# ---------------------------------------------------------------------------
# Mulliken populations (eq:qmulik), SCC Hamiltonian (eq:hscc, eq:hsccvext)
# ---------------------------------------------------------------------------

def reference_populations(sysm):
    """q0_A: neutral valence population (same valence count for every species)."""
    return np.full(sysm.n_atoms, sysm.n_electrons / sysm.n_atoms)


def mulliken(sysm, rho, S):
    """q_A = Tr_A{rho S} (eq:qmulik); the real part is taken (a reading: the
    imaginary part vanishes for Hermitian rho summed over all atoms)."""
    n = sysm.orbs_per_atom
    diag = np.real(np.diag(rho @ S))
    return diag.reshape(-1, n).sum(axis=1)


def field_at(fld, t):
    """E(t) = E0 sin(omega t + phi) f(t) e (eq:pumpf); None -> zero field.

    Envelope readings: 0 none, 1 Gaussian on the field with the stated FWHM
    centred at t_center, 2 sin^2(pi t / fwhm) on [0, fwhm] and zero outside.
    """
    if fld is None:
        return np.zeros(3)
    if fld.envelope == 0:
        f = 1.0
    elif fld.envelope == 1:
        f = math.exp(-((t - fld.t_center) ** 2) * 4.0 * math.log(2.0) / fld.fwhm ** 2)
    else:
        f = math.sin(math.pi * t / fld.fwhm) ** 2 if 0.0 <= t <= fld.fwhm else 0.0
    d = np.asarray(fld.dir, dtype=np.float64)
    return fld.E0 * math.sin(fld.omega * t + fld.phase) * f * d


def atom_potential(gamma, dq, R, E, scc):
    """v_A = sum_C gamma_AC dq_C (if SCC) + V^ext_A, with V^ext_A = R_A . E(t)
    (potential energy of an electron in the field; a reading of Sec. 2.1)."""
    v = R @ E
    if scc:
        v = v + gamma @ dq
    return v


def scc_hamiltonian(sysm, H0, S, v_atom):
    """H_mu_nu = H0_mu_nu + 1/2 S_mu_nu (v_A + v_B), mu in A, nu in B."""
    v = np.repeat(v_atom, sysm.orbs_per_atom)
    return H0 + 0.5 * S * (v[:, None] + v[None, :])


# ---------------------------------------------------------------------------
# Ground state (Sec. 2.1: "consecutive cycles of diagonalization and
# Hamiltonian building until self-consistency")
# ---------------------------------------------------------------------------

def aufbau(eps, n_electrons, degen_tol=1e-8):
    """Occupations f in {0, 2} (kT = 0); a degenerate shell at the Fermi level
    shares its electrons equally (keeps rho_0 unique and stationary)."""
    f = np.zeros_like(eps)
    order = np.argsort(eps)
    k = int(math.ceil(n_electrons / 2.0))
    e_f = eps[order[k - 1]]
    below = eps < e_f - degen_tol
    shell = np.abs(eps - e_f) <= degen_tol
    f[below] = 2.0
    f[shell] = (n_electrons - 2.0 * below.sum()) / shell.sum()
    return f


def fermi_occupations(eps, n_electrons, kT):
    """Spin-degenerate Fermi-Dirac occupations f_i = 2 / (1 + exp((e_i - mu)/kT)),
    mu found by bisection so that sum f = N_e.  kT = 0 falls back to aufbau.
    (The paper leaves the ground-state occupations to DFTB+; an electronic
    temperature is the reading taken for small-gap synthetic systems.)"""
    if kT <= 0.0:
        return aufbau(eps, n_electrons)
    lo, hi = eps.min() - 50.0 * kT, eps.max() + 50.0 * kT

    def occ(mu):
        x = np.clip((eps - mu) / kT, -700.0, 700.0)
        return 2.0 / (1.0 + np.exp(x))
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if occ(mid).sum() > n_electrons:
            hi = mid
        else:
            lo = mid
    return occ(0.5 * (lo + hi))


def electronic_entropy(f):
    """S = -2 sum [p ln p + (1 - p) ln(1 - p)], p = f/2 (units of k_B)."""
    p = np.clip(f / 2.0, 1e-300, 1.0)
    q = np.clip(1.0 - f / 2.0, 1e-300, 1.0)
    return float(-2.0 * np.sum(p * np.log(p) + q * np.log(q)))


@dataclass
class GroundState:
    rho: np.ndarray
    eps: np.ndarray
    C: np.ndarray
    f: np.ndarray
    q: np.ndarray
    dq: np.ndarray
    iters: int
    residual: float


# Electronic temperature floor of the charge-response estimate in the SCC preconditioner.
PRECOND_KT = 0.02


def scc_preconditioned(sysm, eps, gamma, resid, kT):
    """Charge-sloshing preconditioner of the SCC residual (the paper names no mixer;
    the fixed point does not depend on it).

    A potential change dv moves the charges by about chi dv; model chi as a constant
    density of states per atom at the Fermi level, c, acting on the charge-neutral
    subspace: chi = -c (1 - 11^T / n_atoms).  One Newton step of the charge cycle,
    dq_out = dq_in + chi gamma dq_in, is then x = (1 - chi gamma)^-1 resid.  c is
    the Fermi-function derivative summed over the levels, at an electronic
    temperature of at least PRECOND_KT so that a gap at the Fermi level does not
    switch it off."""
    nat = sysm.n_atoms
    ke = max(kT, PRECOND_KT)
    f = fermi_occupations(eps, sysm.n_electrons, ke)
    c = float(np.sum(f * (1.0 - f / 2.0) / ke)) / nat
    chi = -c * (np.eye(nat) - np.full((nat, nat), 1.0 / nat))
    return np.linalg.solve(np.eye(nat) - chi @ gamma, resid)


def ground_state(sysm, S, H0, gamma, R, scc, E_static=None, tol=1e-12, max_iter=400,
                 mix=0.3, history=8, kT=0.0):
    """SCC ground state: Anderson mixing of the preconditioned charge residual
    (scc_preconditioned; the paper names no mixer, and the fixed point does not
    depend on it)."""
    q0 = reference_populations(sysm)
    E = np.zeros(3) if E_static is None else np.asarray(E_static, dtype=np.float64)
    dq = np.zeros(sysm.n_atoms)
    xs, fs = [], []
    res = np.inf
    for it in range(1, max_iter + 1):
        v = atom_potential(gamma, dq, R, E, scc)
        H = scc_hamiltonian(sysm, H0, S, v)
        eps, C = sla.eigh(H, S)
        f = fermi_occupations(eps, sysm.n_electrons, kT)
        rho = (C * f) @ C.T
        q = mulliken(sysm, rho, S)
        dq_out = q - q0
        resid = dq_out - dq
        res = float(np.max(np.abs(resid))) if scc else 0.0
        if not scc or res <= tol:
            return GroundState(rho, eps, C, f, q, dq_out, it, res)
        pres = scc_preconditioned(sysm, eps, gamma, resid, kT)
        xs.append(dq.copy())
        fs.append(pres.copy())
        xs, fs = xs[-history:], fs[-history:]
        if len(xs) > 1:
            dX = np.array([xs[i + 1] - xs[i] for i in range(len(xs) - 1)]).T
            dF = np.array([fs[i + 1] - fs[i] for i in range(len(fs) - 1)]).T
            g, *_ = np.linalg.lstsq(dF, pres, rcond=None)
            dq = dq + mix * pres - (dX + mix * dF) @ g
        else:
            dq = dq + mix * pres
    raise RuntimeError(f"SCC not converged: residual {res}")


# ---------------------------------------------------------------------------
# Kick (eq:rhokick), equation of motion (eq:eomrho), NAC (eq:nac)
# ---------------------------------------------------------------------------

def kick(sysm, rho0, S, Sinv, R, strength, direction):
    """rho(0+) = 1/2 (e^{iV} rho0 S e^{-iV} S^-1 + S^-1 e^{iV} S rho0 e^{-iV}),
    V = -mu.E_kick with the dipole operator read as the on-site position
    operator: V = -E0 diag(e . R_A(mu)) (hbar = 1)."""
    e = np.asarray(direction, dtype=np.float64)
    x = np.repeat(R @ e, sysm.orbs_per_atom)
    V = -strength * x
    eiV = np.diag(np.exp(1j * V))
    emiV = np.diag(np.exp(-1j * V))
    return 0.5 * (eiV @ rho0 @ S @ emiV @ Sinv + Sinv @ eiV @ S @ rho0 @ emiV)


def rho_dot(rho, Sinv, H, D=None):
    """eq:eomrho: -i (S^-1 H rho - rho H S^-1) - (S^-1 D rho + rho D^dagger S^-1)."""
    out = -1j * (Sinv @ H @ rho - rho @ H @ Sinv)
    if D is not None:
        out = out - (Sinv @ D @ rho + rho @ D.conj().T @ Sinv)
    return out


def nac_matrix(sysm, R, V):
    """D_mu_nu = Rdot_B . grad_B S_mu_nu (1 - delta_AB), mu in A, nu in B (eq:nac);
    on-site blocks zero (eq:onsite discussion)."""
    n = sysm.orbs_per_atom
    nat = R.shape[0]
    D4 = np.zeros((nat, n, nat, n))
    iA, iB, _, gS = model_pair_gradients(sysm, R)
    # mu in A, nu in B: the S block depends on R_B - R_A, so grad_B S = +gS
    D4[iA, :, iB, :] = np.einsum("pg,pgij->pij", V[iB], gS)
    # mu in B, nu in A: S_mu_nu = block_AB[nu, mu] and grad_A of it is -gS
    D4[iB, :, iA, :] = np.einsum("pg,pgij->pji", V[iA], -gS)
    return D4.reshape(n * nat, n * nat)


# ---------------------------------------------------------------------------
# Energies and forces
# ---------------------------------------------------------------------------

def repulsive_energy(sysm, R):
    iA, iB = pair_list(R.shape[0])
    r = np.linalg.norm(R[iB] - R[iA], axis=1)
    return float(np.sum(sysm.rep_A * np.exp(-r / sysm.rep_b)))


def energy_terms(sysm, rho, H0, gamma, dq, R, E, Vel, scc):
    """E = Tr{rho H0} + 1/2 sum gamma dq dq + E_rep + KE + sum_A dq_A V^ext_A."""
    e_band = float(np.real(np.sum(rho * H0.T)))
    e_coul = 0.5 * float(dq @ gamma @ dq) if scc else 0.0
    e_rep = repulsive_energy(sysm, R) if sysm.rep_A else 0.0
    e_ext = float(dq @ (R @ E))
    e_kin = 0.0
    if Vel is not None:
        m = sysm.mass[sysm.species] * AMU
        e_kin = 0.5 * float(np.sum(m[:, None] * Vel * Vel))
    return dict(E_band=e_band, E_coul=e_coul, E_rep=e_rep, E_ext=e_ext, E_kin=e_kin,
                E_total=e_band + e_coul + e_rep + e_ext + e_kin)


def forces(sysm, rho, S, Sinv, H, gamma, dq, v_atom, R, E, scc):
    """Ehrenfest force of eq:forces with the velocity-dependent terms dropped
    (as the paper's implementation does).  The S-derivative ("Pulay") terms are
    read in energy-weighted form:

      F_A = -Re Tr{rho dH0/dR_A} - 1/2 Re sum rho_nu_mu dS_mu_nu/dR_A (v_mu + v_nu)
            + Re Tr{W dS/dR_A} - dq_A sum_B dgamma_AB/dR_A dq_B - dE_rep/dR_A - dq_A E(t),
      W = 1/2 (S^-1 H rho + rho H S^-1)
    """
    n = sysm.orbs_per_atom
    nat = R.shape[0]
    F = np.zeros((nat, 3))
    W = 0.5 * (Sinv @ H @ rho + rho @ H @ Sinv)
    iA, iB, gH, gS = model_pair_gradients(sysm, R)
    if iA.size:
        rho4 = rho.reshape(nat, n, nat, n)
        W4 = W.reshape(nat, n, nat, n)
        rho_ab, rho_ba = rho4[iA, :, iB, :], rho4[iB, :, iA, :]
        W_ab, W_ba = W4[iA, :, iB, :], W4[iB, :, iA, :]
        dH_A, dS_A = -gH, -gS      # d/dR_A of the (A, B) blocks
        # sum over mu in A, nu in B of X_nu_mu dY_mu_nu, plus the (B, A) half (dY^T)
        t_h = np.einsum("pji,pgij->pg", rho_ba, dH_A) + np.einsum("pij,pgij->pg", rho_ab, dH_A)
        t_s = np.einsum("pji,pgij->pg", rho_ba, dS_A) + np.einsum("pij,pgij->pg", rho_ab, dS_A)
        t_w = np.einsum("pji,pgij->pg", W_ba, dS_A) + np.einsum("pij,pgij->pg", W_ab, dS_A)
        vv = (v_atom[iA] + v_atom[iB])[:, None]
        f_a = -np.real(t_h) - 0.5 * np.real(t_s) * vv + np.real(t_w)
        np.add.at(F, iA, f_a)
        np.add.at(F, iB, -f_a)
        d = R[iA] - R[iB]
        r = np.linalg.norm(d, axis=1)
        u = d / r[:, None]
        if scc:
            U = sysm.hubbard_U[sysm.species]
            # E_coul = 1/2 sum gamma dq dq: the A-B pair term gives -dq_A dq_B dgamma/dR_A
            fg = -(dq[iA] * dq[iB] * gamma_pair_dR(U[iA], U[iB], r))[:, None] * u
            np.add.at(F, iA, fg)
            np.add.at(F, iB, -fg)
        if sysm.rep_A:
            fr = (sysm.rep_A / sysm.rep_b * np.exp(-r / sysm.rep_b))[:, None] * u
            np.add.at(F, iA, fr)
            np.add.at(F, iB, -fr)
    F -= dq[:, None] * E[None, :]
    return F


# ---------------------------------------------------------------------------
# Propagation (eq:leapfrog with an Euler first step; velocity Verlet nuclei)
# ---------------------------------------------------------------------------

@dataclass
class Trajectory:
    t: np.ndarray            # (K+1,)
    dipole: np.ndarray       # (K+1, 3)
    charges: np.ndarray      # (K+1, n_atoms)
    energy: np.ndarray       # (K+1,) E_total
    trace: np.ndarray        # (K+1,) complex Tr(rho S)
    herm: np.ndarray         # (K+1,) max |rho - rho^dagger|
    work: np.ndarray         # (K+1,) integral of P dt (trapezoid)
    forces: Optional[np.ndarray]
    R: np.ndarray
    V: Optional[np.ndarray]
    rho_prev: np.ndarray
    rho: np.ndarray


def dipole(dq, R):
    """mu = -sum_A dq_A R_A (electrons carry charge -1; monopole approximation)."""
    return -(dq @ R)


def propagate(sysm, run, rho_init, n_steps, R=None, V=None, rho_prev=None, step0=0,
              t0=0.0, dt=None, keep_forces=False):
    """Integrate eq:eomrho with eq:leapfrog from rho_init for n_steps.

    If rho_prev is None the first step is Euler (Sec. 2.3).  Observables are
    recorded for rho_0 ... rho_K.  With moving nuclei, at step n (holding
    R_n, V_{n-1/2}, rho_{n-1}, rho_n): S_n; q(rho_n), H_n; F_n; V_n = V_{n-1/2}
    + F_n dt/2m; D_n(V_n); rho_{n+1}; V_{n+1/2} = V_n + F_n dt/2m;
    R_{n+1} = R_n + dt V_{n+1/2}  (the paper does not fix this order).
    """
    dt = run.dt if dt is None else dt
    R = np.array(sysm.R if R is None else R, dtype=np.float64)
    move = run.move_nuclei
    Vh = None
    if move:
        Vh = np.array(sysm.V if V is None else V, dtype=np.float64)   # V_0 at the start
    m = sysm.mass[sysm.species] * AMU
    q0 = reference_populations(sysm)
    rec = dict(t=[], dip=[], q=[], E=[], tr=[], herm=[], work=[], F=[])
    S, H0 = model_matrices(sysm, R)
    Sinv = sla.cho_solve(sla.cho_factor(S, lower=True), np.eye(S.shape[0]))
    gamma = gamma_matrix(sysm, R) if run.scc else None
    rho = np.array(rho_init, dtype=np.complex128)
    prev = None if rho_prev is None else np.array(rho_prev, dtype=np.complex128)
    work = 0.0
    P_last = None
    first_half = prev is None

    def observe(n, rho, S, H0, gamma, R, Vn, E, dq, P, F):
        rec["t"].append(t0 + n * dt)
        rec["dip"].append(dipole(dq, R))
        rec["q"].append(dq + q0)
        en = energy_terms(sysm, rho, H0, gamma if gamma is not None else np.zeros((1, 1)),
                          dq, R, E, Vn, run.scc)
        rec["E"].append(en["E_total"])
        rec["tr"].append(np.trace(rho @ S))
        rec["herm"].append(float(np.max(np.abs(rho - rho.conj().T))))
        rec["work"].append(work)
        if keep_forces:
            rec["F"].append(F)

    for k in range(n_steps + 1):
        n = step0 + k
        t = t0 + k * dt
        if move and k > 0:
            S, H0 = model_matrices(sysm, R)
            Sinv = sla.cho_solve(sla.cho_factor(S, lower=True), np.eye(S.shape[0]))
            if run.scc:
                gamma = gamma_matrix(sysm, R)
        E = field_at(run.field, t)
        dq = mulliken(sysm, rho, S) - q0
        v = atom_potential(gamma, dq, R, E, run.scc)
        H = scc_hamiltonian(sysm, H0, S, v)
        F = None
        D = None
        Vn = None
        P = 0.0
        if move:
            F = forces(sysm, rho, S, Sinv, H, gamma, dq, v, R, E, run.scc)
            Vn = Vh if (first_half and k == 0) else Vh + F * dt / (2.0 * m[:, None])
            D = nac_matrix(sysm, R, Vn)
            P = float(np.real(np.trace(Sinv @ H @ rho @ (D - D.T))))
            if P_last is not None:
                work += 0.5 * dt * (P + P_last)
            P_last = P
        elif keep_forces:
            F = forces(sysm, rho, S, Sinv, H, gamma, dq, v, R, E, run.scc)
        observe(k, rho, S, H0, gamma, R, Vn, E, dq, P, F)
        if k == n_steps:
            break
        rdot = rho_dot(rho, Sinv, H, D)
        if prev is None:
            new = rho + dt * rdot
        else:
            new = prev + 2.0 * dt * rdot
        prev, rho = rho, new
        if move:
            Vh = Vn + F * dt / (2.0 * m[:, None])
            R = R + dt * Vh
    return Trajectory(np.array(rec["t"]), np.array(rec["dip"]), np.array(rec["q"]),
                      np.array(rec["E"]), np.array(rec["tr"]), np.array(rec["herm"]),
                      np.array(rec["work"]), np.array(rec["F"]) if rec["F"] else None,
                      R, Vh, prev, rho)


def setup(sysm, run, E_static=None):
    """Model, ground state and (optional) kick at t = 0: returns (rho after kick, gs, S, Sinv)."""
    R = np.asarray(sysm.R, dtype=np.float64)
    S, H0 = model_matrices(sysm, R)
    Sinv = sla.cho_solve(sla.cho_factor(S, lower=True), np.eye(S.shape[0]))
    gamma = gamma_matrix(sysm, R) if run.scc else np.zeros((sysm.n_atoms, sysm.n_atoms))
    gs = ground_state(sysm, S, H0, gamma, R, run.scc, E_static=E_static, tol=run.scc_tol,
                      max_iter=run.scc_max_iter, kT=run.kT)
    rho = gs.rho.astype(np.complex128)
    if run.kick:
        rho = kick(sysm, rho, S, Sinv, R, run.kick, run.kick_dir)
    return rho, gs, S, Sinv


def run_trajectory(sysm, run, n_steps=None, keep_forces=False):
    rho, gs, S, Sinv = setup(sysm, run)
    n = run.n_steps if n_steps is None else n_steps
    return propagate(sysm, run, rho, n, keep_forces=keep_forces), gs


# ---------------------------------------------------------------------------
# Windowed propagation with a frozen Hamiltonian, and the per-atom shift network
# (the learned form: a network predicts the window-averaged SCC shift, the window is
# then propagated in closed form)
# ---------------------------------------------------------------------------

def window_propagate(rho_prev, rho, S, H_bar, dt, k):
    """k leapfrog steps of eq:eomrho (eq:leapfrog) with the Hamiltonian frozen at H_bar,
    in closed form.  In the generalised eigenbasis H_bar C = S C eps (C^T S C = 1) the
    leapfrog acts element by element, x_{m+1} = x_{m-1} - 2 i dt w x_m with
    w = eps_a - eps_b, solved by x_m = A l+^m + B l-^m, l+- = -i theta +- sqrt(1 - theta^2),
    theta = w dt (the leapfrog's own modes, not exp(-i w m dt)).  With P = S C,
    rho~ = P^T rho P and rho = C rho~ C^T.  Returns (rho_{n-1+k}, rho_{n+k}) from
    (rho_{n-1}, rho_n)."""
    eps, C = sla.eigh(H_bar, S)
    P = S @ C
    x0 = P.T @ np.asarray(rho_prev, dtype=np.complex128) @ P
    x1 = P.T @ np.asarray(rho, dtype=np.complex128) @ P
    theta = (eps[:, None] - eps[None, :]) * dt
    c = np.sqrt(1.0 - theta ** 2)
    lp = -1j * theta + c
    lm = -1j * theta - c
    A = (x1 - lm * x0) / (lp - lm)
    B = x0 - A
    xk = A * lp ** k + B * lm ** k
    xk1 = A * lp ** (k + 1) + B * lm ** (k + 1)
    return C @ xk @ C.T, C @ xk1 @ C.T


def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    a = (a + 0x7FFF + ((a >> 16) & 1)) & 0xFFFF0000
    return a.astype(np.uint32).view(np.float32).astype(np.float64)


def shiftnet_unpack(params, F, H):
    """Packed parameters: W1 (F x H), b1 (H), W2 (H x H), b2 (H), w3 (H), b3 (1)."""
    p = np.asarray(params, dtype=np.float64)
    o = 0
    W1 = p[o:o + F * H].reshape(F, H); o += F * H
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    w3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def shiftnet_forward(params, X, F, H, bf16=True):
    """Per-atom network y = w3 . tanh(W2^T tanh(W1^T x + b1) + b2) + b3; the weight
    matrices enter rounded to bfloat16 when bf16 is set (biases and activations are
    not rounded).  Returns y and the hidden activations."""
    W1, b1, W2, b2, w3, b3 = shiftnet_unpack(params, F, H)
    if bf16:
        W1, W2, w3 = bf16_round(W1), bf16_round(W2), bf16_round(w3)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.tanh(X @ W1 + b1)
    h2 = np.tanh(h1 @ W2 + b2)
    return h2 @ w3 + b3, (X, h1, h2, W2, w3)


def shiftnet_loss_grad(params, X, Y, F, H, bf16=True):
    """Mean squared error and its gradient with respect to the packed parameters (the
    gradient through the bfloat16 rounding is taken as that of the rounded weights)."""
    y, (X, h1, h2, W2, w3) = shiftnet_forward(params, X, F, H, bf16)
    n = X.shape[0]
    r = y - np.asarray(Y, dtype=np.float64)
    loss = float(np.mean(r * r))
    dy = 2.0 * r / n
    dw3 = h2.T @ dy
    db3 = np.sum(dy)
    dz2 = np.outer(dy, w3) * (1.0 - h2 * h2)
    dW2 = h1.T @ dz2
    db2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2.T) * (1.0 - h1 * h1)
    dW1 = X.T @ dz1
    db1 = dz1.sum(axis=0)
    g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dw3, [db3]])
    return loss, g
