"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test compares the oracle with something that is not the oracle itself:
numerical quadrature, finite differences, closed-form solutions, textbook
special cases and exact invariants.  They are chosen so that a plausible slip
(a dropped factor, a wrong sign, a transposed operand, a wrong time index)
fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla
from scipy import integrate

from oracle import tdb_oracle as O
from paper_1912_03174_gb300 import inputs as I


# ---------------------------------------------------------------------------
# gamma (eq:coul) against a 2-D quadrature of the Coulomb integral
# ---------------------------------------------------------------------------

def _coulomb_integral(tA, tB, R):
    """Integral of n_B(r') phi_A(|r' - R|) over space, n = tau^3/(8 pi) e^{-tau r},
    phi_A the electrostatic potential of n_A (hydrogen-like 1s textbook form),
    by scipy 2-D quadrature in (r', cos theta)."""
    def phiA(s):
        if s < 1e-12:
            return tA / 2.0
        return (1.0 - math.exp(-tA * s) * (1.0 + tA * s / 2.0)) / s

    def nB(r):
        return tB ** 3 / (8 * math.pi) * math.exp(-tB * r)

    def f(ct, r):
        s = math.sqrt(max(r * r + R * R - 2 * r * R * ct, 0.0))
        return nB(r) * phiA(s) * 2 * math.pi * r * r

    rmax = 60.0 / tB
    val, _ = integrate.dblquad(f, 0.0, rmax, -1.0, 1.0, epsabs=1e-11, epsrel=1e-10)
    return val


def test_potential_of_exponential_density_is_the_textbook_form():
    # phi(s) = (1/s) int_0^s n 4 pi r^2 dr + int_s^inf n 4 pi r dr, by 1-D quadrature
    t = 1.3
    n = lambda r: t ** 3 / (8 * math.pi) * math.exp(-t * r)
    for s in (0.3, 1.0, 2.68, 6.0):
        inner, _ = integrate.quad(lambda r: n(r) * 4 * math.pi * r * r, 0, s, epsabs=1e-13)
        outer, _ = integrate.quad(lambda r: n(r) * 4 * math.pi * r, s, np.inf, epsabs=1e-13)
        closed = (1.0 - math.exp(-t * s) * (1.0 + t * s / 2.0)) / s
        assert abs(inner / s + outer - closed) < 1e-11


@pytest.mark.parametrize("UA,UB", [(0.4, 0.4), (0.3, 0.5), (0.35, 0.45)])
@pytest.mark.parametrize("R", [2.68, 5.0])
def test_gamma_matches_coulomb_quadrature(UA, UB, R):
    q = _coulomb_integral(3.2 * UA, 3.2 * UB, R)
    g = float(O.gamma_pair(UA, UB, R))
    assert abs(g - q) < 2e-8, (g, q)


def test_gamma_limits():
    # R -> 0 gives U (tau = 16 U / 5 makes the on-site integral equal U)
    U = 0.4
    assert abs(float(O.gamma_pair(U, U, 1e-5)) - U) < 1e-5
    # R -> infinity gives the bare Coulomb 1/R
    for UA, UB in [(0.4, 0.4), (0.3, 0.5)]:
        assert abs(float(O.gamma_pair(UA, UB, 40.0)) - 1.0 / 40.0) < 1e-12
    # the unequal-exponent branch joins the equal one continuously at the switch
    lo = float(O.gamma_pair(0.4, 0.4 * (1 + 0.999 * O.GAMMA_EQUAL_REL), 3.0))
    hi = float(O.gamma_pair(0.4, 0.4 * (1 + 1.001 * O.GAMMA_EQUAL_REL), 3.0))
    assert abs(lo - hi) < 3e-8


def test_gamma_derivative_finite_difference():
    h = np.finfo(float).eps ** 0.25
    for UA, UB in [(0.4, 0.4), (0.3, 0.5)]:
        for R in (2.4, 3.7, 8.0):
            fd = (float(O.gamma_pair(UA, UB, R + h)) - float(O.gamma_pair(UA, UB, R - h))) / (2 * h)
            assert abs(fd - float(O.gamma_pair_dR(UA, UB, R))) < 1e-8


# ---------------------------------------------------------------------------
# two-centre model: symmetry, rotation covariance, positive overlap, derivatives
# ---------------------------------------------------------------------------

def _systems():
    return [I.chain_c1()[0], I.small_flake(12, seed=7), I.small_cluster(8, seed=11)]


def test_model_symmetric_and_overlap_positive_definite():
    for s in _systems():
        S, H0 = O.model_matrices(s, s.R)
        assert np.array_equal(S, S.T) and np.array_equal(H0, H0.T)
        assert np.linalg.eigvalsh(S).min() > 0.05


def test_model_rotation_covariance():
    # rotating the geometry by Q transforms each atom's (s, p) block by 1 (+) Q
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    for s in _systems():
        S, H0 = O.model_matrices(s, s.R)
        S2, H2 = O.model_matrices(s, s.R @ Q.T)
        T1 = sla.block_diag(1.0, Q)
        T = np.kron(np.eye(s.n_atoms), T1)
        assert np.max(np.abs(T @ S @ T.T - S2)) < 1e-13
        assert np.max(np.abs(T @ H0 @ T.T - H2)) < 1e-13


def test_model_gradients_match_central_difference():
    # eq:overprime: central difference with Delta R = eps^(1/4)
    s = I.small_cluster(5, seed=2)
    h = np.finfo(float).eps ** 0.25
    n = s.orbs_per_atom
    iA, iB, gH, gS = O.model_pair_gradients(s, s.R)
    for p in range(iA.size):
        a, b = iA[p], iB[p]
        for g in range(3):
            Rp, Rm = s.R.copy(), s.R.copy()
            Rp[b, g] += h
            Rm[b, g] -= h
            Sp, Hp = O.model_matrices(s, Rp)
            Sm, Hm = O.model_matrices(s, Rm)
            blk = (slice(a * n, (a + 1) * n), slice(b * n, (b + 1) * n))
            assert np.max(np.abs((Sp - Sm)[blk] / (2 * h) - gS[p, g])) < 1e-8
            assert np.max(np.abs((Hp - Hm)[blk] / (2 * h) - gH[p, g])) < 1e-8


def test_nac_is_the_time_derivative_of_the_overlap():
    # dS/dt = D + D^T along R(t) = R + t V, D_AA = 0 (eq:nac, eq:gradover)
    s = I.small_cluster(6, seed=5)
    V = np.random.default_rng(1).normal(size=(s.n_atoms, 3)) * 1e-2
    D = O.nac_matrix(s, s.R, V)
    h = 1e-4
    Sp, _ = O.model_matrices(s, s.R + h * V)
    Sm, _ = O.model_matrices(s, s.R - h * V)
    assert np.max(np.abs((Sp - Sm) / (2 * h) - (D + D.T))) < 1e-9
    n = s.orbs_per_atom
    for A in range(s.n_atoms):
        assert np.all(D[A * n:(A + 1) * n, A * n:(A + 1) * n] == 0)
    # common velocity (no relative motion): D^T = -D (Sec. 2.1 remark (b))
    Dc = O.nac_matrix(s, s.R, np.tile([1e-2, -2e-2, 3e-3], (s.n_atoms, 1)))
    assert np.max(np.abs(Dc + Dc.T)) < 1e-15


# ---------------------------------------------------------------------------
# kick (eq:rhokick)
# ---------------------------------------------------------------------------

def test_kick_hermitian_trace_exact_and_sign():
    s = I.small_flake(12, seed=9, n_species=2)
    run = I.Run(dt=0.1, n_steps=0, scc=True, kick=1e-3, kT=I.SCC_KT)
    R = s.R
    S, H0 = O.model_matrices(s, R)
    Sinv = np.linalg.inv(S)
    gamma = O.gamma_matrix(s, R)
    gs = O.ground_state(s, S, H0, gamma, R, True, kT=I.SCC_KT)
    rho = O.kick(s, gs.rho.astype(complex), S, Sinv, R, 1e-3, [1, 0, 0])
    assert np.max(np.abs(rho - rho.conj().T)) < 1e-15
    assert abs(np.trace(rho @ S) - s.n_electrons) < 1e-12
    # zero kick returns the ground state
    rho0 = O.kick(s, gs.rho.astype(complex), S, Sinv, R, 0.0, [1, 0, 0])
    assert np.max(np.abs(rho0 - gs.rho)) < 1e-13
    # physical sign: a delta field along +x pushes electrons to -x, so mu_x grows
    tr = O.propagate(s, run, rho, 20)
    assert tr.dipole[5, 0] - tr.dipole[0, 0] > 0
    assert np.all(np.diff(tr.dipole[:20, 0]) > 0)


def test_kick_orthogonal_basis_is_a_phase_transform():
    # S = I: rho(0+) = exp(-i E0 x) rho0 exp(+i E0 x) with x the on-site positions
    s = I.small_flake(8, seed=4, scc=False)
    s.s0 = 0.0
    S, H0 = O.model_matrices(s, s.R)
    assert np.array_equal(S, np.eye(S.shape[0]))
    gs = O.ground_state(s, S, H0, np.zeros((8, 8)), s.R, False)
    x = np.repeat(s.R[:, 0], 4)
    E0 = 0.05
    U = np.diag(np.exp(-1j * E0 * x))
    ref = U @ gs.rho @ U.conj().T
    rho = O.kick(s, gs.rho.astype(complex), S, S, s.R, E0, [1, 0, 0])
    assert np.max(np.abs(rho - ref)) < 1e-15


# ---------------------------------------------------------------------------
# propagation: closed form of the linear (non-SCC) case, Rabi, invariants
# ---------------------------------------------------------------------------

def _leapfrog_closed_form(x0, omega, dt, n):
    """Exact solution of x_{k+1} = x_{k-1} - 2 i dt omega x_k, x_1 = (1 - i omega dt) x_0."""
    root = np.sqrt(1.0 - (omega * dt) ** 2 + 0j)
    lp, lm = -1j * omega * dt + root, -1j * omega * dt - root
    x1 = (1.0 - 1j * omega * dt) * x0
    A = (x1 - lm * x0) / (lp - lm)
    B = x0 - A
    return A * lp ** n + B * lm ** n


def test_leapfrog_matches_closed_form_in_the_eigenbasis():
    s, run = I.chain_c1()
    rho, gs, S, Sinv = O.setup(s, run)
    K = 300
    tr = O.propagate(s, run, rho, K)
    # generalised eigenbasis: C^T S C = 1, S^-1 H0 C = C eps; rho~ = C^T S rho S C
    eps, C = sla.eigh(O.model_matrices(s, s.R)[1], S)
    rt0 = C.T @ S @ rho @ S @ C
    omega = eps[:, None] - eps[None, :]
    rtK = _leapfrog_closed_form(rt0, omega, run.dt, K)
    rtK1 = _leapfrog_closed_form(rt0, omega, run.dt, K - 1)
    assert np.max(np.abs(C @ rtK @ C.T - tr.rho)) < 1e-12
    assert np.max(np.abs(C @ rtK1 @ C.T - tr.rho_prev)) < 1e-12


def _mode_fit_residual(y, n, theta):
    """Relative residual of the least-squares fit of y(n) by {1, cos(theta n), sin(theta n)}."""
    basis = [np.ones_like(y)]
    for th in theta:
        basis += [np.cos(th * n), np.sin(th * n)]
    Bm = np.array(basis).T
    assert Bm.shape[0] > 4 * Bm.shape[1]          # far more samples than columns
    coef, *_ = np.linalg.lstsq(Bm, y, rcond=None)
    return np.max(np.abs(Bm @ coef - y)) / np.max(np.abs(y))


def test_kick_spectrum_peaks_at_orbital_energy_differences():
    # After a weak kick the non-SCC dipole is, to first order in the kick, a sum of modes
    # of the transitions between occupied and empty levels, w = e_a - e_i; the leapfrog carries each mode as
    # lambda_+^n = e^{-i arcsin(w dt) n} plus a small parasitic lambda_-^n = (-1)^n e^{+i ...},
    # so on even steps both are cos/sin of 2 arcsin(w dt) m.  A fit with these frequencies
    # leaves only the second-order (kick^2) terms; over 20000 steps the fit resolves a 0.1%
    # shift of the frequencies and even the leapfrog's arcsin(w dt) against w dt.
    import dataclasses
    s, run = I.chain_c1()
    run = dataclasses.replace(run, kick=1e-6)
    rho, gs, S, Sinv = O.setup(s, run)
    K = 20000
    tr = O.propagate(s, run, rho, K)
    mu = tr.dipole[:, 0] - tr.dipole[0, 0]
    # every pair of levels with different occupations (the chain's HOMO is a degenerate
    # pair sharing two electrons, f = 1 each): first-order amplitude ~ f_i - f_j
    i, j = np.triu_indices(gs.eps.size, 1)
    keep = np.abs(gs.f[i] - gs.f[j]) > 1e-12
    w = gs.eps[j[keep]] - gs.eps[i[keep]]
    n = np.arange(0, K + 1, 2)
    y = mu[n]
    theta = np.arcsin(w * run.dt)                   # phase per step of each transition
    r_true = _mode_fit_residual(y, n, theta)
    r_shift = _mode_fit_residual(y, n, np.arcsin(1.001 * w * run.dt))
    r_naive = _mode_fit_residual(y, n, w * run.dt)  # e^{-i w t} instead of the leapfrog's phase
    assert r_true < 1e-6, r_true
    assert r_shift > 1e-3, r_shift                  # frequencies 0.1% off: most of it left
    assert r_naive > 100 * r_true, (r_naive, r_true)


def test_two_level_rabi_oscillation():
    # two sites, one s orbital, S = I, hopping -t; drive at the leapfrog-resonant frequency
    d, t = 2.0, 0.25
    s = I.two_level(d, t)
    w0 = 2 * t
    dt = 0.2
    wl = math.asin(w0 * dt) / dt
    E0 = 5e-4
    Omega = E0 * d / 2.0
    fld = I.Field(E0=E0, omega=wl, phase=math.pi / 2, envelope=0)
    run = I.Run(dt=dt, n_steps=0, scc=False, field=fld)
    S, H0 = O.model_matrices(s, s.R)
    assert np.array_equal(S, np.eye(2))
    gs = O.ground_state(s, S, H0, np.zeros((2, 2)), s.R, False)
    K = int(round(math.pi / Omega / dt))
    # sample the upper-level population along the way
    a = np.array([1.0, -1.0]) / math.sqrt(2.0)
    rho = gs.rho.astype(complex)
    prev = None
    step = K // 8
    for j in range(8):
        tr = O.propagate(s, run, rho, step, rho_prev=prev, step0=j * step, t0=j * step * dt)
        rho, prev = tr.rho, tr.rho_prev
        tt = (j + 1) * step * dt
        pop = float(np.real(a @ rho @ a))
        assert abs(pop - 2 * math.sin(Omega * tt / 2) ** 2) < 6e-3, (j, pop)


def _kicked_flake(n_atoms=12, seed=21, kick=1e-2, dt=0.2, field=None, scc=True, n_species=1):
    s = I.small_flake(n_atoms, seed=seed, scc=scc, n_species=n_species)
    run = I.Run(dt=dt, n_steps=0, scc=scc, kick=kick, field=field, kT=I.SCC_KT if scc else 0.0)
    rho, gs, S, Sinv = O.setup(s, run)
    return s, run, rho, gs, S


def test_ground_state_is_stationary():
    for scc in (False, True):
        s, run, rho, gs, S = _kicked_flake(16, seed=3, kick=0.0, scc=scc)
        tr = O.propagate(s, run, rho, 2000)
        tol = 1e-12 if not scc else 1e-9
        assert np.max(np.abs(tr.rho - gs.rho)) < tol
        assert np.max(np.abs(tr.dipole - tr.dipole[0])) < tol


def test_trace_and_hermiticity_conserved():
    s, run, rho, gs, S = _kicked_flake(12, seed=5, kick=1e-2)
    tr = O.propagate(s, run, rho, 2000)
    assert np.max(np.abs(tr.trace - s.n_electrons)) / s.n_electrons < 1e-12
    assert np.max(tr.herm) < 1e-13
    assert np.max(np.abs(tr.charges.sum(axis=1) - s.n_electrons)) < 1e-10


def test_time_reversal():
    fld = I.Field(E0=0.02, omega=0.3, phase=0.4, fwhm=40.0, envelope=2)
    s, run, rho, gs, S = _kicked_flake(10, seed=8, kick=1e-2, field=fld)
    K = 300
    fwd = O.propagate(s, run, rho, K)
    # leapfrog run backwards from (rho_K, rho_{K-1}) with -dt returns to rho_0
    back = O.propagate(s, run, fwd.rho_prev, K - 1, rho_prev=fwd.rho, t0=(K - 1) * run.dt,
                       dt=-run.dt)
    assert np.max(np.abs(back.rho - rho)) < 1e-12


def test_scc_energy_conserved_to_second_order():
    # field-free SCC dynamics conserves E = Tr rho H0 + 1/2 dq gamma dq exactly in
    # continuous time (dE/dt = Tr(rho_dot H) = 0); leapfrog keeps it to O(dt^2)
    errs = []
    for dt in (0.2, 0.1):
        s, run, rho, gs, S = _kicked_flake(12, seed=13, kick=5e-2, dt=dt)
        K = int(round(100.0 / dt))
        tr = O.propagate(s, run, rho, K)
        errs.append(np.max(np.abs(tr.energy - tr.energy[0])))
        excitation = tr.energy[0] - O.energy_terms(
            s, gs.rho, O.model_matrices(s, s.R)[1], O.gamma_matrix(s, s.R), gs.dq, s.R,
            np.zeros(3), None, True)["E_total"]
        assert errs[-1] < 0.05 * excitation
    assert 3.0 < errs[0] / errs[1] < 5.0, errs


def test_ground_state_force_equals_minus_energy_gradient():
    # eq:forces at the ground state (rho_dot = 0) is -dE_GS/dR; a static field is on
    s = I.small_cluster(5, seed=17)
    E = np.array([0.01, -0.004, 0.002])

    def egs(R):
        S, H0 = O.model_matrices(s, R)
        G = O.gamma_matrix(s, R)
        gs = O.ground_state(s, S, H0, G, R, True, E_static=E, tol=1e-13)
        return gs, S, H0, G

    gs, S, H0, G = egs(s.R)
    Sinv = np.linalg.inv(S)
    v = O.atom_potential(G, gs.dq, s.R, E, True)
    H = O.scc_hamiltonian(s, H0, S, v)
    F = O.forces(s, gs.rho, S, Sinv, H, G, gs.dq, v, s.R, E, True)
    h = 1e-4
    for A in range(s.n_atoms):
        for g in range(3):
            Rp, Rm = s.R.copy(), s.R.copy()
            Rp[A, g] += h
            Rm[A, g] -= h
            ep = O.energy_terms(s, *(lambda r: (r[0].rho, r[2], r[3], r[0].dq))(egs(Rp)), Rp, E, None, True)
            em = O.energy_terms(s, *(lambda r: (r[0].rho, r[2], r[3], r[0].dq))(egs(Rm)), Rm, E, None, True)
            fd = -(ep["E_total"] - em["E_total"]) / (2 * h)
            assert abs(fd - F[A, g]) < 2e-8, (A, g, fd, F[A, g])
    # no net force without a field (translation invariance); with it, sum F = -sum dq E = 0
    assert np.max(np.abs(F.sum(axis=0))) < 1e-12


def test_ehrenfest_energy_minus_work_is_conserved():
    # dE/dt = P = Re Tr[S^-1 H rho (D - D^T)] once the velocity terms of eq:forces are
    # dropped (Sec. 2.1); E - int P dt is conserved to O(dt^2) while E alone is not
    errs, e_alone = [], []
    for dt in (0.2, 0.1):
        s = I.small_cluster(6, seed=23, T=3000.0)
        run = I.Run(dt=dt, n_steps=0, scc=True, move_nuclei=True, kick=1e-2, kT=I.SCC_KT)
        rho, gs, S, Sinv = O.setup(s, run)
        tr = O.propagate(s, run, rho, int(round(80.0 / dt)))
        bal = tr.energy - tr.work
        errs.append(np.max(np.abs(bal - bal[0])))
        e_alone.append(np.max(np.abs(tr.energy - tr.energy[0])))
        # with moving S the electron count is conserved to O(dt^2) only
        assert np.max(np.abs(tr.trace - s.n_electrons)) < 4e-7 * (dt / 0.2) ** 2
    assert errs[1] < 1e-6
    assert 3.0 < errs[0] / errs[1] < 5.0, errs
    assert e_alone[1] > 2.0 * errs[1], (e_alone, errs)


def test_leapfrog_second_order_against_fine_rk4():
    # N = 8 (two atoms): leapfrog error vs an RK4 reference shrinks ~4x per halving of dt
    s = I.small_flake(2, seed=31)
    run = I.Run(dt=0.1, n_steps=0, scc=True, kick=2e-2)
    rho0, gs, S, Sinv = O.setup(s, run)
    H0 = O.model_matrices(s, s.R)[1]
    G = O.gamma_matrix(s, s.R)
    q0 = O.reference_populations(s)

    def f(rho):
        dq = O.mulliken(s, rho, S) - q0
        H = O.scc_hamiltonian(s, H0, S, O.atom_potential(G, dq, s.R, np.zeros(3), True))
        return O.rho_dot(rho, Sinv, H)

    T = 4.0
    h = 1e-3
    ref = rho0.copy()
    for _ in range(int(round(T / h))):
        k1 = f(ref); k2 = f(ref + 0.5 * h * k1); k3 = f(ref + 0.5 * h * k2); k4 = f(ref + h * k3)
        ref = ref + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    errs = []
    for dt in (0.1, 0.05):
        tr = O.propagate(s, run, rho0, int(round(T / dt)), dt=dt)
        errs.append(np.max(np.abs(tr.rho - ref)))
    assert 3.0 < errs[0] / errs[1] < 5.0, errs


def test_scc_ground_state_is_a_fixed_point_of_the_charge_cycle():
    # Sec. 2.1: the ground state reproduces itself: its charges give the Hamiltonian whose
    # occupied generalized eigenvectors rebuild the same density.  Checked by one plain
    # diagonalisation (scipy), independent of the preconditioned mixer that found it, on a
    # 3-D cluster (the case the preconditioner exists for) and a flake.
    for sysm in (I.small_cluster(40, seed=13, T=300.0), I.small_flake(20, seed=3)):
        run = I.Run(dt=0.2, n_steps=0, scc=True, kT=I.SCC_KT)
        R = np.asarray(sysm.R, dtype=np.float64)
        S, H0 = O.model_matrices(sysm, R)
        gamma = O.gamma_matrix(sysm, R)
        gs = O.ground_state(sysm, S, H0, gamma, R, True, kT=run.kT)
        v = gamma @ gs.dq
        vo = np.repeat(v, sysm.orbs_per_atom)
        H = H0 + 0.5 * S * (vo[:, None] + vo[None, :])
        eps, C = sla.eigh(H, S)
        f = O.fermi_occupations(eps, sysm.n_electrons, run.kT)
        rho = (C * f) @ C.T
        assert np.max(np.abs(rho - gs.rho)) < 1e-10
        q = np.array([np.trace((rho @ S)[4 * a:4 * a + 4, 4 * a:4 * a + 4]) for a in range(sysm.n_atoms)])
        assert np.max(np.abs(q - sysm.n_electrons / sysm.n_atoms - gs.dq)) < 1e-11


def test_window_propagation_equals_leapfrog_with_a_frozen_hamiltonian():
    # non-SCC and field-free, so the plain leapfrog's Hamiltonian is frozen at H0: the
    # closed-form window must reproduce k of its steps
    sysm = I.small_flake(12, seed=21, scc=False)
    run = I.Run(dt=0.2, n_steps=0, scc=False, kick=1e-2)
    rho0, gs, S, Sinv = O.setup(sysm, run)
    S, H0 = O.model_matrices(sysm, np.asarray(sysm.R, dtype=np.float64))
    k = 37
    tr1 = O.propagate(sysm, run, rho0, 1)                 # Euler: rho_0, rho_1
    trk = O.propagate(sysm, run, tr1.rho, k, rho_prev=tr1.rho_prev)
    a, b = O.window_propagate(tr1.rho_prev, tr1.rho, S, H0, run.dt, k)
    assert np.max(np.abs(a - trk.rho_prev)) < 1e-11
    assert np.max(np.abs(b - trk.rho)) < 1e-11
    a0, b0 = O.window_propagate(tr1.rho_prev, tr1.rho, S, H0, run.dt, 0)
    assert np.max(np.abs(a0 - tr1.rho_prev)) < 1e-12 and np.max(np.abs(b0 - tr1.rho)) < 1e-12


def test_window_mean_shift_tracks_the_scc_leapfrog_and_the_frozen_shift_drifts():
    # the premise of the learned form: with the SCC Hamiltonian, windows of k steps whose
    # frozen shift is the mean of the plain run's own shifts over the window stay near the
    # plain leapfrog, while windows frozen at their starting shift drift away
    sysm = I.small_flake(16, seed=7)
    run = I.Run(dt=0.2, n_steps=0, scc=True, kick=0.02, kick_dir=np.array([0.6, 0.8, 0.0]),
                kT=I.SCC_KT)
    rho0, gs, S, Sinv = O.setup(sysm, run)
    R = np.asarray(sysm.R, dtype=np.float64)
    S, H0 = O.model_matrices(sysm, R)
    gamma = O.gamma_matrix(sysm, R)
    q0 = O.reference_populations(sysm)
    k, nw = 10, 20
    tr = O.propagate(sysm, run, rho0, 1 + k * nw)
    v = (tr.charges - q0) @ gamma.T                 # eq:hscc shift of every plain step
    tr1 = O.propagate(sysm, run, rho0, 1)
    err = {}
    for mode in ("mean", "frozen"):
        prev, cur = tr1.rho_prev, tr1.rho
        e = []
        for w in range(nw):
            n = 1 + w * k
            vb = v[n:n + k].mean(axis=0) if mode == "mean" else gamma @ (O.mulliken(sysm, cur, S) - q0)
            prev, cur = O.window_propagate(prev, cur, S, O.scc_hamiltonian(sysm, H0, S, vb),
                                           run.dt, k)
            e.append(np.max(np.abs(O.mulliken(sysm, cur, S) - tr.charges[n + k])))
        err[mode] = np.array(e)
    assert np.max(err["mean"]) < 0.01
    assert err["frozen"][-1] > 20 * err["mean"][-1]


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -3.3, 1e-3])
    r = O.bf16_round(x)
    assert r[0] == 1.0 and r[1] == 1.0                      # tie to even
    assert r[2] == 1.0 + 2.0 ** -6                          # tie to even (up)
    assert np.all(np.abs(r - x) <= np.abs(x) * 2.0 ** -8)


def test_shiftnet_gradient_matches_central_differences():
    rng = np.random.default_rng(5)
    F, H, n = 7, 9, 40
    npar = F * H + H + H * H + H + H + 1
    p = rng.normal(size=npar) * 0.4
    X = rng.normal(size=(n, F))
    Y = rng.normal(size=n)
    loss, g = O.shiftnet_loss_grad(p, X, Y, F, H, bf16=False)
    h = 1e-6
    fd = np.empty(npar)
    for i in range(npar):
        e = np.zeros(npar)
        e[i] = h
        fd[i] = (O.shiftnet_loss_grad(p + e, X, Y, F, H, bf16=False)[0]
                 - O.shiftnet_loss_grad(p - e, X, Y, F, H, bf16=False)[0]) / (2 * h)
    assert np.max(np.abs(g - fd)) < 1e-7 * max(1.0, np.max(np.abs(g)))


def test_fitted_repulsion_zeroes_the_initial_virial():
    # oracle/fit_c3_repulsion.py: with A from the fit, the total ground-state force of the
    # unrelaxed cluster (electronic and repulsive, eq:forces at rest, no field) has zero virial
    import dataclasses
    from oracle import fit_c3_repulsion as FIT
    sysm, run = I.cluster_c3(n_atoms=32)
    A = FIT.virial_repulsion(sysm, run)
    s = dataclasses.replace(sysm, rep_A=A)
    R = np.asarray(s.R, dtype=np.float64)
    rho, gs, S, Sinv = O.setup(s, dataclasses.replace(run, field=None, move_nuclei=False))
    S, H0 = O.model_matrices(s, R)
    gamma = O.gamma_matrix(s, R)
    dq = O.mulliken(s, rho, S) - O.reference_populations(s)
    v = O.atom_potential(gamma, dq, R, np.zeros(3), True)
    F = O.forces(s, rho, S, Sinv, O.scc_hamiltonian(s, H0, S, v), gamma, dq, v, R, np.zeros(3), True)
    Rc = R - R.mean(axis=0)
    assert A > 1.0
    assert abs(np.sum(Rc * F)) < 1e-9 * np.sum(np.abs(Rc * F))
