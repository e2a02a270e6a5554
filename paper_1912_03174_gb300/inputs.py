"""Seeded synthetic inputs for the TD-DFTB propagator and for its CPU oracle.

This module only *draws* inputs: geometries, per-species parameters,
initial velocities and run settings.  It holds none of the method's
arithmetic (no Slater-Koster blocks, no gamma, no charges, no propagation);
both the CUDA library and the oracle receive the arrays made here and build
everything else on their own.

The paper's systems (ZnTPP, the nanodiamond/PDI complex, graphene ribbons)
and their Slater-Koster parameter files are not available, so these
generators make systems of the same shape: a short linear chain, a planar
hexagonal flake, and a random close-packed 3-D cluster, with a minimal
s+p valence basis (4 orbitals per atom, Sec. 2.1 "minimal basis of valence
orbitals").  Units are Hartree atomic units throughout.
"""
from __future__ import annotations

from dataclasses import dataclass, field as dc_field
from typing import Optional

import numpy as np

# physical constants in Hartree atomic units
FS = 41.341374575751          # a.u. of time per femtosecond
AMU = 1822.888486             # electron masses per atomic mass unit
KB = 3.166811563e-6           # Hartree per kelvin
C_LIGHT = 137.035999084       # speed of light


@dataclass
class System:
    """A synthetic tight-binding system (the inputs of ``tdb_create``).

    Radial model (the stand-in for the Slater-Koster tables of Sec. 2.1):
    hopping integrals ``eta_k * t0 * exp(-r / lam_H)`` and overlap integrals
    ``-eta_k * s0 * exp(-r / lam_S)`` for k in (ss-sigma, sp-sigma,
    pp-sigma, pp-pi); on-site energies ``eps_s``/``eps_p`` and Hubbard U per
    species; pair repulsion ``rep_A * exp(-r / rep_b)``.
    """
    name: str
    R: np.ndarray                      # (n_atoms, 3) bohr
    species: np.ndarray                # (n_atoms,) int32 in [0, n_species)
    eps_s: np.ndarray                  # (n_species,) Ha
    eps_p: np.ndarray                  # (n_species,) Ha
    hubbard_U: np.ndarray              # (n_species,) Ha
    mass: np.ndarray                   # (n_species,) amu
    n_electrons: float
    orbs_per_atom: int = 4
    t0: float = 4.0
    lam_H: float = 0.8
    s0: float = 0.3
    lam_S: float = 0.9
    eta: np.ndarray = dc_field(default_factory=lambda: np.array([-1.0, 1.0, 1.0, -0.5]))
    rep_A: float = 0.0
    rep_b: float = 0.5
    V: Optional[np.ndarray] = None     # (n_atoms, 3) bohr / a.u. time

    @property
    def n_atoms(self) -> int:
        return int(self.R.shape[0])

    @property
    def n_orb(self) -> int:
        return self.n_atoms * self.orbs_per_atom

    @property
    def n_species(self) -> int:
        return int(self.eps_s.shape[0])


@dataclass
class Field:
    """Laser field E(t) = E0 sin(omega t + phase) f(t) dir (Sec. 3.1, pump pulse).

    envelope: 0 = none (f = 1); 1 = Gaussian exp(-4 ln2 (t - t_center)^2 / fwhm^2);
    2 = sin^2(pi t / fwhm) on [0, fwhm], zero outside.
    """
    E0: float
    omega: float
    phase: float = 0.0
    t_center: float = 0.0
    fwhm: float = 0.0
    dir: np.ndarray = dc_field(default_factory=lambda: np.array([1.0, 0.0, 0.0]))
    envelope: int = 0


@dataclass
class Run:
    """Run settings of one trajectory."""
    dt: float
    n_steps: int
    scc: bool
    move_nuclei: bool = False
    kick: float = 0.0                  # delta-kick strength E0 (a.u.), 0 = none
    kick_dir: np.ndarray = dc_field(default_factory=lambda: np.array([1.0, 0.0, 0.0]))
    field: Optional[Field] = None
    scc_tol: float = 1e-12
    scc_max_iter: int = 400
    kT: float = 0.0                    # electronic temperature of the ground state (Ha)


def _species_params(rng: np.random.Generator, n_species: int, scc: bool):
    eps_s = rng.uniform(-0.5, -0.1, n_species)
    eps_p = rng.uniform(-0.5, -0.1, n_species)
    U = rng.uniform(0.3, 0.5, n_species) if scc else np.zeros(n_species)
    mass = np.full(n_species, 12.0)
    return eps_s, eps_p, U, mass


def chain(n_atoms: int, bond: float, jitter: float, rng: np.random.Generator) -> np.ndarray:
    """Linear chain along x, bonds ``bond +/- U(-jitter, jitter)``, centred."""
    bonds = bond + rng.uniform(-jitter, jitter, max(n_atoms - 1, 0))
    x = np.concatenate([[0.0], np.cumsum(bonds)])
    R = np.zeros((n_atoms, 3))
    R[:, 0] = x - x.mean()
    return R


def hex_flake(n_atoms: int, bond: float, jitter: float, rng: np.random.Generator) -> np.ndarray:
    """Planar honeycomb flake: the ``n_atoms`` lattice sites nearest a hexagon centre.

    Ties in distance are broken by polar angle, then by generation index.
    Every in-plane coordinate gets a U(-jitter, jitter) displacement.
    """
    a1 = bond * np.array([1.5, np.sqrt(3.0) / 2.0])
    a2 = bond * np.array([1.5, -np.sqrt(3.0) / 2.0])
    basis = [np.zeros(2), np.array([bond, 0.0])]
    centre = np.array([-bond, 0.0])
    span = int(np.ceil(np.sqrt(n_atoms))) + 4
    pts = []
    for i in range(-span, span + 1):
        for j in range(-span, span + 1):
            for b in basis:
                pts.append(i * a1 + j * a2 + b - centre)
    pts = np.array(pts)
    d = np.round(np.hypot(pts[:, 0], pts[:, 1]), 9)
    ang = np.round(np.mod(np.arctan2(pts[:, 1], pts[:, 0]), 2 * np.pi), 9)
    order = np.lexsort((np.arange(len(pts)), ang, d))[:n_atoms]
    xy = pts[order] + rng.uniform(-jitter, jitter, (n_atoms, 2))
    R = np.zeros((n_atoms, 3))
    R[:, :2] = xy
    return R


def random_cluster(n_atoms: int, density: float, d_min: float, rng: np.random.Generator) -> np.ndarray:
    """Random sequential insertion in a sphere of number density ``density``.

    Candidates closer than ``d_min`` to an accepted atom are rejected.
    """
    radius = (3.0 * n_atoms / (4.0 * np.pi * density)) ** (1.0 / 3.0)
    R = np.zeros((0, 3))
    tries = 0
    while R.shape[0] < n_atoms:
        tries += 1
        if tries > 10_000_000:
            raise RuntimeError("random_cluster: packing failed")
        p = rng.uniform(-radius, radius, 3)
        if p @ p > radius * radius:
            continue
        if R.shape[0] and np.min(np.sum((R - p) ** 2, axis=1)) < d_min * d_min:
            continue
        R = np.vstack([R, p])
    return R - R.mean(axis=0)


def maxwell_velocities(masses_amu: np.ndarray, T: float, rng: np.random.Generator) -> np.ndarray:
    """Maxwell-Boltzmann velocities at T, centre-of-mass motion removed,
    rescaled to exactly T over 3*n_atoms - 3 degrees of freedom."""
    m = masses_amu * AMU
    n = m.shape[0]
    V = rng.normal(size=(n, 3)) * np.sqrt(KB * T / m)[:, None]
    V -= (m[:, None] * V).sum(axis=0) / m.sum()
    ekin = 0.5 * np.sum(m[:, None] * V * V)
    target = 0.5 * (3 * n - 3) * KB * T
    return V * np.sqrt(target / ekin)


# ---------------------------------------------------------------------------
# Named workloads.  Seeds are 1000 + k for the k-th workload below.
# ---------------------------------------------------------------------------

# Electronic temperature (Ha) of SCC ground states.  The synthetic flakes and
# clusters are metallic (HOMO-LUMO gaps of ~1e-4 Ha), and integer occupations
# make the charge self-consistency slosh; Fermi smearing at ~950 K settles it.
SCC_KT = 0.003

def chain_c1(seed: int = 1001, n_atoms: int = 10):
    """Non-SCC frozen-nuclei chain: 10 atoms x 4 orbitals (N = 40), 20 electrons,
    bonds 2.6 +/- 0.05 bohr, kick 1e-4 a.u. along x, dt = 0.1, 1000 steps."""
    rng = np.random.default_rng(seed)
    R = chain(n_atoms, 2.6, 0.05, rng)
    eps_s, eps_p, U, mass = _species_params(rng, 1, scc=False)
    species = np.zeros(n_atoms, np.int32)
    sysm = System(f"chain{n_atoms}", R, species, eps_s, eps_p, U, mass,
                  n_electrons=2.0 * n_atoms)
    run = Run(dt=0.1, n_steps=1000, scc=False, kick=1e-4)
    return sysm, run


def flake_c2(seed: int = 1002, n_atoms: int = 256):
    """SCC frozen-nuclei hexagonal flake: 256 atoms (N = 1024), bonds 2.68 bohr
    +/- 0.02 in-plane jitter, Hubbard U ~ U(0.3, 0.5), half filling,
    kick 1e-3 a.u. along x, dt = 0.2, 20000 steps."""
    rng = np.random.default_rng(seed)
    R = hex_flake(n_atoms, 2.68, 0.02, rng)
    eps_s, eps_p, U, mass = _species_params(rng, 1, scc=True)
    species = np.zeros(n_atoms, np.int32)
    sysm = System(f"flake{n_atoms}", R, species, eps_s, eps_p, U, mass,
                  n_electrons=4.0 * n_atoms)
    run = Run(dt=0.2, n_steps=20000, scc=True, kick=1e-3, kT=SCC_KT)
    return sysm, run


def cluster_c3(seed: int = 1003, n_atoms: int = 512):
    """Ehrenfest cluster: 512 atoms (N = 2048) by random insertion at
    0.02 bohr^-3 with a 2.4 bohr minimum distance, 12 amu, 300 K Maxwell
    velocities; SCC; Gaussian-envelope laser E0 = 0.01, omega = 0.1 Ha,
    FWHM 10 fs centred at 20 fs, along x; dt = 0.2, 10000 steps.  Pair repulsion
    A exp(-r / 0.5) with A fitted to zero initial virial (the 512-atom workload)."""
    rng = np.random.default_rng(seed)
    R = random_cluster(n_atoms, 0.02, 2.4, rng)
    eps_s, eps_p, U, mass = _species_params(rng, 1, scc=True)
    species = np.zeros(n_atoms, np.int32)
    V = maxwell_velocities(mass[species], 300.0, rng)
    # pair repulsion amplitude fitted once to zero initial virial of the 512-atom cluster
    # (oracle/fit_c3_repulsion.py); without it the unrelaxed cluster collapses
    rep_A = 66.78242917 if (n_atoms == 512 and seed == 1003) else 1.0
    sysm = System(f"cluster{n_atoms}", R, species, eps_s, eps_p, U, mass,
                  n_electrons=4.0 * n_atoms, rep_A=rep_A, rep_b=0.5, V=V)
    fwhm = 10.0 * FS
    fld = Field(E0=0.01, omega=0.1, phase=0.0, t_center=2.0 * fwhm, fwhm=fwhm, envelope=1)
    run = Run(dt=0.2, n_steps=10000, scc=True, move_nuclei=True, field=fld, kT=SCC_KT)
    return sysm, run


def pump_probe_c4(seed: int = 1004, n_traj: int = 256, sizes=(32, 64, 128, 256)):
    """Batched pump-probe scan: four flakes by the flake rule (32/64/128/256 atoms,
    N = 128..1024), SCC, frozen nuclei, dt = 0.2; the pump is the c3 laser (Gaussian,
    E0 = 0.01, omega = 0.1 Ha, FWHM 10 fs centred at 20 fs, along x), the probe a
    1e-3 a.u. kick along x at delay tau; each of n_traj trajectories draws a size
    uniformly and tau ~ U(0, 200 fs); 5000 post-kick steps.  Returns (systems, run,
    size index per trajectory, tau in a.u. per trajectory); run.kick is the probe
    strength (applied at tau, not at t = 0)."""
    rng = np.random.default_rng(seed)
    systems = []
    for k, n in enumerate(sizes):
        R = hex_flake(n, 2.68, 0.02, rng)
        eps_s, eps_p, U, mass = _species_params(rng, 1, scc=True)
        systems.append(System(f"flake{n}", R, np.zeros(n, np.int32), eps_s, eps_p, U, mass,
                              n_electrons=4.0 * n))
    fwhm = 10.0 * FS
    fld = Field(E0=0.01, omega=0.1, phase=0.0, t_center=2.0 * fwhm, fwhm=fwhm, envelope=1)
    run = Run(dt=0.2, n_steps=5000, scc=True, kick=1e-3, field=fld, kT=SCC_KT)
    which = rng.integers(0, len(sizes), n_traj)
    tau = rng.uniform(0.0, 200.0 * FS, n_traj)
    return systems, run, which, tau


def small_flake(n_atoms: int, seed: int, scc: bool = True, jitter: float = 0.02, n_species: int = 1):
    """A flake built by the flake rule at any size (tests: several tiles plus a ragged tail)."""
    rng = np.random.default_rng(seed)
    R = hex_flake(n_atoms, 2.68, jitter, rng)
    eps_s, eps_p, U, mass = _species_params(rng, n_species, scc=scc)
    species = rng.integers(0, n_species, n_atoms).astype(np.int32)
    return System(f"flake{n_atoms}", R, species, eps_s, eps_p, U, mass,
                  n_electrons=4.0 * n_atoms)


def small_cluster(n_atoms: int, seed: int, T: float = 300.0, rep_A: float = 1.0, n_species: int = 1):
    """A small 3-D cluster with Maxwell velocities (Ehrenfest tests)."""
    rng = np.random.default_rng(seed)
    R = random_cluster(n_atoms, 0.02, 2.4, rng)
    eps_s, eps_p, U, mass = _species_params(rng, n_species, scc=True)
    species = rng.integers(0, n_species, n_atoms).astype(np.int32)
    V = maxwell_velocities(mass[species], T, rng) if n_atoms > 1 else np.zeros((1, 3))
    return System(f"cluster{n_atoms}", R, species, eps_s, eps_p, U, mass,
                  n_electrons=4.0 * n_atoms, rep_A=rep_A, rep_b=0.5, V=V)


def two_level(separation: float, hop: float):
    """Two sites x one s orbital along x with S = I (s0 = 0) and hopping -hop
    between them: the driven two-level system of the Rabi check."""
    R = np.array([[-separation / 2, 0.0, 0.0], [separation / 2, 0.0, 0.0]])
    lam = 0.8
    t0 = hop * np.exp(separation / lam)
    return System("two_level", R, np.zeros(2, np.int32), np.array([0.0]), np.array([0.0]),
                  np.array([0.0]), np.array([12.0]), n_electrons=2.0, orbs_per_atom=1,
                  t0=t0, lam_H=lam, s0=0.0)
