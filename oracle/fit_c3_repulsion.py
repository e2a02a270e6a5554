"""Fit the pair-repulsion amplitude of the Ehrenfest cluster workload (c3) with the oracle.

TEST INFRASTRUCTURE.  Run once (``python oracle/fit_c3_repulsion.py``); it prints the value
that ``paper_1912_03174_gb300/inputs.py`` carries as a literal for the 512-atom cluster.

The synthetic two-centre model has no fitted repulsive potential (the paper's Slater-Koster
sets are not available), so E_rep = A sum_{A<B} exp(-r/b), b = 0.5 bohr, takes its amplitude
from the condition that the initial geometry is under no net pressure: the total virial
sum_A (R_A - R_c) . F_A of the ground-state Ehrenfest forces (eq:forces; at rest the
velocity terms vanish, no field) is zero.  The electronic forces do not depend on A, and the
repulsive force is linear in A, so A = -W_el / W_rep(A = 1).  Without it (A = 1) the
unrelaxed random cluster collapses under its bonding forces within a few hundred steps.
"""
from __future__ import annotations

import dataclasses
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import tdb_oracle as O  # noqa: E402
from paper_1912_03174_gb300 import inputs as I  # noqa: E402


def virial_repulsion(sysm, run) -> float:
    """A with sum_A (R_A - R_c) . F_A = 0 at the ground state of sysm (E_rep = A exp(-r/rep_b))."""
    s0 = dataclasses.replace(sysm, rep_A=0.0)
    R = np.asarray(s0.R, dtype=np.float64)
    rho, gs, S, Sinv = O.setup(s0, dataclasses.replace(run, field=None, move_nuclei=False))
    S, H0 = O.model_matrices(s0, R)
    gamma = O.gamma_matrix(s0, R)
    dq = O.mulliken(s0, rho, S) - O.reference_populations(s0)
    v = O.atom_potential(gamma, dq, R, np.zeros(3), True)
    H = O.scc_hamiltonian(s0, H0, S, v)
    F_el = O.forces(s0, rho, S, Sinv, H, gamma, dq, v, R, np.zeros(3), True)
    iA, iB = O.pair_list(R.shape[0])
    d = R[iA] - R[iB]
    r = np.linalg.norm(d, axis=1)
    fr = (np.exp(-r / s0.rep_b) / s0.rep_b)[:, None] * d / r[:, None]
    F_rep = np.zeros_like(R)
    np.add.at(F_rep, iA, fr)
    np.add.at(F_rep, iB, -fr)
    Rc = R - R.mean(axis=0)
    return -float(np.sum(Rc * F_el)) / float(np.sum(Rc * F_rep))


if __name__ == "__main__":
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 512
    sysm, run = I.cluster_c3(n_atoms=n)
    print(f"cluster of {n} atoms: rep_A = {virial_repulsion(sysm, run):.10g}")
