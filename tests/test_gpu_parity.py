"""Parity of the CUDA propagator (through the C ABI) with the FP64 CPU oracle.

Tolerances.  The FP64 form differs from the oracle only in summation order
(~1e-16 relative per operation), so after hundreds of steps of a bounded
oscillation the dipole, the charges and rho agree to ~1e-12; the tests allow
1e-10 (rho, charges) and 1e-10 a.u. (dipole), four orders under the 1e-6 a.u.
dipole target.  The reduced-precision forms act on rho - rho_gs with FP32
products: their error is ~1e-7 relative to |rho - rho_gs| per step, and the
tests hold them to the 1e-6 a.u. dipole target.
"""
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


def _gpu_run(B, sysm, run, n, precision="fp64"):
    with B.Propagator(sysm, run, precision) as p:
        it, res = p.setup()
        rho0 = B.tdb_get_rho(p.ctx)
        p.step(n)
        hist = B.tdb_dipole_history(p.ctx, n)
        obs = p.observables()
        rho, prev = B.tdb_get_rho(p.ctx, prev=True)
    return dict(it=it, res=res, rho0=rho0, hist=hist, obs=obs, rho=rho, prev=prev)


def _oracle(sysm, run, n):
    rho, gs, S, Sinv = O.setup(sysm, run)
    tr = O.propagate(sysm, run, rho, n)
    return rho, gs, tr


def _compare(g, rho0, tr, n, tol_rho=1e-10, tol_mu=1e-10):
    assert np.max(np.abs(g["rho0"] - rho0)) < tol_rho
    mu = np.vstack([g["hist"], g["obs"]["dipole"][None, :]])
    assert mu.shape == tr.dipole.shape
    err_mu = np.max(np.abs(mu - tr.dipole))
    assert err_mu < tol_mu, err_mu
    assert np.max(np.abs(g["obs"]["charges"] - tr.charges[-1])) < tol_rho * 10
    assert np.max(np.abs(g["rho"] - tr.rho)) < tol_rho
    assert np.max(np.abs(g["prev"] - tr.rho_prev)) < tol_rho
    return err_mu


def test_c1_chain_full_run_matches_oracle(B):
    sysm, run = I.chain_c1()
    g = _gpu_run(B, sysm, run, run.n_steps)
    rho0, gs, tr = _oracle(sysm, run, run.n_steps)
    _compare(g, rho0, tr, run.n_steps)
    # Tr(rho S) exact and rho exactly Hermitian on the device
    assert abs(g["obs"]["trace_re"] - sysm.n_electrons) / sysm.n_electrons < 1e-12
    assert g["obs"]["herm_err"] == 0.0


@pytest.mark.parametrize("n_atoms,n_species,seed", [(10, 1, 3), (22, 2, 5), (33, 1, 8)])
def test_scc_flakes_match_oracle(B, n_atoms, n_species, seed):
    # N = 40, 88, 132: several 32-tiles and 64-GEMM tiles plus ragged tails
    sysm = I.small_flake(n_atoms, seed=seed, n_species=n_species)
    run = I.Run(dt=0.2, n_steps=0, scc=True, kick=1e-2, kT=I.SCC_KT)
    n = 300
    g = _gpu_run(B, sysm, run, n)
    rho0, gs, tr = _oracle(sysm, run, n)
    _compare(g, rho0, tr, n)
    assert g["it"] >= 1 and g["res"] <= run.scc_tol


def test_laser_field_matches_oracle(B):
    sysm = I.small_flake(16, seed=12, n_species=2)
    fld = I.Field(E0=0.02, omega=0.3, phase=0.3, t_center=20.0, fwhm=15.0, envelope=1,
                  dir=np.array([0.6, 0.8, 0.0]))
    run = I.Run(dt=0.2, n_steps=0, scc=True, kick=0.0, field=fld, kT=I.SCC_KT)
    n = 400
    g = _gpu_run(B, sysm, run, n)
    rho0, gs, tr = _oracle(sysm, run, n)
    _compare(g, rho0, tr, n)
    assert abs(g["obs"]["E_ext"]) > 0


def test_orbs_per_atom_one_and_two_level_system(B):
    sysm = I.two_level(2.0, 0.25)
    fld = I.Field(E0=1e-2, omega=0.5, phase=np.pi / 2, envelope=0)
    run = I.Run(dt=0.2, n_steps=0, scc=False, field=fld)
    g = _gpu_run(B, sysm, run, 500)
    rho0, gs, tr = _oracle(sysm, run, 500)
    _compare(g, rho0, tr, 500)


def test_observables_energy_terms_match_oracle(B):
    sysm = I.small_flake(12, seed=4, n_species=2)
    run = I.Run(dt=0.2, n_steps=0, scc=True, kick=5e-2, kT=I.SCC_KT)
    n = 100
    g = _gpu_run(B, sysm, run, n)
    rho0, gs, tr = _oracle(sysm, run, n)
    assert abs(g["obs"]["E_total"] - tr.energy[-1]) < 1e-10
    assert abs(g["obs"]["trace_re"] - sysm.n_electrons) < 1e-11
    assert abs(g["obs"]["trace_im"]) < 1e-12
    assert g["obs"]["step"] == n and abs(g["obs"]["t"] - n * run.dt) < 1e-12


def test_checkpoint_resume_is_bitwise(B):
    sysm = I.small_flake(12, seed=6)
    run = I.Run(dt=0.2, n_steps=0, scc=True, kick=1e-2, kT=I.SCC_KT)
    with B.Propagator(sysm, run) as a, B.Propagator(sysm, run) as b:
        a.setup()
        b.setup()
        a.step(37)
        blob = B.tdb_get_state(a.ctx)
        B.tdb_set_state(b.ctx, blob)
        a.step(50)
        b.step(50)
        ra = B.tdb_get_rho(a.ctx)
        rb = B.tdb_get_rho(b.ctx)
        assert np.array_equal(ra, rb)
        oa, ob = a.observables(), b.observables()
        assert np.array_equal(oa["dipole"], ob["dipole"]) and oa["step"] == ob["step"] == 87


def test_replicas_are_bitwise_identical(B):
    sysm = I.small_flake(20, seed=9)
    run = I.Run(dt=0.2, n_steps=0, scc=True, kick=1e-2, kT=I.SCC_KT)
    out = []
    for _ in range(2):
        with B.Propagator(sysm, run) as p:
            p.setup()
            p.step(120)
            out.append(B.tdb_get_rho(p.ctx))
    assert np.array_equal(out[0], out[1])


def test_error_paths(B):
    sysm, run = I.chain_c1()
    with B.Propagator(sysm, run) as p:
        with pytest.raises(B.TdbError) as e:
            p.step(1)                       # before the ground state
        assert e.value.status == 2
        p.setup()
        with pytest.raises(B.TdbError) as e:
            B.tdb_step(p.ctx, -1)
        assert e.value.status == 1
    bad = I.Run(dt=5.0, n_steps=0, scc=False)   # dt * spectral width >> 0.9
    with B.Propagator(sysm, bad) as p:
        p.setup()
        with pytest.raises(B.TdbError) as e:
            p.step(1)
        assert e.value.status == 6
    s2 = I.small_flake(4, seed=1)
    s2.species = np.array([0, 0, 0, 5], np.int32)
    with pytest.raises(B.TdbError) as e:
        B.tdb_create(s2, B.make_params(run))
    assert e.value.status == 1
    md = I.Run(dt=0.2, n_steps=0, scc=True, move_nuclei=True)
    with pytest.raises(B.TdbError) as e:      # moving nuclei: FP64, FP64_SLICED and FP32 only
        B.tdb_create(I.small_cluster(6, seed=1), B.make_params(md, "fp16x6"))
    assert e.value.status == 10


def test_invariant_monitor_flags_a_corrupted_state(B):
    # a state blob with a scaled density (host-made fault, no device fault)
    sysm = I.small_flake(10, seed=2)
    run = I.Run(dt=0.2, n_steps=0, scc=True, kick=1e-2, kT=I.SCC_KT)
    with B.Propagator(sysm, run) as p:
        p.setup()
        p.step(5)
        B.tdb_check(p.ctx, 1e-10)
        blob = bytearray(B.tdb_get_state(p.ctx))
        hdr = len(blob) - 4 * 8 * sysm.n_orb ** 2 - 6 * 8 * sysm.n_atoms
        arr = np.frombuffer(bytes(blob[hdr:hdr + 4 * 8 * sysm.n_orb ** 2]), dtype=np.float64).copy()
        arr *= 1.01
        blob[hdr:hdr + arr.nbytes] = arr.tobytes()
        B.tdb_set_state(p.ctx, bytes(blob))
        with pytest.raises(B.TdbError) as e:
            B.tdb_check(p.ctx, 1e-10)
        assert e.value.status == 7
        with pytest.raises(B.TdbError):
            p.step(1)                       # sticky after a numeric error
        p.observables()                     # still readable


_C2_ORACLE = {}


@pytest.mark.parametrize("form,tol", [("fp64", 1e-10), ("fp16x6", 1e-6)])
def test_c2_flake_full_size_prefix(B, form, tol):
    # the N = 1024 SCC flake at its full size, in the bench's launch configuration (FP16X6:
    # 176-wide X tiles, the width the tuner picks there): a 12-step prefix against the oracle
    # (the oracle run is shared by both forms)
    sysm, run = I.flake_c2()
    n = 12
    if form == "fp16x6":
        with B.Propagator(sysm, run, form) as p:
            B.tdb_set_x_tile(p.ctx, 176)
            p.setup()
            rho0 = B.tdb_get_rho(p.ctx)
            p.step(n)
            g = dict(rho0=rho0, hist=B.tdb_dipole_history(p.ctx, n), obs=p.observables())
            g["rho"], g["prev"] = B.tdb_get_rho(p.ctx, prev=True)
    else:
        g = _gpu_run(B, sysm, run, n)
    if not _C2_ORACLE:
        _C2_ORACLE["r"] = _oracle(sysm, run, n)
    rho0, gs, tr = _C2_ORACLE["r"]
    _compare(g, rho0, tr, n, tol_rho=tol, tol_mu=tol)


# reduced-precision forms: (form, dipole tolerance in a.u., rho tolerance)
# fp64s: integer-slice products carry ~7 2^-42 K max|M| max|rho| per product, which over
# 500 steps reaches a few 1e-9 in the dipole (the FP64 form stays at ~1e-12)
REDUCED = [("fp32", 1e-6, 1e-6), ("fp16x6", 1e-6, 1e-6), ("fp16x3", 1e-5, 1e-5),
           ("bf16x3", 2e-5, 2e-5), ("fp64s", 2e-8, 2e-8)]


@pytest.mark.parametrize("form,tol_mu,tol_rho", REDUCED)
@pytest.mark.parametrize("n_atoms", [10, 33, 64, 130])
def test_reduced_precision_forms_match_oracle(B, n_atoms, form, tol_mu, tol_rho):
    # N = 40, 132, 256, 520: one tile, ragged tails (132 is not a multiple of 64), several
    # tiles, 256-wide X tiles with a ragged tail (520 = 2 x 256 + 8)
    sysm = I.small_flake(n_atoms, seed=8)
    run = I.Run(dt=0.2, n_steps=0, scc=True, kick=1e-3, kT=I.SCC_KT)
    n = 500
    g = _gpu_run(B, sysm, run, n, form)
    rho0, gs, tr = _oracle(sysm, run, n)
    mu = np.vstack([g["hist"], g["obs"]["dipole"][None, :]])
    err = np.max(np.abs(mu - tr.dipole))
    assert err < tol_mu, err
    assert np.max(np.abs(g["rho"] - tr.rho)) < tol_rho
    assert abs(g["obs"]["trace_re"] - sysm.n_electrons) / sysm.n_electrons < 1e-10
    assert g["obs"]["herm_err"] == 0.0


_ORACLE_920 = {}


@pytest.mark.parametrize("form,tol_mu,tol_rho", [("fp16x6", 1e-6, 1e-6), ("bf16x3", 2e-5, 2e-5)])
def test_reduced_forms_with_176_wide_x_tiles_match_oracle(B, form, tol_mu, tol_rho):
    # 230 atoms, N = 920: the X products run in 128 x 176 tiles (six column tiles, the
    # last one 40 columns wide, its TMA box reaching past the matrix)
    sysm = I.small_flake(230, seed=8)
    run = I.Run(dt=0.2, n_steps=0, scc=True, kick=1e-3, kT=I.SCC_KT)
    n = 40
    if "tr" not in _ORACLE_920:
        _ORACLE_920["tr"] = _oracle(sysm, run, n)[2]
    tr = _ORACLE_920["tr"]
    g = _gpu_run(B, sysm, run, n, form)
    mu = np.vstack([g["hist"], g["obs"]["dipole"][None, :]])
    err = np.max(np.abs(mu - tr.dipole))
    assert err < tol_mu, err
    assert np.max(np.abs(g["rho"] - tr.rho)) < tol_rho
    assert np.max(np.abs(g["obs"]["charges"] - tr.charges[-1])) < tol_rho
    assert abs(g["obs"]["trace_re"] - sysm.n_electrons) / sysm.n_electrons < 1e-10
    assert g["obs"]["herm_err"] == 0.0


@pytest.mark.parametrize("form", ["fp32", "fp16x6", "bf16x3"])
def test_reduced_form_checkpoint_resume_is_bitwise(B, form):
    # the state of a reduced form carries its FP32-pair master and scale bookkeeping
    sysm = I.small_flake(33, seed=6)
    run = I.Run(dt=0.2, n_steps=0, scc=True, kick=1e-3, kT=I.SCC_KT)
    with B.Propagator(sysm, run, form) as a, B.Propagator(sysm, run, form) as b:
        a.setup()
        b.setup()
        a.step(37)
        B.tdb_set_state(b.ctx, B.tdb_get_state(a.ctx))
        a.step(50)
        b.step(50)
        assert B.tdb_get_state(a.ctx) == B.tdb_get_state(b.ctx)
        oa, ob = a.observables(), b.observables()
        assert np.array_equal(oa["dipole"], ob["dipole"]) and oa["step"] == ob["step"] == 87


@pytest.mark.parametrize("form,tol", [("fp16x6", 5e-7), ("fp16x3", 5e-5)])
def test_reduced_forms_at_n2048_track_the_fp64_form(B, form, tol):
    # N = 2048 (512-atom flake): the X products run as two K slices of 1024 and delta M
    # keeps two exact head accumulators; the FP64 form is the reference (it matches the
    # oracle at N = 1024 and below)
    sysm = I.small_flake(512, seed=12)
    run = I.Run(dt=0.2, n_steps=0, scc=True, kick=1e-3, kT=I.SCC_KT)
    n = 300
    ref = _gpu_run(B, sysm, run, n, "fp64")
    g = _gpu_run(B, sysm, run, n, form)
    err = np.max(np.abs(g["hist"] - ref["hist"]))
    assert err < tol, err
    assert np.max(np.abs(g["rho"] - ref["rho"])) < 10 * tol
    assert g["obs"]["herm_err"] == 0.0
    assert abs(g["obs"]["trace_re"] - sysm.n_electrons) / sysm.n_electrons < 1e-10


@pytest.mark.parametrize("form", ["fp32", "bf16x3", "fp16x3", "fp16x6", "fp64s"])
def test_every_form_conserves_the_electron_number_over_a_long_run(B, form):
    # Sec. 2.3: with S frozen the leapfrog conserves Tr(rho S) = N_e exactly; the reduced
    # products do not, so the reduced forms renormalise the base level of every update to
    # N_e.  130 atoms (N = 520), 2400 steps, Tr(rho S) (FP64 view) sampled every 200 steps.
    sysm = I.small_flake(130, seed=8)
    run = I.Run(dt=0.2, n_steps=0, scc=True, kick=1e-3, kT=I.SCC_KT)
    worst = 0.0
    with B.Propagator(sysm, run, form) as p:
        p.setup()
        for _ in range(12):
            p.step(200)
            o = p.observables(charges=False)
            worst = max(worst, abs(o["trace_re"] - sysm.n_electrons) / sysm.n_electrons)
            assert o["herm_err"] == 0.0
    assert worst < 1e-10, worst


def test_exact_head_form_beats_the_hi_lo_forms(B):
    # the hi/lo forms are limited by the biased tensor-core accumulation; the
    # exact-head form is not
    sysm = I.small_flake(64, seed=8)
    run = I.Run(dt=0.2, n_steps=0, scc=True, kick=1e-3, kT=I.SCC_KT)
    n = 400
    ref = _gpu_run(B, sysm, run, n, "fp64")
    e = {}
    for form in ("fp16x6", "fp16x3", "bf16x3"):
        g = _gpu_run(B, sysm, run, n, form)
        e[form] = np.max(np.abs(g["hist"] - ref["hist"]))
    assert e["fp16x6"] < e["fp16x3"] / 4, e
    assert e["fp16x6"] < e["bf16x3"] / 4, e


# ---------------------------------------------------------------------------
# moving nuclei (Ehrenfest, eq:forces, eq:nac, velocity Verlet)
# ---------------------------------------------------------------------------

def _md_gpu(B, sysm, run, n, precision="fp64"):
    with B.Propagator(sysm, run, precision) as p:
        p.setup()
        p.step(n)
        hist = B.tdb_dipole_history(p.ctx, n)
        obs = p.observables(forces=True)
        rho, prev = B.tdb_get_rho(p.ctx, prev=True)
        blob = B.tdb_get_state(p.ctx)
    nat = sysm.n_atoms
    tail = np.frombuffer(blob[len(blob) - 6 * 8 * nat:], dtype=np.float64)
    return dict(hist=hist, obs=obs, rho=rho, prev=prev, R=tail[:3 * nat].reshape(nat, 3),
                V=tail[3 * nat:].reshape(nat, 3))


@pytest.mark.parametrize("n_atoms,seed,laser", [(6, 23, False), (12, 5, True), (33, 7, False)])
def test_ehrenfest_matches_oracle(B, n_atoms, seed, laser):
    sysm = I.small_cluster(n_atoms, seed=seed, T=3000.0)
    fld = I.Field(E0=0.01, omega=0.1, phase=0.2, t_center=20.0, fwhm=20.0, envelope=1) if laser else None
    run = I.Run(dt=0.2, n_steps=0, scc=True, move_nuclei=True, kick=1e-2 if not laser else 0.0,
                field=fld, kT=I.SCC_KT)
    n = 200
    g = _md_gpu(B, sysm, run, n)
    rho0, gs, S, Sinv = O.setup(sysm, run)
    tr = O.propagate(sysm, run, rho0, n, keep_forces=True)
    mu = np.vstack([g["hist"], g["obs"]["dipole"][None, :]])
    assert np.max(np.abs(mu - tr.dipole)) < 1e-9
    assert np.max(np.abs(g["R"] - tr.R)) < 1e-9
    assert np.max(np.abs(g["V"] - tr.V)) < 1e-12
    assert np.max(np.abs(g["obs"]["forces"] - tr.forces[-1])) < 1e-9
    assert np.max(np.abs(g["obs"]["charges"] - tr.charges[-1])) < 1e-9
    assert np.max(np.abs(g["rho"] - tr.rho)) < 1e-9
    assert abs(g["obs"]["E_total"] - tr.energy[-1]) < 1e-9
    assert abs(g["obs"]["work"] - tr.work[-1]) < 1e-10
    assert abs(g["obs"]["trace_re"] - tr.trace[-1].real) < 1e-10
    assert g["obs"]["herm_err"] == 0.0


@pytest.mark.parametrize("n_atoms,seed,laser", [(12, 5, True), (33, 7, False)])
def test_ehrenfest_fp64_sliced_form_matches_oracle(B, n_atoms, seed, laser):
    # integer-slice products (S^-1 H, M rho, S^-1 D, Y rho), FP64 everything else
    sysm = I.small_cluster(n_atoms, seed=seed, T=3000.0)
    fld = I.Field(E0=0.01, omega=0.1, phase=0.2, t_center=20.0, fwhm=20.0, envelope=1) if laser else None
    run = I.Run(dt=0.2, n_steps=0, scc=True, move_nuclei=True, kick=1e-2 if not laser else 0.0,
                field=fld, kT=I.SCC_KT)
    n = 200
    g = _md_gpu(B, sysm, run, n, "fp64s")
    rho0, gs, S, Sinv = O.setup(sysm, run)
    tr = O.propagate(sysm, run, rho0, n, keep_forces=True)
    mu = np.vstack([g["hist"], g["obs"]["dipole"][None, :]])
    err = dict(mu=np.max(np.abs(mu - tr.dipole)), R=np.max(np.abs(g["R"] - tr.R)),
               F=np.max(np.abs(g["obs"]["forces"] - tr.forces[-1])),
               rho=np.max(np.abs(g["rho"] - tr.rho)))
    assert err["mu"] < 1e-8 and err["R"] < 1e-9 and err["F"] < 1e-8 and err["rho"] < 1e-8, err
    assert abs(g["obs"]["work"] - tr.work[-1]) < 1e-9, err
    assert g["obs"]["herm_err"] == 0.0


def test_ehrenfest_fp32_form_tracks_the_oracle(B):
    # FP32 products (M = S^-1 H, X = M rho, Y = S^-1 D, Z = Y rho) with the FP64
    # density, forces and update
    sysm = I.small_cluster(33, seed=7, T=3000.0)
    run = I.Run(dt=0.2, n_steps=0, scc=True, move_nuclei=True, kick=1e-2, kT=I.SCC_KT)
    n = 200
    g = _md_gpu(B, sysm, run, n, "fp32")
    rho0, gs, S, Sinv = O.setup(sysm, run)
    tr = O.propagate(sysm, run, rho0, n, keep_forces=True)
    mu = np.vstack([g["hist"], g["obs"]["dipole"][None, :]])
    err = dict(mu=np.max(np.abs(mu - tr.dipole)), R=np.max(np.abs(g["R"] - tr.R)),
               F=np.max(np.abs(g["obs"]["forces"] - tr.forces[-1])),
               rho=np.max(np.abs(g["rho"] - tr.rho)))
    assert err["mu"] < 1e-5 and err["R"] < 1e-7 and err["F"] < 1e-4 and err["rho"] < 1e-5, err
    assert abs(g["obs"]["trace_re"] - tr.trace[-1].real) < 1e-6, err
    assert g["obs"]["herm_err"] == 0.0


def test_ehrenfest_energy_balance_on_gpu(B):
    # E - int P dt stays constant to O(dt^2) on the device too (the oracle's pin, GPU form)
    sysm = I.small_cluster(8, seed=29, T=3000.0)
    run = I.Run(dt=0.1, n_steps=0, scc=True, move_nuclei=True, kick=1e-2, kT=I.SCC_KT)
    bal = []
    with B.Propagator(sysm, run, "fp64") as p:
        p.setup()
        for _ in range(8):
            o = p.observables()
            bal.append(o["E_total"] - o["work"])
            p.step(100)
    assert np.max(np.abs(np.array(bal) - bal[0])) < 1e-6


def test_ehrenfest_checkpoint_resume_is_bitwise(B):
    sysm = I.small_cluster(10, seed=3, T=1000.0)
    run = I.Run(dt=0.2, n_steps=0, scc=True, move_nuclei=True, kick=1e-2, kT=I.SCC_KT)
    with B.Propagator(sysm, run) as a, B.Propagator(sysm, run) as b:
        a.setup()
        b.setup()
        a.step(23)
        B.tdb_set_state(b.ctx, B.tdb_get_state(a.ctx))
        a.step(40)
        b.step(40)
        assert np.array_equal(B.tdb_get_rho(a.ctx), B.tdb_get_rho(b.ctx))
        assert B.tdb_get_state(a.ctx) == B.tdb_get_state(b.ctx)


def test_a_bounded_device_wait_that_runs_out_makes_the_context_sticky(B):
    # failure detection without a GPU fault: a kernel waits on an mbarrier that nothing
    # arrives on, gives up after a bounded number of polls and records a time-out; the host
    # reads TDB_ERR_TIMEOUT at its next synchronising call, after which only observables,
    # state reads and destroy are allowed -- and the GPU stays usable
    sysm = I.small_flake(10, seed=3)
    run = I.Run(dt=0.2, n_steps=0, scc=True, kick=1e-3, kT=I.SCC_KT)
    with B.Propagator(sysm, run, "fp16x6") as p:
        p.setup()
        p.step(5)
        B.tdb_wait_probe(p.ctx, 1000)
        with pytest.raises(B.TdbError) as e:
            p.observables()
        assert e.value.status == 8
        with pytest.raises(B.TdbError) as e:
            p.step(1)
        assert e.value.status == 2
        o = p.observables()            # allowed on a sticky context
        assert o["step"] == 5
        assert len(B.tdb_get_state(p.ctx)) > 0
    # a fresh context on the same device works normally
    with B.Propagator(sysm, run, "fp16x6") as p:
        p.setup()
        p.step(5)
        assert p.observables()["step"] == 5


def test_the_x_tile_width_changes_the_time_not_the_result(B):
    # every output element of the X product keeps its order of accumulation whatever the
    # tile width, so trajectories with 128-, 176- and 256-wide tiles agree bit for bit
    sysm = I.small_flake(256, seed=7)
    run = I.Run(dt=0.2, n_steps=0, scc=True, kick=1e-3, kT=I.SCC_KT)
    got = {}
    for w in (128, 176, 256, 0):
        with B.Propagator(sysm, run, "fp16x6") as p:
            p.setup()
            B.tdb_set_x_tile(p.ctx, w)
            assert B.tdb_x_tile(p.ctx) == w
            p.step(40)
            if w == 0:
                assert B.tdb_x_tile(p.ctx) in (128, 176, 256)   # tuned at the first steps
            got[w] = (B.tdb_get_rho(p.ctx), B.tdb_dipole_history(p.ctx, 40))
    for w in (176, 256, 0):
        assert np.array_equal(got[w][0], got[128][0])
        assert np.array_equal(got[w][1], got[128][1])
    with B.Propagator(sysm, run, "fp16x6") as p:
        for bad in (64, 100, -1):
            with pytest.raises(B.TdbError) as e:
                B.tdb_set_x_tile(p.ctx, bad)
            assert e.value.status == 1
    with B.Propagator(I.small_flake(10, seed=3), run, "fp64") as p:
        with pytest.raises(B.TdbError) as e:
            B.tdb_set_x_tile(p.ctx, 128)
        assert e.value.status == 10
        assert B.tdb_x_tile(p.ctx) == -1
