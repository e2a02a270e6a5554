"""The learned form on the GPU: the shift network's forward pass and gradient against the
oracle, Adam training, the closed-form window against the oracle's window, and the gain
of the trained network over windows with the shift frozen at the window's start."""
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


def _random_params(rng, F, H, scale=0.5):
    return (rng.normal(size=F * H + 3 * H + H * H + 1) * scale).astype(np.float32)


@pytest.mark.parametrize("F,H,n", [(8, 32, 1000), (16, 64, 300), (1, 1, 5), (32, 17, 129)])
def test_shiftnet_forward_and_gradient_match_the_oracle(B, F, H, n):
    # n spans several 128-sample blocks with a ragged tail (and a single partial block)
    rng = np.random.default_rng(F * 100 + H)
    p = _random_params(rng, F, H)
    X = rng.normal(size=(n, F)).astype(np.float32)
    Y = rng.normal(size=n).astype(np.float32)
    with B.ShiftNet(F, H, seed=1) as net:
        assert net.n_params == p.size
        net.set_params(p)
        assert np.array_equal(net.params(), p)
        y = net.predict(X)
        y_ref = O.shiftnet_forward(p.astype(np.float64), X.astype(np.float64), F, H, bf16=True)[0]
        # FP32 sums of at most 64 terms of size <= ~10 against FP64
        np.testing.assert_allclose(y, y_ref, rtol=0, atol=2e-5 * max(1.0, np.max(np.abs(y_ref))))
        loss, g = net.gradient(X, Y)
        l_ref, g_ref = O.shiftnet_loss_grad(p.astype(np.float64), X.astype(np.float64),
                                            Y.astype(np.float64), F, H, bf16=True)
        assert loss == pytest.approx(l_ref, rel=1e-5)
        np.testing.assert_allclose(g, g_ref, rtol=0, atol=2e-5 * np.max(np.abs(g_ref)))


def test_shiftnet_adam_step_matches_numpy_adam_on_the_oracle_gradient(B):
    rng = np.random.default_rng(2)
    F, H, n = 8, 32, 512
    p = _random_params(rng, F, H)
    X = rng.normal(size=(n, F)).astype(np.float32)
    Y = rng.normal(size=n).astype(np.float32)
    lr = 1e-3
    with B.ShiftNet(F, H) as net:
        net.set_params(p)
        net.train(X, Y, epochs=1, batch=n, lr=lr)
        q = net.params()
    _, g = O.shiftnet_loss_grad(p.astype(np.float64), X.astype(np.float64), Y.astype(np.float64),
                                F, H, bf16=True)
    # first Adam step: m / sqrt(v) = g / |g| (bias-corrected), so p - lr sign(g) where g is
    # well above the rounding of the FP32 sums
    big = np.abs(g) > 1e-3 * np.max(np.abs(g))
    want = p.astype(np.float64) - lr * g / (np.abs(g) + 1e-8)
    np.testing.assert_allclose(q[big], want[big], rtol=0, atol=1e-6)
    assert np.all(np.abs(q - p) <= lr * 1.001)


def test_shiftnet_training_fits_a_smooth_function(B):
    rng = np.random.default_rng(4)
    F, H, n = 4, 32, 4096
    X = rng.uniform(-1.5, 1.5, size=(n, F)).astype(np.float32)
    Y = (np.sin(2 * X[:, 0]) + 0.5 * X[:, 1] * X[:, 2] - 0.3 * X[:, 3]).astype(np.float32)
    with B.ShiftNet(F, H, seed=3) as net:
        l0, _ = net.gradient(X, Y)
        loss = net.train(X, Y, epochs=150, batch=256, lr=3e-3)
        l1, _ = net.gradient(X, Y)
    assert l1 < 0.02 * l0 and l1 < 5e-3
    # the reported loss is the mean over the last epoch, taken while the weights move
    assert 0 < loss < 10 * l1 + 1e-4


def test_shiftnet_rejects_bad_shapes(B):
    with pytest.raises(B.TdbError):
        B.ShiftNet(33, 8)
    with pytest.raises(B.TdbError):
        B.ShiftNet(4, 65)


def _window_case(B, n_atoms, form, seed):
    sysm = I.small_flake(n_atoms, seed=seed)
    run = I.Run(dt=0.2, n_steps=0, scc=True, kick=0.02, kick_dir=np.array([0.6, 0.8, 0.0]),
                kT=I.SCC_KT)
    return sysm, run, B.Propagator(sysm, run, form)


@pytest.mark.parametrize("n_atoms,form,k", [(16, "fp64", 10), (33, "fp64", 7), (33, "fp64s", 12)])
def test_window_matches_the_oracle_window(B, n_atoms, form, k):
    sysm, run, p = _window_case(B, n_atoms, form, seed=8)
    with p:
        p.setup()
        p.step(5)
        rho, prev = B.tdb_get_rho(p.ctx, prev=True)
        v, dq_gpu = B.tdb_scc_shift(p.ctx, charges=True)
        # the shift of rho_n is gamma dq(rho_n)
        R = np.asarray(sysm.R)
        S, H0 = O.model_matrices(sysm, R)
        gamma = O.gamma_matrix(sysm, R)
        dq = O.mulliken(sysm, rho, S) - O.reference_populations(sysm)
        np.testing.assert_allclose(dq_gpu, dq, rtol=0, atol=1e-12)
        np.testing.assert_allclose(v, gamma @ dq, rtol=0, atol=1e-11)
        v_bar = v + np.random.default_rng(1).normal(size=v.size) * 1e-3
        B.tdb_step_window(p.ctx, v_bar, k)
        rho_w, prev_w = B.tdb_get_rho(p.ctx, prev=True)
        a, b = O.window_propagate(prev, rho, S, O.scc_hamiltonian(sysm, H0, S, v_bar), run.dt, k)
        # FP64 products; in the sliced form integer-slice products (about 2e-12 of
        # K max|A| max|B| each, four in a row)
        tol = 1e-10 if form == "fp64" else 2e-9
        assert np.max(np.abs(prev_w - a)) < tol
        assert np.max(np.abs(rho_w - b)) < tol
        obs = p.observables()
        assert obs["step"] == 5 + k
        assert obs["t"] == pytest.approx((5 + k) * run.dt)
        assert abs(obs["trace_re"] - sysm.n_electrons) < 1e-9
        # the leapfrog continues from the window's two levels
        p.step(3)
        assert p.observables()["step"] == 8 + k


def test_window_argument_and_state_errors(B):
    sysm, run, p = _window_case(B, 10, "fp64", seed=3)
    with p:
        p.setup()
        v = np.zeros(10)
        with pytest.raises(B.TdbError):          # right after the kick: Euler step pending
            B.tdb_step_window(p.ctx, v, 5)
        p.step(1)
        with pytest.raises(B.TdbError):
            B.tdb_step_window(p.ctx, v, 0)
        B.tdb_set_field(p.ctx, I.Field(E0=1e-3, omega=0.3))
        with pytest.raises(B.TdbError):
            B.tdb_step_window(p.ctx, v, 5)
    _, _, q = _window_case(B, 10, "fp16x6", seed=3)
    with q:
        q.setup()
        q.step(1)
        with pytest.raises(B.TdbError):
            B.tdb_step_window(q.ctx, np.zeros(10), 5)


K_WIN, L_HIST = 10, 8


@pytest.fixture(scope="module")
def trained(B):
    """Network trained on shift records of three plain runs (kicks along three directions)
    of a 16-atom flake; the fourth direction is held out."""
    from paper_1912_03174_gb300 import learned as Lrn
    sysm = I.small_flake(16, seed=7)
    rng = np.random.default_rng(0)
    dirs = [d / np.linalg.norm(d) for d in rng.normal(size=(4, 3))]
    Xs, Ys = [], []
    for d in dirs[:3]:
        run = I.Run(dt=0.2, n_steps=0, scc=True, kick=0.02, kick_dir=d, kT=I.SCC_KT)
        with B.Propagator(sysm, run, "fp64") as p:
            p.setup()
            p.step(1)
            X, Y = Lrn.training_set(Lrn.record(p.ctx, 2000), K_WIN, L_HIST)
            Xs.append(X)
            Ys.append(Y)
    model = Lrn.ShiftModel(k=K_WIN, L=L_HIST, hidden=32, seed=5)
    model.fit(np.concatenate(Xs), np.concatenate(Ys), epochs=60, batch=256, lr=3e-3)
    yield sysm, dirs[3], model
    model.close()


def _learned_run(B, sysm, d, model, mode, n_windows, **kw):
    from paper_1912_03174_gb300 import learned as Lrn
    run = I.Run(dt=0.2, n_steps=0, scc=True, kick=0.02, kick_dir=d, kT=I.SCC_KT)
    p = B.Propagator(sysm, run, "fp64")
    p.setup()
    p.step(1)
    lp = Lrn.LearnedPropagator(p.ctx, model, mode=mode, **kw)
    q = []
    lp.warm_up()
    for _ in range(n_windows):
        lp.run(1)
        q.append(B.tdb_observables(p.ctx)["charges"])
    return p, lp, np.array(q)


def _plain_reference(B, sysm, d, n_windows):
    run = I.Run(dt=0.2, n_steps=0, scc=True, kick=0.02, kick_dir=d, kT=I.SCC_KT)
    with B.Propagator(sysm, run, "fp64") as p:
        p.setup()
        p.step(1 + L_HIST * K_WIN)
        q = []
        for _ in range(n_windows):
            p.step(K_WIN)
            q.append(p.observables()["charges"])
    return np.array(q)


def test_trained_network_beats_the_frozen_shift(B, trained):
    sysm, d, model = trained
    # the target is scaled to unit variance: the fit explains over 95 % of it
    assert model.losses[-1] < 0.05
    nw = 40
    q_ref = _plain_reference(B, sysm, d, nw)
    err = {}
    for mode in ("frozen", "net"):
        p, lp, q = _learned_run(B, sysm, d, model, mode, nw)
        p.close()
        assert lp.stats.windows == nw and not lp.stats.taken_over
        err[mode] = np.max(np.abs(q - q_ref), axis=1)
    # held-out kick direction: after 40 windows (400 steps) the frozen shift has drifted
    # far off while the network's windows stay near the plain leapfrog
    assert err["net"][-1] < 0.05
    assert err["net"][-1] < 0.1 * err["frozen"][-1]
    assert np.max(err["net"]) < 0.5 * np.max(err["frozen"])


def test_referee_takes_over_and_continues_as_the_plain_leapfrog(B, trained):
    sysm, d, model = trained
    nw = 6
    q_ref = _plain_reference(B, sysm, d, nw)
    # a bound below any window error: the referee keeps its own state at the first window
    # and plain steps follow, which is the plain run bit for bit
    p, lp, q = _learned_run(B, sysm, d, model, "net", nw, referee_every=2, bound=0.0)
    p.close()
    assert lp.stats.taken_over and lp.stats.refereed == 1 and lp.stats.windows == 1
    assert np.array_equal(q, q_ref)
    # a loose bound: refereed every second window, never taken over
    p, lp, q = _learned_run(B, sysm, d, model, "net", nw, referee_every=2, bound=1.0)
    p.close()
    assert not lp.stats.taken_over and lp.stats.refereed == 3 and lp.stats.windows == nw
    assert all(e < 0.02 for e in lp.stats.referee_err)
