"""Host logic of the learned form (no GPU): training samples and window features."""
import numpy as np
import pytest

from paper_1912_03174_gb300 import learned as Lrn
from oracle import tdb_oracle as O


def test_training_set_on_a_ramp():
    # v_A(n) = a_A n + c_A: window mean minus start = a (k - 1) / 2, features -a j k
    k, L, T = 5, 3, 40
    a = np.array([0.1, -0.02, 0.003])
    v = np.arange(T)[:, None] * a[None, :] + np.array([1.0, 2.0, 3.0])
    X, Y = Lrn.training_set(v, k, L)
    n_win = T - k + 1 - L * k
    assert X.shape == (n_win * 3, L) and Y.shape == (n_win * 3,)
    np.testing.assert_allclose(Y.reshape(n_win, 3), np.tile(a * (k - 1) / 2, (n_win, 1)), atol=1e-12)
    want = -np.outer(a, np.arange(1, L + 1) * k)
    np.testing.assert_allclose(X[:3], want, atol=1e-12)


def test_training_set_window_mean_by_brute_force():
    rng = np.random.default_rng(3)
    k, L = 4, 2
    v = rng.normal(size=(30, 2))
    X, Y = Lrn.training_set(v, k, L)
    n0 = L * k
    for i, n in enumerate(range(n0, 30 - k + 1)):
        for A in range(2):
            assert Y[2 * i + A] == pytest.approx(np.mean(v[n:n + k, A]) - v[n, A], abs=1e-13)
            assert X[2 * i + A, 1] == pytest.approx(v[n - 2 * k, A] - v[n, A], abs=1e-15)


def test_training_set_too_short_is_empty():
    X, Y = Lrn.training_set(np.zeros((10, 3)), 5, 2)
    assert X.shape == (0, 2) and Y.shape == (0,)


def test_window_features_order():
    hist = [np.array([1.0]), np.array([3.0]), np.array([6.0])]
    np.testing.assert_allclose(Lrn.window_features(hist, 2), [[-3.0, -5.0]])
    # two channels (shift, charge): all shift differences first, then the charges'
    hist = [np.array([[1.0, 10.0]]), np.array([[3.0, 20.0]]), np.array([[6.0, 50.0]])]
    np.testing.assert_allclose(Lrn.window_features(hist, 2), [[-3.0, -5.0, -30.0, -40.0]])


def test_training_set_with_charges_targets_the_shift_only():
    rng = np.random.default_rng(8)
    k, L = 3, 2
    rec = rng.normal(size=(20, 4, 2))
    X, Y = Lrn.training_set(rec, k, L)
    X1, Y1 = Lrn.training_set(rec[:, :, 0], k, L)
    assert X.shape[1] == 2 * L
    np.testing.assert_array_equal(Y, Y1)
    np.testing.assert_array_equal(X[:, :L], X1)
    n = L * k
    np.testing.assert_allclose(X[0, L:], [rec[n - k, 0, 1] - rec[n, 0, 1], rec[n - 2 * k, 0, 1] - rec[n, 0, 1]])


def test_oracle_bf16_gradient_is_that_of_the_rounded_weights():
    # the straight-through reading: the gradient with rounding equals the gradient of the
    # unrounded network evaluated at the rounded weights
    rng = np.random.default_rng(9)
    F, H, n = 5, 6, 30
    p = rng.normal(size=F * H + 3 * H + H * H + 1)
    q = p.copy()
    W1, b1, W2, b2, w3, b3 = O.shiftnet_unpack(q, F, H)   # views into q
    W1[:] = O.bf16_round(W1)
    W2[:] = O.bf16_round(W2)
    w3[:] = O.bf16_round(w3)
    X = rng.normal(size=(n, F))
    Y = rng.normal(size=n)
    l1, g1 = O.shiftnet_loss_grad(p, X, Y, F, H, bf16=True)
    l2, g2 = O.shiftnet_loss_grad(q, X, Y, F, H, bf16=False)
    assert l1 == l2
    np.testing.assert_array_equal(g1, g2)


class _FakeCtx:
    """A stand-in context: charges follow q(t) = sin(0.1 t) per atom; a window of k
    steps lands on q(t + k) + err, plain steps exactly on q(t + k)."""

    def __init__(self, n_atoms=3, t=0, err=0.0):
        self.n_atoms, self.t, self.err = n_atoms, t, err

    def q(self):
        return np.sin(0.1 * self.t + np.arange(self.n_atoms)) + self.err


class _FakeB:
    """Window m (counted from 1) adds window_err (grow: window_err * m) to the charges."""

    def __init__(self, window_err, grow=False):
        self.window_err, self.grow = window_err, grow
        self.windows, self.plain, self.clones, self.destroyed, self.loaded = 0, 0, 0, 0, 0

    def tdb_scc_shift(self, ctx, charges=False):
        v = 2.0 * ctx.q()
        return (v, ctx.q()) if charges else v

    def tdb_step(self, ctx, n):
        self.plain += n
        ctx.t += n

    def tdb_step_window(self, ctx, v_bar, k):
        assert v_bar.shape == (ctx.n_atoms,)
        self.windows += 1
        ctx.t += k
        ctx.err += self.window_err * (self.windows if self.grow else 1)

    def tdb_clone(self, ctx):
        self.clones += 1
        return _FakeCtx(ctx.n_atoms, ctx.t, ctx.err)

    def tdb_observables(self, ctx):
        q = ctx.q()
        return {"charges": q, "dipole": np.array([q.sum(), 0.0, 0.0])}

    def tdb_get_state(self, ctx):
        return (ctx.t, ctx.err)

    def tdb_set_state(self, ctx, blob):
        self.loaded += 1
        ctx.t, ctx.err = blob

    def tdb_destroy(self, ctx):
        self.destroyed += 1


class _FakeModel:
    k, L = 4, 3

    def increment(self, X):
        assert X.shape == (3, 2 * self.L)
        return np.full(X.shape[0], 0.5)


def _propagator(monkeypatch, window_err, grow=False, **kw):
    fake = _FakeB(window_err, grow)
    monkeypatch.setattr(Lrn, "B", fake)
    ctx = _FakeCtx()
    return fake, ctx, Lrn.LearnedPropagator(ctx, _FakeModel(), **kw)


def test_driver_warms_up_then_runs_windows(monkeypatch):
    fake, ctx, lp = _propagator(monkeypatch, 0.0)
    st = lp.run(5)
    assert fake.plain == 3 * 4 and fake.windows == 5 and ctx.t == 12 + 20
    assert st.windows == 5 and st.refereed == 0 and not st.taken_over
    assert len(lp.history) == _FakeModel.L + 1
    # the network's shift: v + increment; the frozen mode passes v itself
    np.testing.assert_allclose(lp.v_bar(), 2.0 * ctx.q() + 0.5)
    lp.mode = "frozen"
    np.testing.assert_allclose(lp.v_bar(), 2.0 * ctx.q())


def test_referee_samples_every_nth_window_and_keeps_the_window_below_the_bound(monkeypatch):
    fake, ctx, lp = _propagator(monkeypatch, 1e-3, referee_every=3, bound=1e-2)
    st = lp.run(7)
    assert st.refereed == 3 and fake.clones == 3 and fake.destroyed == 3   # windows 0, 3, 6
    assert not st.taken_over and fake.loaded == 0 and fake.windows == 7
    np.testing.assert_allclose(st.referee_err, [1e-3, 1e-3, 1e-3], rtol=1e-9)
    np.testing.assert_allclose(st.referee_dipole_err, [3e-3, 3e-3, 3e-3], rtol=1e-9)
    assert ctx.err == pytest.approx(7e-3)


def test_referee_takes_over_on_the_charge_or_the_dipole_bound(monkeypatch):
    # charges: the referee measures each sampled window from its own start state; window
    # errors 1e-3, 2e-3, 3e-3, ... and refereed windows 1, 3, 5: the second one (3e-3)
    # exceeds the bound
    fake, ctx, lp = _propagator(monkeypatch, 1e-3, grow=True, referee_every=2, bound=2.5e-3)
    st = lp.run(6)
    assert st.taken_over and st.refereed == 2 and st.windows == 3
    np.testing.assert_allclose(st.referee_err, [1e-3, 3e-3], rtol=1e-9)
    assert fake.loaded == 1 and ctx.err == pytest.approx(3e-3)    # the referee's state
    assert st.plain_steps == 3 * 4 + 3 * 4                         # warm-up, then plain
    assert ctx.t == 12 + 6 * 4
    # dipole: the charge bound is loose, the dipole one (3 atoms x 1e-3) is not
    fake, ctx, lp = _propagator(monkeypatch, 1e-3, referee_every=1, bound=1.0, dipole_bound=2e-3)
    st = lp.run(2)
    assert st.taken_over and st.refereed == 1 and ctx.err == 0.0
