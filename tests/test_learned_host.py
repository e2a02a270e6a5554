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
