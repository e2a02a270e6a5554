"""The learned form of the propagator: windows of k leapfrog steps taken in closed form
(tdb_step_window) with the Hamiltonian frozen at a window-mean SCC shift that a small
per-atom network predicts from the shift and charge history at earlier window ends.

Without the network the window would freeze the shift at its value at the window's
start; with an SCC Hamiltonian (eq:hscc) that lags the charges by half a window and the
error grows from window to window.  The network (tdb_shiftnet_*, trained on the GPU by
the library's own forward and backward kernels) is fitted on records of plain leapfrog
runs (eq:leapfrog): its input for atom A at the start n of a window is
(v_A(n - j k) - v_A(n)) and (dq_A(n - j k) - dq_A(n)), j = 1..L (2 L values), its
target the mean of v_A over the steps n..n+k-1 minus v_A(n).  The plain leapfrog
re-runs sampled windows from the same state as a referee; when the window's charges or
dipole differ from the referee's by more than their bounds the referee's state is kept and
the run continues with plain steps.

Everything here is host orchestration over the C ABI; each step runs in the library.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import binding as B


def sample(ctx: B.Context) -> np.ndarray:
    """(n_atoms, 2): the SCC shift v and the charge fluctuation dq of rho_n per atom."""
    v, dq = B.tdb_scc_shift(ctx, charges=True)
    return np.stack([v, dq], axis=1)


def record(ctx: B.Context, n_steps: int) -> np.ndarray:
    """Plain leapfrog for n_steps; (n_steps + 1, n_atoms, 2) samples of rho_0..rho_n."""
    out = [sample(ctx)]
    for _ in range(n_steps):
        B.tdb_step(ctx, 1)
        out.append(sample(ctx))
    return np.array(out)


def window_features(history, L: int) -> np.ndarray:
    """(n_atoms, L * channels) network input from samples at the last L + 1 window ends
    (oldest first, each n_atoms or n_atoms x channels): differences to the newest,
    channel by channel."""
    h = [np.asarray(x).reshape(len(x), -1) for x in history[-(L + 1):]]
    cur = h[-1]
    return np.concatenate([np.stack([h[-1 - j][:, c] - cur[:, c] for j in range(1, L + 1)], axis=1)
                           for c in range(cur.shape[1])], axis=1)


def training_set(rec: np.ndarray, k: int, L: int):
    """Samples from a per-step record (n, n_atoms) of shifts or (n, n_atoms, channels)
    with the shift first: for each window start n with L earlier window ends and k
    following steps, features of every atom and the target mean(v(n..n+k-1)) - v(n)."""
    rec = np.asarray(rec)
    if rec.ndim == 2:
        rec = rec[:, :, None]
    v = rec[:, :, 0]
    X, Y = [], []
    csum = np.concatenate([np.zeros((1, v.shape[1])), np.cumsum(v, axis=0)])
    for n in range(L * k, rec.shape[0] - k + 1):
        X.append(window_features([rec[n - j * k] for j in range(L, -1, -1)], L))
        Y.append((csum[n + k] - csum[n]) / k - v[n])
    if not X:
        return np.zeros((0, L * rec.shape[2])), np.zeros(0)
    return np.concatenate(X), np.concatenate(Y)


@dataclass
class ShiftModel:
    """The network with its input and output scales (features / sx, target / sy)."""
    k: int
    L: int = 8
    hidden: int = 32
    seed: int = 0
    channels: int = 2
    sx: np.ndarray = None
    sy: float = 1.0
    net: B.ShiftNet = None
    losses: list = field(default_factory=list)

    def __post_init__(self):
        if self.net is None:
            self.net = B.ShiftNet(self.L * self.channels, self.hidden, self.seed)

    def fit(self, X, Y, epochs=60, batch=256, lr=3e-3, seed=0):
        """Adam on the mean squared error of the scaled target (samples shuffled once);
        each channel's features are scaled by their standard deviation."""
        sx = X.reshape(len(X), self.channels, self.L).std(axis=(0, 2))
        self.sx = np.repeat(np.where(sx > 0, sx, 1.0), self.L)
        self.sy = float(np.std(Y)) or 1.0
        perm = np.random.default_rng(seed).permutation(len(Y))
        Xs = (X[perm] / self.sx).astype(np.float32)
        Ys = (Y[perm] / self.sy).astype(np.float32)
        for _ in range(epochs):
            self.losses.append(self.net.train(Xs, Ys, 1, batch, lr))
        return self.losses[-1]

    def increment(self, X) -> np.ndarray:
        return self.net.predict((np.asarray(X) / self.sx).astype(np.float32)).astype(np.float64) * self.sy

    def close(self):
        self.net.close()


@dataclass
class WindowStats:
    windows: int = 0
    refereed: int = 0
    taken_over: bool = False
    plain_steps: int = 0
    referee_err: list = field(default_factory=list)          # max |dq| per refereed window
    referee_dipole_err: list = field(default_factory=list)   # max |d mu| per refereed window


class LearnedPropagator:
    """Advance ctx (FP64 or FP64_SLICED form, frozen nuclei, no field) in windows of
    model.k steps.  mode 'net' uses the network's shift, 'frozen' the shift at the
    window's start (the method without the network).  referee_every: every so many
    windows a clone of the context takes the k plain steps instead and the charges
    (max |dq|) and dipoles (max |d mu|, a.u.) are compared; above bound or
    dipole_bound the referee's state is kept and plain steps follow."""

    def __init__(self, ctx: B.Context, model: ShiftModel, mode="net", referee_every=0, bound=1e-2,
                 dipole_bound=float("inf")):
        self.ctx, self.model, self.mode = ctx, model, mode
        self.referee_every, self.bound, self.dipole_bound = referee_every, bound, dipole_bound
        self.history = []
        self.stats = WindowStats()

    def warm_up(self):
        """L windows of plain steps (they also give the first history)."""
        k, L = self.model.k, self.model.L
        for _ in range(L):
            self.history.append(sample(self.ctx))
            B.tdb_step(self.ctx, k)
            self.stats.plain_steps += k

    def v_bar(self) -> np.ndarray:
        s = sample(self.ctx)
        self.history.append(s)
        self.history = self.history[-(self.model.L + 1):]
        if self.mode == "frozen":
            return s[:, 0]
        return s[:, 0] + self.model.increment(window_features(self.history, self.model.L))

    def run(self, n_windows: int) -> WindowStats:
        k = self.model.k
        if len(self.history) < self.model.L:
            self.warm_up()
        for _ in range(n_windows):
            if self.stats.taken_over:
                B.tdb_step(self.ctx, k)
                self.stats.plain_steps += k
                continue
            vb = self.v_bar()
            referee = None
            if self.referee_every and self.stats.windows % self.referee_every == 0:
                referee = B.tdb_clone(self.ctx)
            B.tdb_step_window(self.ctx, vb, k)
            self.stats.windows += 1
            if referee is not None:
                try:
                    B.tdb_step(referee, k)
                    oa = B.tdb_observables(self.ctx)
                    ob = B.tdb_observables(referee)
                    err = float(np.max(np.abs(oa["charges"] - ob["charges"])))
                    derr = float(np.max(np.abs(np.asarray(oa["dipole"]) - np.asarray(ob["dipole"]))))
                    self.stats.refereed += 1
                    self.stats.referee_err.append(err)
                    self.stats.referee_dipole_err.append(derr)
                    if err > self.bound or derr > self.dipole_bound:
                        B.tdb_set_state(self.ctx, B.tdb_get_state(referee))
                        self.stats.taken_over = True
                finally:
                    B.tdb_destroy(referee)
        return self.stats
