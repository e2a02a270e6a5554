"""The learned form of the propagator: windows of k leapfrog steps taken in closed form
(tdb_step_window) with the Hamiltonian frozen at a window-mean SCC shift that a small
per-atom network predicts from the shift history at earlier window ends.

Without the network the window would freeze the shift at its value at the window's
start; with an SCC Hamiltonian (eq:hscc) that lags the charges by half a window and the
error grows from window to window.  The network (tdb_shiftnet_*, trained on the GPU by
the library's own forward and backward kernels) is fitted on shift histories of plain
leapfrog runs (eq:leapfrog): its input for atom A at the start n of a window is
(v_A(n - j k) - v_A(n)), j = 1..L, its target the mean of v_A over the steps n..n+k-1
minus v_A(n).  The plain leapfrog re-runs sampled windows from the same state as a
judge; when the window's charges differ from the judge's by more than a bound the
judge's state is kept and the run continues with plain steps.

Everything here is host orchestration over the C ABI; each step runs in the library.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import binding as B


def record_shifts(ctx: B.Context, n_steps: int) -> np.ndarray:
    """Plain leapfrog for n_steps; returns v(rho_n) for n = 0..n_steps, (n_steps + 1, n_atoms)."""
    out = [B.tdb_scc_shift(ctx)]
    for _ in range(n_steps):
        B.tdb_step(ctx, 1)
        out.append(B.tdb_scc_shift(ctx))
    return np.array(out)


def window_features(history, L: int) -> np.ndarray:
    """(n_atoms, L) network input from shifts at the last L + 1 window ends (oldest first)."""
    cur = history[-1]
    return np.stack([history[-1 - j] - cur for j in range(1, L + 1)], axis=1)


def training_set(shifts: np.ndarray, k: int, L: int):
    """Samples from a per-step shift record (n, n_atoms): for each window start n with
    L earlier window ends and k following steps, features of every atom and the target
    mean(v(n..n+k-1)) - v(n)."""
    X, Y = [], []
    csum = np.concatenate([np.zeros((1, shifts.shape[1])), np.cumsum(shifts, axis=0)])
    for n in range(L * k, shifts.shape[0] - k + 1):
        hist = [shifts[n - j * k] for j in range(L, -1, -1)]
        X.append(window_features(hist, L))
        Y.append((csum[n + k] - csum[n]) / k - shifts[n])
    if not X:
        return np.zeros((0, L)), np.zeros(0)
    return np.concatenate(X), np.concatenate(Y)


@dataclass
class ShiftModel:
    """The network with its input and output scales (features / sx, target / sy)."""
    k: int
    L: int = 8
    hidden: int = 32
    seed: int = 0
    sx: float = 1.0
    sy: float = 1.0
    net: B.ShiftNet = None
    losses: list = field(default_factory=list)

    def __post_init__(self):
        if self.net is None:
            self.net = B.ShiftNet(self.L, self.hidden, self.seed)

    def fit(self, X, Y, epochs=60, batch=256, lr=3e-3, seed=0):
        """Adam on the mean squared error of the scaled target (samples shuffled once)."""
        self.sx = float(np.std(X)) or 1.0
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
    judged: int = 0
    taken_over: bool = False
    plain_steps: int = 0
    judge_err: list = field(default_factory=list)


class LearnedPropagator:
    """Advance ctx (FP64 or FP64_SLICED form, frozen nuclei, no field) in windows of
    model.k steps.  mode 'net' uses the network's shift, 'frozen' the shift at the
    window's start (the method without the network).  judge_every: every so many
    windows a clone of the context takes the k plain steps instead and the charges are
    compared (max |dq|); above bound the judge's state is kept and plain steps follow."""

    def __init__(self, ctx: B.Context, model: ShiftModel, mode="net", judge_every=0, bound=1e-2):
        self.ctx, self.model, self.mode = ctx, model, mode
        self.judge_every, self.bound = judge_every, bound
        self.history = []
        self.stats = WindowStats()

    def warm_up(self):
        """L windows of plain steps (they also give the first history)."""
        k, L = self.model.k, self.model.L
        for _ in range(L):
            self.history.append(B.tdb_scc_shift(self.ctx))
            B.tdb_step(self.ctx, k)
            self.stats.plain_steps += k

    def v_bar(self) -> np.ndarray:
        v = B.tdb_scc_shift(self.ctx)
        self.history.append(v)
        self.history = self.history[-(self.model.L + 1):]
        if self.mode == "frozen":
            return v
        return v + self.model.increment(window_features(self.history, self.model.L))

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
            judge = None
            if self.judge_every and self.stats.windows % self.judge_every == 0:
                judge = B.tdb_clone(self.ctx)
            B.tdb_step_window(self.ctx, vb, k)
            self.stats.windows += 1
            if judge is not None:
                try:
                    B.tdb_step(judge, k)
                    qa = B.tdb_observables(self.ctx)["charges"]
                    qb = B.tdb_observables(judge)["charges"]
                    err = float(np.max(np.abs(qa - qb)))
                    self.stats.judged += 1
                    self.stats.judge_err.append(err)
                    if err > self.bound:
                        B.tdb_set_state(self.ctx, B.tdb_get_state(judge))
                        self.stats.taken_over = True
                finally:
                    B.tdb_destroy(judge)
        return self.stats
