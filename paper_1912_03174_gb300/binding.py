"""Thin ctypes binding of ``libtdb.so`` (include/tdb.h).

Argument marshalling only: every step of the propagation runs in the CUDA
library.  If the library is missing this module raises; there is no CPU
fallback.  Function names follow the C ABI.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import build as _build

TDB_FP64, TDB_FP32, TDB_BF16X3, TDB_FP16X3, TDB_FP16X6, TDB_FP64_SLICED = 0, 1, 2, 3, 4, 5
PRECISIONS = {"fp64": TDB_FP64, "fp32": TDB_FP32, "bf16x3": TDB_BF16X3, "fp16x3": TDB_FP16X3,
              "fp16x6": TDB_FP16X6, "fp64s": TDB_FP64_SLICED}

_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_ip = ctypes.POINTER(ctypes.c_int)


class TdbSystem(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int), ("orbs_per_atom", ctypes.c_int), ("n_species", ctypes.c_int),
                ("species", _ip), ("R", _dp), ("V", _dp), ("eps_s", _dp), ("eps_p", _dp),
                ("hubbard_U", _dp), ("mass", _dp), ("t0", ctypes.c_double), ("lam_H", ctypes.c_double),
                ("s0", ctypes.c_double), ("lam_S", ctypes.c_double), ("eta", ctypes.c_double * 4),
                ("rep_A", ctypes.c_double), ("rep_b", ctypes.c_double), ("n_electrons", ctypes.c_double)]


class TdbParams(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("scc", ctypes.c_int), ("move_nuclei", ctypes.c_int),
                ("precision", ctypes.c_int), ("window", ctypes.c_int), ("scc_tol", ctypes.c_double),
                ("scc_max_iter", ctypes.c_int), ("kT", ctypes.c_double), ("scc_mix", ctypes.c_double),
                ("history_cap", ctypes.c_long), ("cuda_stream", ctypes.c_void_p)]


class TdbField(ctypes.Structure):
    _fields_ = [("E0", ctypes.c_double), ("omega", ctypes.c_double), ("phase", ctypes.c_double),
                ("t_center", ctypes.c_double), ("fwhm", ctypes.c_double), ("dir", ctypes.c_double * 3),
                ("envelope", ctypes.c_int)]


class TdbObs(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("step", ctypes.c_long), ("dipole", ctypes.c_double * 3),
                ("E_total", ctypes.c_double), ("E_band", ctypes.c_double), ("E_coul", ctypes.c_double),
                ("E_rep", ctypes.c_double), ("E_kin", ctypes.c_double), ("E_ext", ctypes.c_double),
                ("work", ctypes.c_double), ("trace_re", ctypes.c_double), ("trace_im", ctypes.c_double),
                ("herm_err", ctypes.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["dipole"] = np.array(self.dipole[:])
        return d


# symbol -> (restype, argtypes); every function of include/tdb.h
SIGNATURES = {
    "tdb_default_params": (None, [ctypes.POINTER(TdbParams)]),
    "tdb_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(TdbSystem), ctypes.POINTER(TdbParams)]),
    "tdb_create": (ctypes.c_int, [ctypes.POINTER(TdbSystem), ctypes.POINTER(TdbParams), ctypes.c_void_p,
                                  ctypes.c_size_t, ctypes.POINTER(ctypes.c_void_p)]),
    "tdb_ground_state": (ctypes.c_int, [ctypes.c_void_p, _ip, _dp]),
    "tdb_kick": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, _dp]),
    "tdb_set_field": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(TdbField)]),
    "tdb_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_long]),
    "tdb_scc_shift": (ctypes.c_int, [ctypes.c_void_p, _dp, _dp]),
    "tdb_step_window": (ctypes.c_int, [ctypes.c_void_p, _dp, ctypes.c_int]),
    "tdb_shiftnet_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_ulonglong,
                                           ctypes.POINTER(ctypes.c_void_p)]),
    "tdb_shiftnet_param_count": (ctypes.c_long, [ctypes.c_void_p]),
    "tdb_shiftnet_get_params": (ctypes.c_int, [ctypes.c_void_p, _fp]),
    "tdb_shiftnet_set_params": (ctypes.c_int, [ctypes.c_void_p, _fp]),
    "tdb_shiftnet_predict": (ctypes.c_int, [ctypes.c_void_p, _fp, ctypes.c_long, _fp]),
    "tdb_shiftnet_gradient": (ctypes.c_int, [ctypes.c_void_p, _fp, _fp, ctypes.c_long, _fp, _dp]),
    "tdb_shiftnet_train": (ctypes.c_int, [ctypes.c_void_p, _fp, _fp, ctypes.c_long, ctypes.c_int,
                                          ctypes.c_long, ctypes.c_float, _dp]),
    "tdb_shiftnet_destroy": (None, [ctypes.c_void_p]),
    "tdb_clone": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                  ctypes.POINTER(ctypes.c_void_p)]),
    "tdb_step_batch": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_long]),
    "tdb_observables": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(TdbObs), _dp, _dp]),
    "tdb_dipole_history": (ctypes.c_int, [ctypes.c_void_p, _dp, ctypes.c_long, ctypes.POINTER(ctypes.c_long)]),
    "tdb_get_rho": (ctypes.c_int, [ctypes.c_void_p, _dp, _dp, _dp, _dp]),
    "tdb_state_bytes": (ctypes.c_size_t, [ctypes.c_void_p]),
    "tdb_get_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "tdb_set_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "tdb_check": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    "tdb_last_launch_count": (ctypes.c_long, [ctypes.c_void_p]),
    "tdb_wait_probe": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong]),
    "tdb_set_x_tile": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "tdb_x_tile": (ctypes.c_int, [ctypes.c_void_p]),
    "tdb_step_profiled": (ctypes.c_int, [ctypes.c_void_p, _dp, ctypes.POINTER(ctypes.c_char_p), ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int)]),
    "tdb_split_gemm": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_int, _dp, _dp]),
    "tdb_slice_gemm": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp]),
    "tdb_split_gemm_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "tdb_batch_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "tdb_batch_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_long]),
    "tdb_batch_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int), _dp]),
    "tdb_batch_destroy": (None, [ctypes.c_void_p]),
    "tdb_damped_transform": (ctypes.c_int, [ctypes.c_int, ctypes.c_long, _dp, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_int, _dp, _dp, _dp]),
    "tdb_destroy": (None, [ctypes.c_void_p]),
    "tdb_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "tdb_last_error": (ctypes.c_char_p, []),
}

_lib = None


class TdbError(RuntimeError):
    def __init__(self, func, status, message):
        self.status = status
        super().__init__(f"{func}: {message} (status {status})")


def library_path() -> str:
    return _build.LIB


def load(path: Optional[str] = None):
    """Load libtdb.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or _build.LIB
    if not os.path.exists(p):
        raise RuntimeError(f"libtdb.so not found at {p}: run __graft_entry__.build() first")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _check(func, status):
    if status != 0:
        lib = load()
        msg = lib.tdb_last_error().decode()
        raise TdbError(func, status, f"{lib.tdb_status_string(status).decode()}: {msg}")


def _ptr(a):
    return a.ctypes.data_as(_dp)


class _SystemArgs:
    """Holds the numpy arrays behind a TdbSystem for the duration of a call."""

    def __init__(self, sysm):
        self.species = np.ascontiguousarray(sysm.species, dtype=np.int32)
        self.R = np.ascontiguousarray(sysm.R, dtype=np.float64)
        self.V = None if sysm.V is None else np.ascontiguousarray(sysm.V, dtype=np.float64)
        self.eps_s = np.ascontiguousarray(sysm.eps_s, dtype=np.float64)
        self.eps_p = np.ascontiguousarray(sysm.eps_p, dtype=np.float64)
        self.U = np.ascontiguousarray(sysm.hubbard_U, dtype=np.float64)
        self.mass = np.ascontiguousarray(sysm.mass, dtype=np.float64)
        s = TdbSystem()
        s.n_atoms = self.R.shape[0]
        s.orbs_per_atom = int(sysm.orbs_per_atom)
        s.n_species = self.eps_s.shape[0]
        s.species = self.species.ctypes.data_as(_ip)
        s.R = _ptr(self.R)
        s.V = _ptr(self.V) if self.V is not None else _dp()
        s.eps_s, s.eps_p, s.hubbard_U, s.mass = _ptr(self.eps_s), _ptr(self.eps_p), _ptr(self.U), _ptr(self.mass)
        s.t0, s.lam_H, s.s0, s.lam_S = sysm.t0, sysm.lam_H, sysm.s0, sysm.lam_S
        for k in range(4):
            s.eta[k] = float(sysm.eta[k])
        s.rep_A, s.rep_b = sysm.rep_A, sysm.rep_b
        s.n_electrons = float(sysm.n_electrons)
        self.struct = s


def tdb_default_params() -> TdbParams:
    p = TdbParams()
    load().tdb_default_params(ctypes.byref(p))
    return p


def make_params(run, precision="fp64", stream=None, history_cap=65536, window=100) -> TdbParams:
    p = tdb_default_params()
    p.dt = run.dt
    p.scc = int(run.scc)
    p.move_nuclei = int(run.move_nuclei)
    p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    p.window = window
    p.scc_tol = run.scc_tol
    p.scc_max_iter = run.scc_max_iter
    p.kT = run.kT
    p.history_cap = history_cap
    p.cuda_stream = stream
    return p


def make_field(fld) -> Optional[TdbField]:
    if fld is None:
        return None
    f = TdbField()
    f.E0, f.omega, f.phase, f.t_center, f.fwhm = fld.E0, fld.omega, fld.phase, fld.t_center, fld.fwhm
    for k in range(3):
        f.dir[k] = float(fld.dir[k])
    f.envelope = int(fld.envelope)
    return f


def tdb_workspace_bytes(sysm, params: TdbParams) -> int:
    a = _SystemArgs(sysm)
    return int(load().tdb_workspace_bytes(ctypes.byref(a.struct), ctypes.byref(params)))


@dataclass
class Context:
    handle: ctypes.c_void_p
    n_atoms: int
    n_orb: int
    workspace: object = None    # keeps a caller-supplied (torch) workspace alive


def tdb_create(sysm, params: TdbParams, workspace=None) -> Context:
    """workspace: None (library allocates) or a CUDA uint8 torch tensor of at least
    tdb_workspace_bytes() bytes."""
    lib = load()
    a = _SystemArgs(sysm)
    h = ctypes.c_void_p()
    ptr, nbytes = None, 0
    if workspace is not None:
        ptr, nbytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    _check("tdb_create", lib.tdb_create(ctypes.byref(a.struct), ctypes.byref(params), ptr, nbytes,
                                        ctypes.byref(h)))
    return Context(h, a.R.shape[0], a.R.shape[0] * int(sysm.orbs_per_atom), workspace)


def tdb_ground_state(ctx: Context):
    it = ctypes.c_int()
    res = ctypes.c_double()
    _check("tdb_ground_state", load().tdb_ground_state(ctx.handle, ctypes.byref(it), ctypes.byref(res)))
    return it.value, res.value


def tdb_kick(ctx: Context, strength: float, direction):
    d = np.ascontiguousarray(direction, dtype=np.float64)
    _check("tdb_kick", load().tdb_kick(ctx.handle, float(strength), _ptr(d)))


def tdb_set_field(ctx: Context, fld):
    f = make_field(fld) if fld is not None and not isinstance(fld, TdbField) else fld
    _check("tdb_set_field", load().tdb_set_field(ctx.handle, ctypes.byref(f) if f is not None else None))


def tdb_step(ctx: Context, n: int):
    _check("tdb_step", load().tdb_step(ctx.handle, int(n)))


def tdb_scc_shift(ctx: Context, charges=False):
    """The SCC shift of rho_n per atom; with charges=True also dq: (shift, dq)."""
    out = np.zeros(ctx.n_atoms)
    dq = np.zeros(ctx.n_atoms) if charges else None
    _check("tdb_scc_shift", load().tdb_scc_shift(ctx.handle, _ptr(out), _ptr(dq) if charges else None))
    return (out, dq) if charges else out


def tdb_step_window(ctx: Context, v_bar, k: int):
    v = np.ascontiguousarray(v_bar, dtype=np.float64)
    assert v.shape == (ctx.n_atoms,)
    _check("tdb_step_window", load().tdb_step_window(ctx.handle, _ptr(v), int(k)))


def _fptr(a):
    return a.ctypes.data_as(_fp)


class ShiftNet:
    """The per-atom shift network on the GPU (tdb_shiftnet_*)."""

    def __init__(self, n_features: int, hidden: int = 64, seed: int = 0):
        self.F, self.H = int(n_features), int(hidden)
        self.handle = ctypes.c_void_p()
        _check("tdb_shiftnet_create", load().tdb_shiftnet_create(self.F, self.H, int(seed),
                                                                 ctypes.byref(self.handle)))
        self.n_params = int(load().tdb_shiftnet_param_count(self.handle))

    def params(self) -> np.ndarray:
        p = np.zeros(self.n_params, dtype=np.float32)
        _check("tdb_shiftnet_get_params", load().tdb_shiftnet_get_params(self.handle, _fptr(p)))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.shape == (self.n_params,)
        _check("tdb_shiftnet_set_params", load().tdb_shiftnet_set_params(self.handle, _fptr(p)))

    def predict(self, X) -> np.ndarray:
        X = np.ascontiguousarray(X, dtype=np.float32)
        Y = np.zeros(X.shape[0], dtype=np.float32)
        _check("tdb_shiftnet_predict", load().tdb_shiftnet_predict(self.handle, _fptr(X), X.shape[0], _fptr(Y)))
        return Y

    def gradient(self, X, Y):
        X = np.ascontiguousarray(X, dtype=np.float32)
        Y = np.ascontiguousarray(Y, dtype=np.float32)
        g = np.zeros(self.n_params, dtype=np.float32)
        loss = ctypes.c_double()
        _check("tdb_shiftnet_gradient", load().tdb_shiftnet_gradient(
            self.handle, _fptr(X), _fptr(Y), X.shape[0], _fptr(g), ctypes.byref(loss)))
        return loss.value, g

    def train(self, X, Y, epochs: int, batch: int, lr: float) -> float:
        X = np.ascontiguousarray(X, dtype=np.float32)
        Y = np.ascontiguousarray(Y, dtype=np.float32)
        loss = ctypes.c_double()
        _check("tdb_shiftnet_train", load().tdb_shiftnet_train(
            self.handle, _fptr(X), _fptr(Y), X.shape[0], int(epochs), int(batch), float(lr),
            ctypes.byref(loss)))
        return loss.value

    def close(self):
        if self.handle:
            load().tdb_shiftnet_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def tdb_clone(ctx: Context, stream=None) -> Context:
    """A new context in ctx's current state (device-to-device copy), with its own stream."""
    h = ctypes.c_void_p()
    _check("tdb_clone", load().tdb_clone(ctx.handle, stream, None, 0, ctypes.byref(h)))
    return Context(handle=h, n_atoms=ctx.n_atoms, n_orb=ctx.n_orb)


def tdb_step_batch(ctxs, n: int):
    """Advance independent contexts by n steps each, interleaved across their streams."""
    arr = (ctypes.c_void_p * len(ctxs))(*[c.handle.value if isinstance(c.handle, ctypes.c_void_p)
                                          else c.handle for c in ctxs])
    _check("tdb_step_batch", load().tdb_step_batch(arr, len(ctxs), int(n)))


class Batch:
    """A grouped batch of contexts (tdb_batch_*): every phase of a step is one launch over
    all of them."""

    def __init__(self, ctxs):
        arr = (ctypes.c_void_p * len(ctxs))(*[c.handle for c in ctxs])
        h = ctypes.c_void_p()
        _check("tdb_batch_create", load().tdb_batch_create(arr, len(ctxs), ctypes.byref(h)))
        self.handle = h
        self.ctxs = list(ctxs)

    def step(self, n: int):
        _check("tdb_batch_step", load().tdb_batch_step(self.handle, int(n)))

    def tuning(self):
        bn, sch, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _check("tdb_batch_tuning", load().tdb_batch_tuning(self.handle, ctypes.byref(bn),
                                                           ctypes.byref(sch), ctypes.byref(ms)))
        return {"x_bn": bn.value, "schedule": sch.value, "x_ms": ms.value}

    def close(self):
        if self.handle:
            load().tdb_batch_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def tdb_observables(ctx: Context, charges=True, forces=False):
    o = TdbObs()
    q = np.zeros(ctx.n_atoms) if charges else None
    f = np.zeros((ctx.n_atoms, 3)) if forces else None
    _check("tdb_observables", load().tdb_observables(
        ctx.handle, ctypes.byref(o), _ptr(q) if q is not None else None, _ptr(f) if f is not None else None))
    d = o.as_dict()
    if q is not None:
        d["charges"] = q
    if f is not None:
        d["forces"] = f
    return d


def tdb_dipole_history(ctx: Context, cap: int) -> np.ndarray:
    out = np.zeros((cap, 3))
    n = ctypes.c_long()
    _check("tdb_dipole_history", load().tdb_dipole_history(ctx.handle, _ptr(out), int(cap), ctypes.byref(n)))
    return out[:n.value]


def tdb_get_rho(ctx: Context, prev=False):
    N = ctx.n_orb
    re, im = np.zeros((N, N)), np.zeros((N, N))
    pre = np.zeros((N, N)) if prev else None
    pim = np.zeros((N, N)) if prev else None
    _check("tdb_get_rho", load().tdb_get_rho(ctx.handle, _ptr(re), _ptr(im),
                                            _ptr(pre) if prev else None, _ptr(pim) if prev else None))
    rho = re + 1j * im
    return (rho, pre + 1j * pim) if prev else rho


def tdb_state_bytes(ctx: Context) -> int:
    return int(load().tdb_state_bytes(ctx.handle))


def tdb_get_state(ctx: Context) -> bytes:
    n = tdb_state_bytes(ctx)
    buf = ctypes.create_string_buffer(n)
    _check("tdb_get_state", load().tdb_get_state(ctx.handle, buf, n))
    return buf.raw


def tdb_set_state(ctx: Context, blob: bytes):
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check("tdb_set_state", load().tdb_set_state(ctx.handle, buf, len(blob)))


def tdb_check(ctx: Context, tol_trace: float = 1e-10):
    _check("tdb_check", load().tdb_check(ctx.handle, float(tol_trace)))


def tdb_wait_probe(ctx: Context, polls: int):
    """Enqueue a kernel whose bounded device wait runs out (failure-detection probe)."""
    _check("tdb_wait_probe", load().tdb_wait_probe(ctx.handle, int(polls)))


def tdb_set_x_tile(ctx: Context, width: int):
    """Fix the X product's tile width (128, 176, 256), or 0 to time the candidates."""
    _check("tdb_set_x_tile", load().tdb_set_x_tile(ctx.handle, int(width)))


def tdb_x_tile(ctx: Context) -> int:
    return int(load().tdb_x_tile(ctx.handle))


def tdb_last_launch_count(ctx: Context) -> int:
    return int(load().tdb_last_launch_count(ctx.handle))


def tdb_step_profiled(ctx: Context, cap: int = 32):
    """One step with per-kernel CUDA-event timing: returns [(kernel name, ms), ...]."""
    ms = np.zeros(cap)
    names = (ctypes.c_char_p * cap)()
    n = ctypes.c_int()
    _check("tdb_step_profiled", load().tdb_step_profiled(ctx.handle, _ptr(ms), names, cap, ctypes.byref(n)))
    return [(names[i].decode(), float(ms[i])) for i in range(n.value)]


def tdb_split_gemm(A, B, fmt=0):
    """C = A @ B on the tensor-core split GEMM; returns (C, kernel ms)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    M, K = A.shape
    K2, N = B.shape
    assert K == K2
    C = np.zeros((M, N))
    ms = ctypes.c_double()
    _check("tdb_split_gemm", load().tdb_split_gemm(M, N, K, _ptr(A), _ptr(B), int(fmt), _ptr(C), ctypes.byref(ms)))
    return C, ms.value


def tdb_slice_gemm(A, B):
    """C = A @ B with FP64-accurate integer-slice tensor-core products; returns (C, kernel ms)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    M, K = A.shape
    K2, N = B.shape
    assert K == K2
    C = np.zeros((M, N))
    ms = ctypes.c_double()
    _check("tdb_slice_gemm", load().tdb_slice_gemm(M, N, K, _ptr(A), _ptr(B), _ptr(C), ctypes.byref(ms)))
    return C, ms.value


def tdb_split_gemm_noalloc(M, N, K, a_ptr, b_ptr, fmt, c_ptr, stream=None):
    """C = A B with caller-owned device buffers (raw pointers); allocates nothing.
    Returns without synchronising ``stream``."""
    _check("tdb_split_gemm_noalloc", load().tdb_split_gemm_noalloc(
        int(M), int(N), int(K), a_ptr, b_ptr, int(fmt), c_ptr, stream))


def tdb_damped_transform(x, dt: float, t_damp: float, omega):
    """F_s(w) = dt sum_n x_s[n] exp(-n dt / t_damp) exp(i w n dt) on the GPU.  x: [nsig, K] (or
    [K]); t_damp = inf or 0 for none.  Returns complex [nsig, nw] (or [nw])."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    one = x.ndim == 1
    x2 = x.reshape(1, -1) if one else x.reshape(-1, x.shape[-1])
    om = np.ascontiguousarray(omega, dtype=np.float64).ravel()
    re = np.zeros((x2.shape[0], om.size))
    im = np.zeros_like(re)
    td = 0.0 if not np.isfinite(t_damp) else float(t_damp)
    _check("tdb_damped_transform", load().tdb_damped_transform(
        int(x2.shape[0]), int(x2.shape[1]), _ptr(x2), float(dt), td, int(om.size), _ptr(om),
        _ptr(re), _ptr(im)))
    out = re + 1j * im
    return out[0] if one else out.reshape(x.shape[:-1] + (om.size,))


def tdb_destroy(ctx: Context):
    if ctx.handle:
        load().tdb_destroy(ctx.handle)
        ctx.handle = ctypes.c_void_p()


def tdb_status_string(status: int) -> str:
    return load().tdb_status_string(int(status)).decode()


def tdb_last_error() -> str:
    return load().tdb_last_error().decode()


# ---------------------------------------------------------------------------
# convenience wrapper (marshalling only)
# ---------------------------------------------------------------------------

class Propagator:
    """One trajectory: create -> ground state -> (kick) -> step ... -> observables."""

    def __init__(self, sysm, run, precision="fp64", stream=None, workspace=None, history_cap=65536,
                 window=100):
        self.sysm, self.run = sysm, run
        self.params = make_params(run, precision, stream, history_cap, window)
        self.ctx = tdb_create(sysm, self.params, workspace)

    def setup(self):
        it, res = tdb_ground_state(self.ctx)
        if self.run.field is not None:
            tdb_set_field(self.ctx, self.run.field)
        if self.run.kick:
            tdb_kick(self.ctx, self.run.kick, self.run.kick_dir)
        return it, res

    def step(self, n):
        tdb_step(self.ctx, n)

    def observables(self, **kw):
        return tdb_observables(self.ctx, **kw)

    def close(self):
        tdb_destroy(self.ctx)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
