"""Benchmark: steps/s of the density-matrix propagation step on one GB300.

Workload (default): SCC frozen-nuclei hexagonal flake, 256 atoms x 4 orbitals
(N = 1024), half filling, delta kick 1e-3 a.u. along x, dt = 0.2 a.u.  A step
is one pass of the whole hot path: Mulliken charges, SCC potential and
dipole, M = S^-1 H, X = M rho, leapfrog update (eq:leapfrog, eq:eomrho).

The headline value is the reduced-precision form (the fastest form built);
the FP64 form runs on the same trajectory as the accuracy reference (it is
itself pinned to the CPU oracle by the parity tests) and as the speed
baseline.  One JSON line is printed by rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "steps/s at N=1024/2048 orbitals: mixed-precision vs FP64 at fixed dipole error"
WORKLOAD = ("SCC frozen-nuclei hexagonal flake, 256 atoms x 4 orbitals (N=1024), "
            "half filling, kick 1e-3 a.u. along x, dt=0.2 a.u.")
L2_FLUSH_BYTES = 256 << 20

# algorithmic FLOPs per launch of each kernel of a frozen-nuclei step, as a function of N.
# The method's products per step are M = S^-1 H (2N^3, real) and X = M rho (4N^3, real
# times complex); rho H S^-1 = X^dagger is read transposed, so a step is 6N^3.  The reduced
# forms evaluate X as dM rho_ref + M Re(rho - rho_ref) + i M Im rho (6N^3 executed): the
# extra dM rho_ref part comes from the deviation form and is not counted as method work.
KERNEL_FLOPS = {
    "gemm_M_f64": lambda N: 2 * N ** 3,
    "gemm_Xre_f64": lambda N: 2 * N ** 3,
    "gemm_Xim_f64": lambda N: 2 * N ** 3,
    "gemm_dM_f32": lambda N: 2 * N ** 3,
    "gemm_Xre_f32": lambda N: 2 * N ** 3,
    "gemm_Xim_f32": lambda N: 2 * N ** 3,
    # tensor-core split GEMMs: algorithmic flops (the split products execute 3x or 6x this)
    "tc_gemm_dM": lambda N: 2 * N ** 3,
    "tc_gemm_X": lambda N: 4 * N ** 3,
    # integer-slice products (21 slice products each)
    "oz_gemm_M": lambda N: 2 * N ** 3,
    "oz_gemm_X": lambda N: 4 * N ** 3,
}
STEP_FLOPS = lambda N: 6 * N ** 3   # noqa: E731  (M and X of one step)
# algorithmic bytes per launch of the O(N^2) kernels and of the tensor-core products'
# operands (16-bit pieces read once, outputs written once)
KERNEL_BYTES = {
    # reads X (re, im; both halves once), rho_{n-1}, S; writes rho_{n+1} (+ operands)
    "update_f64": lambda N: N * N * 8 * (2 + 2 + 1 + 2),
    # reduced forms update the FP32-pair master of rho - rho_ref: read X (2 x f32), the
    # base master (4 x f32) and S (f32), write the new master (4 x f32) ...
    "update_f32": lambda N: N * N * (4 * 2 + 4 * 4 + 4 + 4 * 4),
    # ... and the operand pieces (hi/lo: 4 x 16 bit)
    "update_tc": lambda N: N * N * (4 * 2 + 4 * 4 + 4 + 4 * 4 + 2 * 4),
    # ... FP16X6: X has a third FP32 part, 6 x 16-bit pieces
    "update_fp16x6": lambda N: N * N * (4 * 3 + 4 * 4 + 4 + 4 * 4 + 2 * 6),
    # reads S (f32) and writes the pieces of delta H (2 or 3 x 16 bit)
    "split_dH": lambda N: N * N * (4 + 2 * 2),
    "split_dH_fp16x6": lambda N: N * N * (4 + 2 * 3),
    # FP16X6 delta M: reads 3 pieces of S^-1 and of delta H and M_gs (f32), writes the
    # 3 pieces of delta M and of M_gs + delta M
    "tc_gemm_dM_fp16x6": lambda N: N * N * (2 * 3 + 2 * 3 + 4 + 2 * 6),
    # FP16X6 X: reads 3 pieces of [dM | M] (2N columns) and of [rho_ref | Re drho] (2N)
    # and of -Im rho (N), writes three FP32 partial products
    "tc_gemm_X_fp16x6": lambda N: N * N * (2 * 3 * 2 + 2 * 3 * 2 + 2 * 3 + 4 * 3),
}


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch of a kernel from
# one ncu capture of the bench workload (N = 1024 flake, FP16X6, X tiles 176 wide, ncu's
# default cache control: every launch starts from a flushed L2, so a product's traffic
# includes the lines it prefetches for the next kernel and the next kernel's traffic does
# not profit from them).  An entry holds while the kernel's source files are byte-identical
# to the ones captured (sha256); otherwise the bench reports traffic as null.
_TC = ("paper_1912_03174_gb300/csrc/kern_tc.cu", "c3cb02abd3c1cfa1c50e7e74abb6cf13ecaf276604e4cf806ed2d5ebabdafa6f")
_ST = ("paper_1912_03174_gb300/csrc/kern_step.cu", "4047e2d09196f7fe91eed8888acb921e008f116d925834a93b0482ff1ca0fe4e")
_API = ("paper_1912_03174_gb300/csrc/tdb_api.cu", "967fde2a7f0ef345f223c57b3fc52b4923160094c02ab92db6f1ac7aba39a1aa")
PROFILED_TRAFFIC: dict = {
    ("tc_gemm_X", "fp16x6"): {"bytes": 52518400, "sources": [_TC, _API]},
    ("tc_gemm_dM", "fp16x6"): {"bytes": 42322432, "sources": [_TC, _API]},
    ("split_dH", "fp16x6"): {"bytes": 4207104, "sources": [_TC, _API]},
    ("update", "fp16x6"): {"bytes": 33682944, "sources": [_ST, _API]},
}


def _traffic(name: str, form: str):
    e = PROFILED_TRAFFIC.get((name, form))
    if not e:
        return None
    import hashlib
    for path, sha in e["sources"]:
        try:
            with open(os.path.join(ROOT, path), "rb") as fh:
                if hashlib.sha256(fh.read()).hexdigest() != sha:
                    return None
        except OSError:
            return None
    return e["bytes"]


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


# cuBLAS rates measured on a GB300 with `bench.py --measure-peaks` (n = 8192): context
# for the SIMT forms' ALU roofline.
CUBLAS_TFLOPS = {"f64": 1.072, "f32": 69.7, "tf32": 1050.5}


def alu_peak_tflops(kind: str, sm_mhz: float) -> float:
    """SIMT peaks from unit counts: 152 SMs x 128 FP32 lanes x 2 flop/FMA x clock;
    FP64 at the GB300 nominal 1.25 TFLOP/s (its FP64 units are 1/64 of FP32)."""
    if kind == "f32":
        return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
    return 1.25


def measure_peaks(torch, n=8192):
    """cuBLAS GEMM rates on this GPU (TFLOP/s at n x n x n, CUDA events): FP64 (DGEMM),
    FP32 with TF32 off (SGEMM) and TF32 — the denominators that the measured-peaks file
    does not carry, for the SIMT FP64 and FP32 forms."""
    out = {}
    for name, dt, tf32, reps in (("fp64", torch.float64, False, 3), ("fp32", torch.float32, False, 10),
                                 ("tf32", torch.float32, True, 20)):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        g = torch.Generator(device="cuda").manual_seed(7)
        a = torch.randn(n, n, dtype=dt, device="cuda", generator=g)
        b = torch.randn(n, n, dtype=dt, device="cuda", generator=g)
        c = torch.empty(n, n, dtype=dt, device="cuda")
        torch.matmul(a, b, out=c)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            torch.matmul(a, b, out=c)
        e1.record()
        torch.cuda.synchronize()
        out[name + "_tflops"] = 2.0 * n ** 3 * reps / (e0.elapsed_time(e1) * 1e-3) / 1e12
        del a, b, c
    torch.backends.cuda.matmul.allow_tf32 = False
    return out


class ClockSampler:
    """nvidia-smi samples during the timed region (clocks and throttle reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = [r.split(",") for r in (getattr(self, "out", "") or "").strip().splitlines() if r.strip()]
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


TENSOR_FORMS = ("bf16x3", "fp16x3", "fp16x6")


def run_form(B, torch, sysm, run, precision, steps, warmup, flush, stream, x_tile=0):
    """Ground state + kick, W warm-up steps, K timed steps (per-step events, L2
    flushed between them).  Returns timing and the dipole trajectory.  x_tile: the X
    product's tile width of the tensor-core forms (0: timed at the first step)."""
    p = B.Propagator(sysm, run, precision, stream=stream.cuda_stream, history_cap=warmup + steps + 8)
    try:
        if x_tile and precision in TENSOR_FORMS:
            B.tdb_set_x_tile(p.ctx, x_tile)
        p.setup()
        with torch.cuda.stream(stream):
            p.step(warmup)
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(steps)]
            launches = 0
            for k in range(steps):
                flush.add_(1.0)                         # > L2: evicts the working set
                ev[k][0].record(stream)
                p.step(1)
                ev[k][1].record(stream)
                launches += B.tdb_last_launch_count(p.ctx)
            torch.cuda.synchronize()
        ms = [a.elapsed_time(b) for a, b in ev]
        hist = B.tdb_dipole_history(p.ctx, warmup + steps)
        # per-kernel times (events between the kernels of a step, same stream)
        prof = {}
        for _ in range(10):
            flush.add_(1.0)
            torch.cuda.synchronize()
            for name, t in B.tdb_step_profiled(p.ctx):
                prof.setdefault(name, []).append(t)
        obs = p.observables()
        tile = B.tdb_x_tile(p.ctx)
    finally:
        p.close()
    return dict(ms=ms, hist=hist, prof={k: float(np.mean(v)) for k, v in prof.items()}, obs=obs,
                launches=launches, x_tile=tile)


def form_summary(res: dict, forms, n_electrons: float) -> dict:
    """Per form: steps/s, and against the FP64 form (when it ran) the largest dipole
    error over the run and the charge error at its end; the relative trace drift
    |Tr(rho S) - N_e| / N_e and the Hermiticity error at the end."""
    ref = res.get("fp64")
    out = {}
    for f in forms:
        r = res[f]
        o = r["obs"]
        out[f] = {
            "steps_per_s": 1000.0 / float(np.mean(r["ms"])),
            "max_dipole_err_vs_fp64_au": (float(np.max(np.abs(r["hist"] - ref["hist"])))
                                          if ref is not None else None),
            "final_charge_err_vs_fp64": (float(np.max(np.abs(np.asarray(o["charges"])
                                                             - np.asarray(ref["obs"]["charges"]))))
                                         if ref is not None else None),
            "trace_rel_drift": abs(float(o["trace_re"]) - n_electrons) / n_electrons,
            "herm_err": float(o["herm_err"]),
        }
    return out


def replica_timing(ms_step: float, world: int, dist=None):
    """Replicas only: every rank propagates its own copy of the workload, with no
    data-path collective.  The slowest rank's time per step sets the pace (a max over
    ranks on the host, gloo) and the whole-job value is world x its steps/s."""
    if dist is not None:
        import torch
        t = torch.tensor([ms_step], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
    return ms_step, world * 1000.0 / ms_step


def n2048_runs(B, torch, flush, stream, reduced_steps):
    """The N = 2048 points of the metric, reported beside the N = 1024 headline:
    a 512-atom flake with frozen nuclei in every form (dipole error of each form
    against the FP64 form over the FP64 form's steps), and the c3 Ehrenfest cluster
    (512 atoms, 300 K, laser) in the FP64 form, the one that moves nuclei."""
    from paper_1912_03174_gb300 import inputs as I
    sysm = I.small_flake(512, seed=1012)
    run = I.Run(dt=0.2, n_steps=0, scc=True, kick=1e-3, kT=I.SCC_KT)
    out = {"frozen": {"workload": "SCC frozen-nuclei hexagonal flake, 512 atoms (N=2048), "
                                  "kick 1e-3 a.u. along x, dt=0.2 a.u.", "forms": {}}}
    res = {}
    for f, k in (("fp64", 20), ("fp64s", 60), ("fp16x3", reduced_steps), ("fp16x6", reduced_steps)):
        res[f] = run_form(B, torch, sysm, run, f, k, 3, flush, stream)
    n64 = len(res["fp64"]["hist"])
    for f, r in res.items():
        out["frozen"]["forms"][f] = {
            "steps_per_s": 1000.0 / float(np.mean(r["ms"])), "timed_steps": len(r["ms"]),
            "max_dipole_err_vs_fp64_au": float(np.max(np.abs(r["hist"][:n64] - res["fp64"]["hist"]))),
            "compared_steps": n64}
    sysm3, run3 = I.cluster_c3()
    r3 = {f: run_form(B, torch, sysm3, run3, f, 5, 3, flush, stream) for f in ("fp64", "fp64s", "fp32")}
    out["ehrenfest_c3"] = {
        "workload": "Ehrenfest cluster, 512 atoms (N=2048), 300 K, Gaussian laser E0=0.01 "
                    "omega=0.1, dt=0.2 a.u.",
        "forms": {f: {"steps_per_s": 1000.0 / float(np.mean(r["ms"])), "timed_steps": len(r["ms"]),
                      "max_dipole_err_vs_fp64_au": float(np.max(np.abs(r["hist"] - r3["fp64"]["hist"]))),
                      "phase_ms": r["prof"]}
                  for f, r in r3.items()},
        "note": "moving nuclei run in the FP64, FP64-sliced (integer-slice tensor-core products) "
                "and FP32 forms; density, forces and update in FP64"}
    return out


def c4_runs(B, torch, n_traj, post_steps, form="fp16x6"):
    """Batched pump-probe scan (probe runs branched from pump runs, Sec. 3.2): four flakes
    (N = 128..1024), each probe a clone of its size's pump run at its delay tau (rounded to
    the step grid), kicked 1e-3 a.u. along x.  Pump runs, branching, the Euler step and the
    batch's autotuning and graph capture are untimed.  Timed (host clock between
    device-wide synchronisations, the probes run on many streams): every probe advancing
    post_steps steps as one grouped batch (every phase one launch over all probes), then
    stream-interleaved (tdb_step_batch), then one probe after another.  The FP64 form runs
    the probe with the shortest delay of each size (pump and probe) for the dipole error of
    the FP16X6 probes and the FP64 time per step of each size."""
    import dataclasses
    from paper_1912_03174_gb300 import inputs as I
    systems, run, which, tau = I.pump_probe_c4(n_traj=n_traj)
    pump_run = dataclasses.replace(run, kick=0.0)
    probes, meta = [], []
    pump_steps = 0
    for s_idx, sysm in enumerate(systems):
        idx = np.where(which == s_idx)[0]
        if len(idx) == 0:
            continue
        steps = np.rint(tau[idx] / run.dt).astype(np.int64)
        with B.Propagator(sysm, pump_run, form) as p:
            p.setup()
            at = 0
            for st in np.sort(steps):
                B.tdb_step(p.ctx, int(st - at))
                at = int(st)
                c = B.tdb_clone(p.ctx)
                B.tdb_kick(c, run.kick, run.kick_dir)
                probes.append(c)
                meta.append((s_idx, int(st)))
            pump_steps += at
    total = 1 + 3 * post_steps
    try:
        batch = B.Batch(probes)
        try:
            batch.step(1)                               # Euler step, context by context
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            batch.step(post_steps)
            torch.cuda.synchronize()
            t_group = time.perf_counter() - t0
            tuning = batch.tuning()
        finally:
            batch.close()
        t0 = time.perf_counter()
        B.tdb_step_batch(probes, post_steps)
        torch.cuda.synchronize()
        t_stream = time.perf_counter() - t0
        t0 = time.perf_counter()
        for c in probes:
            B.tdb_step(c, post_steps)
            torch.cuda.synchronize()
        t_seq = time.perf_counter() - t0
        # FP64 check: the shortest-delay probe of each size, pump and probe in the FP64 form
        check = {}
        for s_idx, sysm in enumerate(systems):
            mine = [i for i, m in enumerate(meta) if m[0] == s_idx]
            if not mine:
                continue
            i = min(mine, key=lambda j: meta[j][1])
            with B.Propagator(sysm, pump_run, "fp64", history_cap=meta[i][1] + total + 8) as p:
                p.setup()
                B.tdb_step(p.ctx, meta[i][1])
                c = B.tdb_clone(p.ctx)
                try:
                    B.tdb_kick(c, run.kick, run.kick_dir)
                    B.tdb_step(c, 1)
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    B.tdb_step(c, total - 1)
                    torch.cuda.synchronize()
                    t64 = (time.perf_counter() - t0) / (total - 1)
                    h64 = B.tdb_dipole_history(c, total)
                finally:
                    B.tdb_destroy(c)
            h16 = B.tdb_dipole_history(probes[i], total)
            check[int(sysm.n_orb)] = {"delay_steps": meta[i][1],
                                      "max_dipole_err_vs_fp64_au": float(np.max(np.abs(h16 - h64))),
                                      "fp64_ms_per_step": 1000.0 * t64, "compared_steps": total}
    finally:
        for c in probes:
            B.tdb_destroy(c)
    units = len(probes) * post_steps
    sizes = [int(systems[m[0]].n_orb) for m in meta]
    t_fp64 = sum(post_steps * check[n]["fp64_ms_per_step"] * 1e-3 for n in sizes if n in check)
    return {"workload": f"pump-probe scan: {len(probes)} probe runs over flakes of "
                        f"{'/'.join(str(s.n_atoms) for s in systems)} atoms (N = 128..1024), "
                        f"laser pump E0=0.01 omega=0.1, probe kick 1e-3 at tau ~ U(0, 200 fs), "
                        f"dt=0.2, {post_steps} post-kick steps timed per probe",
            "precision": form, "probes": len(probes), "pump_steps_untimed": int(pump_steps),
            "sizes": sizes,
            "trajectory_steps_per_s_batched": units / t_group,
            "trajectory_steps_per_s_stream_interleaved": units / t_stream,
            "trajectory_steps_per_s_one_by_one": units / t_seq,
            "grouped_speedup_over_one_by_one": t_seq / t_group,
            "grouped_speedup_over_stream_interleaved": t_stream / t_group,
            "autotuner": tuning,
            "fp64_check": check,
            "fp64_trajectory_steps_per_s_estimate": units / t_fp64 if t_fp64 > 0 else None,
            "speedup_over_fp64": t_fp64 / t_group if t_fp64 > 0 else None,
            "max_dipole_err_vs_fp64_au": max((v["max_dipole_err_vs_fp64_au"] for v in check.values()),
                                             default=None),
            "timing": "host clock between device-wide synchronisations; FP64: the probe's steps "
                      "timed per size and summed over the scan's size mix"}


def c4_fractions(c4: dict, peaks: dict) -> None:
    """HBM and tensor fractions of the batched scan: the mean probe step's algorithmic bytes
    (FP16X6 step bytes at its N) and method flops (6 N^3) times the probe steps per second."""
    if not c4 or c4.get("precision") != "fp16x6" or "sizes" not in c4:
        return
    sizes = np.asarray(c4["sizes"], dtype=np.float64)
    rate = c4["trajectory_steps_per_s_batched"]
    b = float(np.mean([step_bytes("fp16x6", int(n)) for n in sizes]))
    f = float(np.mean([STEP_FLOPS(int(n)) for n in sizes]))
    c4["roofline"] = {"bytes_per_traj_step": b, "flops_per_traj_step": f,
                      "achieved_gbs": b * rate / 1e9, "hbm_frac": b * rate / 1e9 / peaks["hbm_gbs"],
                      "achieved_tflops": f * rate / 1e12,
                      "tensor_frac": f * rate / 1e12 / peaks["bf16_tflops"],
                      "note": "bytes: FP16X6 step arrays read or written once; flops: the method's "
                              "M and X products"}


def c5_runs(B, torch, k=16, L=8, hidden=64, n_train=4, train_steps=1200, windows=12,
            epochs=20, form="fp64s"):
    """The learned form on the 256-atom flake (N = 1024): shift and charge records of
    n_train plain runs (kicks of seeded strength 1e-3..3e-3 a.u. along seeded directions)
    train the per-atom network (L shift and L charge samples at window ends, two hidden
    layers of `hidden`, BF16 weights) on the GPU; a held-out run (the flake's own kick, 1e-3 a.u. along x)
    then advances in windows of k steps with the network's shift, with the shift frozen
    at the window's start, and in plain steps.  Reported: data and training time, time
    per window against k plain steps, and the charge and dipole errors at window ends
    against the plain run."""
    import dataclasses
    from paper_1912_03174_gb300 import inputs as I, learned as Lrn
    sysm, run = I.flake_c2()
    rng = np.random.default_rng(1005)
    Xs, Ys = [], []
    t0 = time.perf_counter()
    for _ in range(n_train):
        d = rng.normal(size=3)
        r = dataclasses.replace(run, kick=float(rng.uniform(1e-3, 3e-3)), kick_dir=d / np.linalg.norm(d))
        with B.Propagator(sysm, r, form) as p:
            p.setup()
            p.step(1)
            X, Y = Lrn.training_set(Lrn.record(p.ctx, train_steps), k, L)
            Xs.append(X)
            Ys.append(Y)
    t_data = time.perf_counter() - t0
    X, Y = np.concatenate(Xs), np.concatenate(Ys)
    model = Lrn.ShiftModel(k=k, L=L, hidden=hidden, seed=5)
    t0 = time.perf_counter()
    model.fit(X, Y, epochs=epochs, batch=512, lr=2e-3)
    t_train = time.perf_counter() - t0

    def start():
        p = B.Propagator(sysm, run, form)
        p.setup()
        p.step(1)
        return p

    out = {}
    # plain reference: warm-up windows, then `windows` windows of k plain steps
    p = start()
    try:
        p.step(L * k)
        q_ref, mu_ref, t_plain = [], [], []
        for _ in range(windows):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            torch.cuda.nvtx.range_push("c5_plain")
            B.tdb_step(p.ctx, k)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
            t_plain.append(time.perf_counter() - t0)
            o = p.observables()
            q_ref.append(o["charges"])
            mu_ref.append(o["dipole"])
    finally:
        p.close()
    q_ref, mu_ref = np.array(q_ref), np.array(mu_ref)
    for mode in ("frozen", "net"):
        p = start()
        try:
            lp = Lrn.LearnedPropagator(p.ctx, model, mode=mode)
            lp.warm_up()
            q, mu, t_win = [], [], []
            for _ in range(windows):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                torch.cuda.nvtx.range_push(f"c5_window_{mode}")
                lp.run(1)
                torch.cuda.synchronize()
                torch.cuda.nvtx.range_pop()
                t_win.append(time.perf_counter() - t0)
                o = p.observables()
                q.append(o["charges"])
                mu.append(o["dipole"])
        finally:
            p.close()
        eq = np.max(np.abs(np.array(q) - q_ref), axis=1)
        emu = np.max(np.abs(np.array(mu) - mu_ref), axis=1)
        out[mode] = {"max_charge_err": float(eq.max()), "final_charge_err": float(eq[-1]),
                     "max_dipole_err_au": float(emu.max()), "final_dipole_err_au": float(emu[-1]),
                     "ms_per_window": 1000.0 * float(np.median(t_win[1:] or t_win))}
    # the referee at the stated dipole bound, every fourth window
    p = start()
    try:
        lp = Lrn.LearnedPropagator(p.ctx, model, mode="net", referee_every=4, bound=float("inf"),
                                   dipole_bound=1e-5)
        lp.warm_up()
        lp.run(windows)
        st = lp.stats
        referee = {"dipole_bound_au": 1e-5, "referee_every": 4, "windows_run": st.windows,
                 "refereed": st.refereed, "taken_over": st.taken_over,
                 "plain_steps_after_warm_up": st.plain_steps - L * k,
                 "referee_dipole_err_au": st.referee_dipole_err, "referee_charge_err": st.referee_err}
    finally:
        p.close()
    model.close()
    ms_plain = 1000.0 * float(np.median(t_plain))
    ms_win = out["net"]["ms_per_window"]
    return {"workload": f"learned form on the SCC flake, 256 atoms (N=1024), form {form}: "
                        f"{n_train} training runs x {train_steps} steps, held-out kick 1e-3 a.u. along x, "
                        f"windows of k={k} steps (dt=0.2), {windows} windows after {L} plain warm-up windows",
            "training": {"samples": int(len(Y)), "epochs": epochs, "data_s": t_data, "train_s": t_train,
                         "samples_per_s": epochs * len(Y) / t_train,
                         "final_loss_scaled": float(model.losses[-1])},
            "ms_k_plain_steps": ms_plain, "ms_per_window": ms_win,
            "effective_steps_per_s_window": 1000.0 * k / ms_win,
            "steps_per_s_plain": 1000.0 * k / ms_plain,
            "window_vs_plain_speedup": ms_plain / ms_win,
            "errors_vs_plain": out,
            "referee": referee,
            "gain_charge_err_frozen_over_net": out["frozen"]["max_charge_err"] / max(out["net"]["max_charge_err"], 1e-300),
            "timing": "host clock between device synchronisations (window: shift readback, "
                      "network inference, eigensolve and products)"}


def c5_k_sweep(B, ks=(2, 4, 8, 16, 32, 64), forms=("fp64s", "fp64"), warm=129):
    """The learned form's floor and cost against the window length k on the 256-atom flake
    (N = 1024): from one state (warm plain steps after the kick), a clone takes k plain steps
    (timed), another records the SCC shift at each of those steps, and a third takes one
    closed-form window with the exact window-mean shift (the best any predictor can give,
    timed) and one with the shift frozen at the window's start.  Errors are the dipole and
    charge differences to the plain steps at the window's end.  break_even_k: the window
    length at which one window costs as much as k plain steps."""
    from paper_1912_03174_gb300 import inputs as I, learned as Lrn
    sysm, run = I.flake_c2()
    out = {}
    for form in forms:
        rows = []
        with B.Propagator(sysm, run, form) as p:
            p.setup()
            p.step(warm)
            for k in ks:
                c = B.tdb_clone(p.ctx)
                try:
                    B.tdb_step(c, 1)                    # graph capture outside the timing
                    B.tdb_set_state(c, B.tdb_get_state(p.ctx))
                    t0 = time.perf_counter()
                    B.tdb_step(c, k)
                    o_plain = B.tdb_observables(c)
                    t_plain = time.perf_counter() - t0
                finally:
                    B.tdb_destroy(c)
                a = B.tdb_clone(p.ctx)
                try:
                    vs = []
                    for _ in range(k):
                        vs.append(Lrn.sample(a)[:, 0])
                        B.tdb_step(a, 1)
                finally:
                    B.tdb_destroy(a)
                res = {}
                for mode, vbar in (("exact_mean_shift", np.mean(vs, axis=0)), ("frozen_shift", vs[0])):
                    b = B.tdb_clone(p.ctx)
                    try:
                        t0 = time.perf_counter()
                        B.tdb_step_window(b, vbar, k)
                        o = B.tdb_observables(b)
                        t_win = time.perf_counter() - t0
                    finally:
                        B.tdb_destroy(b)
                    res[mode] = {"dipole_err_au": float(np.max(np.abs(np.asarray(o["dipole"])
                                                                       - np.asarray(o_plain["dipole"])))),
                                 "charge_err": float(np.max(np.abs(o["charges"] - o_plain["charges"]))),
                                 "window_ms": 1000.0 * t_win}
                rows.append({"k": k, "plain_ms": 1000.0 * t_plain, **res})
        per_step = float(np.median([r["plain_ms"] / r["k"] for r in rows]))
        win = float(np.median([r["exact_mean_shift"]["window_ms"] for r in rows]))
        out[form] = {"rows": rows, "plain_ms_per_step": per_step, "window_ms": win,
                     "break_even_k": win / per_step}
    return {"workload": "SCC flake, 256 atoms (N=1024), kick 1e-3 a.u. along x, windows from the "
                        f"state {warm} steps after the kick", "forms": out,
            "timing": "host clock, each call synchronised (plain steps include the observables "
                      "read-back, as the windows do)"}


def shard_throughput(units: float, seconds: float, dist=None):
    """Sharded independent work (each rank its own share, no data-path collective):
    the whole job's units over the slowest rank's time, both reduced over ranks on the
    host (gloo).  Returns (total units, max seconds, units per second)."""
    if dist is not None:
        import torch
        u = torch.tensor([float(units)], dtype=torch.float64)
        t = torch.tensor([float(seconds)], dtype=torch.float64)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        units, seconds = float(u.item()), float(t.item())
    return units, seconds, (units / seconds if seconds > 0 else 0.0)


def c4_sharded(B, torch, dist, rank, world, n_traj, post_steps, form="fp16x6"):
    """The pump-probe scan of c4_runs over world ranks: the probe runs shared out by
    longest-processing-time on N^3 x steps, each rank branching and stepping its own
    share (scan.run_shard), timed between barriers; value = all probe steps over the
    slowest rank's time."""
    from paper_1912_03174_gb300 import inputs as I, scan
    systems, run, which, tau = I.pump_probe_c4(n_traj=n_traj)
    parts = scan.lpt_partition(scan.probe_costs(systems, which, post_steps), world)

    def sync():
        torch.cuda.synchronize()
        dist.barrier()

    n, pump_steps, t, _ = scan.run_shard(B, systems, run, which, tau, parts[rank], post_steps,
                                         form, sync=sync)
    units, t_max, rate = shard_throughput(n * post_steps, t, dist)
    return {"workload": f"pump-probe scan: {len(which)} probe runs over flakes of "
                        f"{'/'.join(str(s.n_atoms) for s in systems)} atoms (N = 128..1024), "
                        f"shared out over {world} ranks by longest-processing-time on N^3 x steps, "
                        f"{post_steps} post-kick steps timed per probe",
            "precision": form, "probes": int(units // post_steps), "probes_this_rank": n,
            "pump_steps_untimed_this_rank": int(pump_steps),
            "trajectory_steps_per_s_batched": rate, "seconds_slowest_rank": t_max,
            "scaling": "strong",
            "timing": "host clock between barriers after device synchronisation"}


def e2e_run(B, sysm, run, precision, steps, warmup):
    """End to end through the public API, one step at a time: the field of the step is
    set from the host (H2D), the step runs, and its result, the dipole mu(t_n) of the
    history ring, is read back (D2H, which synchronises)."""
    p = B.Propagator(sysm, run, precision)
    try:
        p.setup()
        from paper_1912_03174_gb300 import inputs as I
        fld = B.make_field(I.Field(E0=0.0, omega=0.0))
        for _ in range(warmup):
            B.tdb_set_field(p.ctx, fld)
            p.step(1)
            B.tdb_dipole_history(p.ctx, 1)
        t0 = time.perf_counter()
        for _ in range(steps):
            B.tdb_set_field(p.ctx, fld)
            p.step(1)
            B.tdb_dipole_history(p.ctx, 1)
        dt = time.perf_counter() - t0
    finally:
        p.close()
    h2d = 88                                     # field parameters
    d2h = 3 * 8                                  # the step's dipole
    return {"value": steps / dt, "unit": "steps/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "per_step": "set field (H2D), one step, read its dipole back (D2H, synchronising)"}


def accuracy_c2(B, sysm, run, forms, total, sample_every=1000):
    """Run-length accuracy on the N = 1024 flake: every form runs `total` steps from the same
    kicked ground state; the dipole of every step is compared with the FP64 form's, and
    Tr(rho S) is sampled every `sample_every` steps (relative deviation from N_e)."""
    hist, drift, secs = {}, {}, {}
    for f in forms:
        t0 = time.perf_counter()
        with B.Propagator(sysm, run, f, history_cap=total + 8) as p:
            p.setup()
            worst = 0.0
            done = 0
            while done < total:
                k = min(sample_every, total - done)
                p.step(k)
                done += k
                o = p.observables(charges=False)
                worst = max(worst, abs(o["trace_re"] - sysm.n_electrons) / sysm.n_electrons)
            hist[f] = B.tdb_dipole_history(p.ctx, total)
            drift[f] = worst
        secs[f] = time.perf_counter() - t0
    out = {"workload": f"{WORKLOAD}, {total} steps per form", "steps": total, "forms": {}}
    for f in forms:
        e = float(np.max(np.abs(hist[f] - hist["fp64"]))) if "fp64" in hist else None
        out["forms"][f] = {"max_dipole_err_vs_fp64_au": e, "max_trace_rel_drift": drift[f],
                           "within_1e-6_au": (e is not None and e <= 1e-6), "wall_s": secs[f]}
    return out


def accuracy_c3(B, total, every=20, nudge=1e-12):
    """Run-length accuracy of the Ehrenfest cluster (512 atoms, N = 2048): the FP64-sliced
    form against the FP64 form over `total` steps, all advanced in lockstep; every `every`
    steps the dipole, the forces and Tr(rho S) are compared.  A third run, FP64-sliced with
    an extra kick of `nudge` a.u. at t = 0, measures how fast the dynamics itself separates
    two nearby trajectories: an arithmetic difference cannot be resolved below that
    envelope."""
    from paper_1912_03174_gb300 import inputs as I
    sysm, run = I.cluster_c3()
    t0 = time.perf_counter()
    a = B.Propagator(sysm, run, "fp64", history_cap=total + 8)
    b = B.Propagator(sysm, run, "fp64s", history_cap=total + 8)
    c = B.Propagator(sysm, run, "fp64s", history_cap=total + 8)
    series = []
    try:
        a.setup()
        b.setup()
        c.setup()
        B.tdb_kick(c.ctx, nudge, np.array([1.0, 0.0, 0.0]))
        ef, ed, tr, tr64, env_d, env_f = 0.0, 0.0, 0.0, 0.0, 0.0, 0.0
        done = 0
        while done < total:
            k = min(every, total - done)
            for p in (a, b, c):
                p.step(k)
            done += k
            oa, ob, oc = (p.observables(forces=True) for p in (a, b, c))
            e_f = float(np.max(np.abs(oa["forces"] - ob["forces"])))
            e_d = float(np.max(np.abs(np.asarray(oa["dipole"]) - np.asarray(ob["dipole"]))))
            n_f = float(np.max(np.abs(oc["forces"] - ob["forces"])))
            n_d = float(np.max(np.abs(np.asarray(oc["dipole"]) - np.asarray(ob["dipole"]))))
            ef, ed = max(ef, e_f), max(ed, e_d)
            env_f, env_d = max(env_f, n_f), max(env_d, n_d)
            tr = max(tr, abs(ob["trace_re"] - sysm.n_electrons) / sysm.n_electrons)
            tr64 = max(tr64, abs(oa["trace_re"] - sysm.n_electrons) / sysm.n_electrons)
            if done % 100 == 0 or done == total:
                series.append({"step": done, "fp64s_vs_fp64_dipole": e_d, "fp64s_vs_fp64_force": e_f,
                               "nudged_vs_fp64s_dipole": n_d, "nudged_vs_fp64s_force": n_f})
        ha, hb = B.tdb_dipole_history(a.ctx, total), B.tdb_dipole_history(b.ctx, total)
        ed = max(ed, float(np.max(np.abs(ha - hb))))
    finally:
        a.close()
        b.close()
        c.close()
    return {"workload": "Ehrenfest cluster, 512 atoms (N=2048), 300 K, Gaussian laser E0=0.01 "
                        f"omega=0.1, dt=0.2 a.u., {total} steps", "steps": total,
            "fp64s_vs_fp64": {"max_dipole_err_au": ed, "max_force_err_ha_bohr": ef,
                              "max_trace_rel_drift_fp64s": tr, "max_trace_rel_drift_fp64": tr64,
                              "force_compared_every": every},
            "separation_of_nudged_runs": {"nudge_kick_au": nudge, "max_dipole_au": env_d,
                                          "max_force_ha_bohr": env_f},
            "series": series,
            "within_bounds": ed <= 1e-6 and ef <= 1e-6, "wall_s": time.perf_counter() - t0,
            "note": "with moving nuclei S changes every step, so Tr(rho S) is conserved only "
                    "approximately by the leapfrog (its drift is reported, not bounded)"}


def cpu_baseline(sysm, run, n_steps, warmup=1, budget_s=None):
    """The CPU oracle as it stands, timed on this host's cores: ground state untimed,
    `warmup` untimed oracle steps, then n_steps timed ones (fewer when budget_s is set
    and the warm-up steps say that n_steps would take longer).  Returns (steps/s,
    warm-up steps done, steps timed)."""
    from oracle import tdb_oracle as O
    rho, gs, S, Sinv = O.setup(sysm, run)
    w = max(1, warmup)
    t0 = time.perf_counter()
    tr = O.propagate(sysm, run, rho, w)
    t_warm = (time.perf_counter() - t0) / w
    n = n_steps
    if budget_s is not None:
        n = max(1, min(n_steps, int(budget_s / max(t_warm, 1e-9))))
    t0 = time.perf_counter()
    O.propagate(sysm, run, tr.rho, n, rho_prev=tr.rho_prev, step0=w, t0=w * run.dt)
    dt = time.perf_counter() - t0
    # propagate() also evaluates observables of rho_0..rho_K: K+1 evaluations, K steps
    return n / dt, w, n


def reference_arm(args, sysm, run, rank):
    if rank != 0:
        return
    cores = len(os.sched_getaffinity(0))
    v, w, n = cpu_baseline(sysm, run, args.steps, warmup=min(args.warmup, 3), budget_s=150.0)
    sample = (f"ground state untimed, {w} untimed and {n} timed oracle steps of the same "
              f"workload ({args.steps} requested; timed steps bounded to ~150 s of oracle time)")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": n, "warmup": w, "requested_steps": args.steps, "requested_warmup": args.warmup,
            "ms_per_step": 1000.0 / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": sysm.n_orb, "parallelism": "replicas"},
            "cpu_baseline": {"value": v, "unit": "steps/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def kernel_roofline(name: str, t_ms: float, form: str, N: int, peaks: dict, src: str) -> dict:
    """Roofline entry of one kernel of a frozen-nuclei step: algorithmic flops (tensor or
    ALU bound) or bytes (HBM bound) per launch over its mean event time."""
    if name.startswith(("tc_gemm", "oz_gemm")):
        ach = KERNEL_FLOPS[name](N) / (t_ms * 1e-3) / 1e12
        peak = peaks["bf16_tflops"]
        products = {"bf16x3": 3, "fp16x3": 3, "fp16x6": 6, "fp64s": 21}.get(form, 3)
        executed = {"tc_gemm_X": 6 * N ** 3}.get(name, KERNEL_FLOPS[name](N)) * products
        out = {"kernel": name, "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
               "frac": ach / peak, "traffic": _traffic(name, form),
               "peak_source": f"{src} dense bf16 burst (fp16 runs at the same rate)",
               "executed_tflops": executed / (t_ms * 1e-3) / 1e12,
               "executed_frac": executed / (t_ms * 1e-3) / 1e12 / peak,
               "note": f"achieved counts the method's flops ({KERNEL_FLOPS[name](N):.3g} per launch); "
                       f"executed counts {products} tensor-core products per algorithmic product"
                       + (" and the deviation form's extra dM rho_ref part" if name == "tc_gemm_X" else "")}
        key = f"{name}_fp16x6"
        if form == "fp16x6" and key in KERNEL_BYTES:
            gbs = KERNEL_BYTES[key](N) / (t_ms * 1e-3) / 1e9
            out["operand_gbs"] = gbs
            out["operand_hbm_frac"] = gbs / peaks["hbm_gbs"]
        return out
    if name in KERNEL_FLOPS:
        kind = "f64" if name.endswith("f64") else "f32"
        ach = KERNEL_FLOPS[name](N) / (t_ms * 1e-3) / 1e12
        peak = alu_peak_tflops(kind, peaks.get("sm_max_mhz", 2070.0))
        return {"kernel": name, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": None,
                "peak_source": f"derived from unit counts at {peaks.get('sm_max_mhz', 2070.0):.0f} MHz"
                if kind == "f32" else "GB300 nominal FP64 1.25 TFLOP/s",
                "cublas_tflops": CUBLAS_TFLOPS[kind], "frac_of_cublas": ach / CUBLAS_TFLOPS[kind]}
    key = None
    if name == "update":
        key = {"fp64": "update_f64", "fp64s": "update_f64", "fp32": "update_f32",
               "fp16x6": "update_fp16x6"}.get(form, "update_tc")
    elif name == "split_dH":
        key = "split_dH_fp16x6" if form == "fp16x6" else "split_dH"
    if key is None:
        return {"kernel": name, "bound": "latency", "time_us": 1000.0 * t_ms,
                "note": "O(N_atoms^2) work: bound by launch and reduction latency, not by a unit"}
    ach = KERNEL_BYTES[key](N) / (t_ms * 1e-3) / 1e9
    return {"kernel": name, "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": ach / peaks["hbm_gbs"], "traffic": _traffic(name, form), "peak_source": src}


def step_bytes(form: str, N: int) -> int:
    """Algorithmic HBM bytes of one frozen-nuclei step of a tensor-core form: every
    O(N^2) array and operand piece array read or written once (charges and potential
    are O(N_atoms^2) and left out)."""
    if form == "fp16x6":
        return (KERNEL_BYTES["update_fp16x6"](N) + KERNEL_BYTES["split_dH_fp16x6"](N)
                + KERNEL_BYTES["tc_gemm_dM_fp16x6"](N) + KERNEL_BYTES["tc_gemm_X_fp16x6"](N))
    return 0


def roofline(prof: dict, form: str, N: int, peaks: dict, src: str, ms_step_dev: float) -> dict:
    """The dominant kernel's entry (top-level keys), every kernel's entry, and the step as
    a whole: its time against max(method flops / tensor peak, algorithmic bytes / HBM)."""
    name, t_ms = max(prof.items(), key=lambda kv: kv[1])
    out = kernel_roofline(name, t_ms, form, N, peaks, src)
    out["kernels"] = {k: kernel_roofline(k, t, form, N, peaks, src) for k, t in prof.items()}
    nb = step_bytes(form, N)
    if nb:
        t_tensor = STEP_FLOPS(N) / (peaks["bf16_tflops"] * 1e12)
        t_hbm = nb / (peaks["hbm_gbs"] * 1e9)
        floor = max(t_tensor, t_hbm)
        out["step"] = {"time_us": 1000.0 * ms_step_dev, "tensor_floor_us": 1e6 * t_tensor,
                       "hbm_floor_us": 1e6 * t_hbm, "bound": "hbm" if t_hbm >= t_tensor else "tensor",
                       "algorithmic_bytes": nb, "method_flops": STEP_FLOPS(N),
                       "frac": floor / (ms_step_dev * 1e-3)}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--forms", default="fp64,fp64s,fp32,bf16x3,fp16x3,fp16x6")
    ap.add_argument("--atoms", type=int, default=256)
    ap.add_argument("--cpu-steps", type=int, default=12)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-n2048", action="store_true")
    ap.add_argument("--c4-probes", type=int, default=64, help="pump-probe scan size (0: skip)")
    ap.add_argument("--c4-steps", type=int, default=200, help="timed post-kick steps per probe")
    ap.add_argument("--no-c5", action="store_true", help="skip the learned-form section")
    ap.add_argument("--x-tile", type=int, default=0,
                    help="X product tile width of the tensor-core forms (0: timed at the first step)")
    ap.add_argument("--measure-peaks", action="store_true",
                    help="print cuBLAS FP64/FP32/TF32 GEMM rates and exit")
    ap.add_argument("--c5-runs", type=int, default=4, help="learned form: training runs")
    ap.add_argument("--c5-steps", type=int, default=1200, help="learned form: steps per training run")
    ap.add_argument("--c5-epochs", type=int, default=20)
    ap.add_argument("--c5-windows", type=int, default=12)
    ap.add_argument("--accuracy-c2-steps", type=int, default=20000,
                    help="run-length accuracy on the N=1024 flake, steps per form (0: skip)")
    ap.add_argument("--accuracy-c2-forms", default="fp64,fp64s,bf16x3,fp16x3,fp16x6")
    ap.add_argument("--accuracy-c3-steps", type=int, default=1000,
                    help="run-length accuracy of the Ehrenfest cluster, FP64-sliced vs FP64 (0: skip)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    from paper_1912_03174_gb300 import inputs as I
    sysm, run = I.flake_c2(n_atoms=args.atoms)

    if args.impl == "reference":
        reference_arm(args, sysm, run, rank)
        return

    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if args.measure_peaks:
        with ClockSampler(local) as clk:
            peaks = measure_peaks(torch)
        print(json.dumps({"cublas_gemm_n8192": peaks, "clocks": clk.summary()}), flush=True)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo", init_method="env://")
    import __graft_entry__ as g
    g.build()
    from paper_1912_03174_gb300 import binding as B

    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    forms = args.forms.split(",")
    res = {}
    secs = {}
    peaks, src = _peaks()
    with ClockSampler(local) as clk:
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for f in forms:
            res[f] = run_form(B, torch, sysm, run, f, args.steps, args.warmup, flush, stream,
                              x_tile=args.x_tile)
        secs["forms"] = time.perf_counter() - t0
        n2048 = None
        if not args.no_n2048:
            t0 = time.perf_counter()
            n2048 = n2048_runs(B, torch, flush, stream, min(args.steps, 200))
            secs["n2048"] = time.perf_counter() - t0
        c4 = None
        if args.c4_probes > 0:
            t0 = time.perf_counter()
            if world > 1:
                c4 = c4_sharded(B, torch, dist, rank, world, args.c4_probes, args.c4_steps)
            else:
                c4 = c4_runs(B, torch, args.c4_probes, args.c4_steps)
            c4_fractions(c4, peaks)
            secs["c4"] = time.perf_counter() - t0
        c5 = None
        if not args.no_c5:
            t0 = time.perf_counter()
            c5 = c5_runs(B, torch, n_train=args.c5_runs, train_steps=args.c5_steps,
                         windows=args.c5_windows, epochs=args.c5_epochs)
            c5["k_sweep"] = c5_k_sweep(B)
            secs["c5"] = time.perf_counter() - t0
        if dist:
            dist.barrier()
    clocks = clk.summary()
    accuracy = {}
    if args.accuracy_c2_steps > 0:
        t0 = time.perf_counter()
        accuracy["c2"] = accuracy_c2(B, sysm, run, args.accuracy_c2_forms.split(","),
                                     args.accuracy_c2_steps)
        secs["accuracy_c2"] = time.perf_counter() - t0
    if args.accuracy_c3_steps > 0:
        t0 = time.perf_counter()
        accuracy["c3"] = accuracy_c3(B, args.accuracy_c3_steps)
        secs["accuracy_c3"] = time.perf_counter() - t0

    head = forms[-1]
    r = res[head]
    ms_step = float(np.mean(r["ms"]))
    ms_step, value = replica_timing(ms_step, world, dist)
    ms64 = float(np.mean(res["fp64"]["ms"])) if "fp64" in res else None
    err = None
    if "fp64" in res and head != "fp64":
        err = float(np.max(np.abs(r["hist"] - res["fp64"]["hist"])))
    N = sysm.n_orb
    roof = roofline(r["prof"], head, N, peaks, src, ms_step_dev=float(np.mean(r["ms"])))
    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp64": "f64", "fp64s": "f64 (int7x6 slices)", "fp32": "f32",
                                       "bf16x3": "bf16x3", "fp16x3": "fp16x3", "fp16x6": "fp16x6"}[head],
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N, "precision": head, "parallelism": "replicas",
                   "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MB write)",
                   "fp64_steps_per_s": (1000.0 / ms64) if ms64 else None,
                   "speedup_vs_fp64": (ms64 / float(np.mean(r['ms']))) if ms64 else None,
                   "max_dipole_err_vs_fp64_au": err,
                   "forms": form_summary(res, forms, sysm.n_electrons),
                   "x_tile": {f: res[f]["x_tile"] for f in forms if res[f]["x_tile"] > 0},
                   "kernel_ms": {f: res[f]["prof"] for f in forms},
                   "n2048": n2048,
                   "pump_probe_c4": c4,
                   "learned_c5": c5,
                   "accuracy": accuracy or None,
                   "section_seconds": secs},
        "roofline": roof,
        "gpu_launches": int(r["launches"]),
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = len(os.sched_getaffinity(0))
        v, w, n = cpu_baseline(sysm, run, args.cpu_steps)
        line["cpu_baseline"] = {"value": v, "unit": "steps/s", "cores": cores, "kind": "oracle",
                                "sample": f"ground state and {w} oracle step untimed, then {n} oracle "
                                          f"steps of the same workload"}
    if rank == 0:
        if not args.no_e2e:
            line["e2e"] = e2e_run(B, sysm, run, head, min(args.steps, 100), args.warmup)
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
