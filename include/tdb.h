/*
 * tdb.h -- C ABI of the GB300 real-time TD-DFTB density-matrix propagator.
 *
 * The library propagates the one-body density matrix rho of a tight-binding
 * (DFTB-form) system under the generalised Liouville-von Neumann equation of
 * Bonafe et al., "A real-time time-dependent density functional tight-binding
 * implementation for semiclassical excited state electron-nuclear dynamics
 * and pump-probe spectroscopy simulations" (arXiv 1912.03174):
 *
 *   drho/dt = -i (S^-1 H rho - rho H S^-1) - (S^-1 D rho + rho D^T S^-1)   (eq:eomrho)
 *
 * with the leapfrog scheme rho_{n+1} = rho_{n-1} + 2 dt drho_n and an Euler
 * first step (eq:leapfrog, Sec. 2.3), SCC Hamiltonian rebuild from Mulliken
 * charges (eq:hscc, eq:hsccvext, eq:qmulik), the delta kick of eq:rhokick, the
 * laser pulse of eq:pumpf, Ehrenfest forces (eq:forces) and velocity-Verlet
 * nuclei (Sec. 2.3).  Units: Hartree atomic units throughout.
 *
 * Conventions for every call:
 *  - Host pointers are read during the call only; the caller keeps ownership.
 *    Device memory is owned by the context (or by the caller when a workspace
 *    is passed to tdb_create; the library then never frees it).
 *  - Matrices on the device are row-major, orbitals atom-major with
 *    orbs_per_atom (1 or 4: s, px, py, pz) consecutive orbitals per atom.
 *  - No call aborts or exits, and no call falls back to a CPU path.  Errors are
 *    returned as tdb_status; tdb_last_error() gives a message for the calling
 *    thread.  After TDB_ERR_NUMERIC or TDB_ERR_TIMEOUT a context is "sticky":
 *    only tdb_observables, tdb_get_state, tdb_get_rho and tdb_destroy work.
 *  - A context is thread-compatible, not thread-safe.  All GPU work of a
 *    context runs on the stream given in tdb_params (NULL = a stream the
 *    context creates).  tdb_step is asynchronous; calls that return host
 *    data synchronise that stream.
 */
#ifndef TDB_H
#define TDB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tdb_ctx tdb_ctx;

typedef enum {
    TDB_OK = 0,
    TDB_ERR_ARG = 1,          /* invalid argument (NULL, size, range) */
    TDB_ERR_STATE = 2,        /* call out of order (e.g. tdb_step before tdb_ground_state) */
    TDB_ERR_CUDA = 3,         /* a CUDA runtime / library call failed */
    TDB_ERR_NOT_SPD = 4,      /* overlap matrix S is not positive definite */
    TDB_ERR_SCC_NOCONV = 5,   /* ground-state charge self-consistency did not converge */
    TDB_ERR_UNSTABLE = 6,     /* dt * (spectral width of S^-1 H) >= 0.9: leapfrog unstable */
    TDB_ERR_NUMERIC = 7,      /* NaN/Inf or invariant violation found by tdb_check */
    TDB_ERR_TIMEOUT = 8,      /* a bounded device-side wait gave up */
    TDB_ERR_NOMEM = 9,        /* device allocation failed or workspace too small */
    TDB_ERR_UNSUPPORTED = 10  /* valid request this build does not implement */
} tdb_status;

/* Arithmetic of the per-step matrix products (eq:eomrho).  The density matrix
 * master copy, charges, potentials, energies and forces are FP64 in every mode. */
typedef enum {
    TDB_FP64 = 0,     /* FP64 products (SIMT DFMA) */
    TDB_FP32 = 1,     /* FP32 products (SIMT FFMA) on the deviation rho - rho_gs */
    TDB_BF16X3 = 2,   /* tcgen05 tensor cores, BF16 hi/lo pieces (~16 bits), 3 products,
                         FP32 accumulate, on the deviation rho - rho_gs */
    TDB_FP16X3 = 3,   /* tcgen05 tensor cores, power-of-two scaled FP16 hi/lo pieces
                         (~22 bits), 3 products, FP32 accumulate, on rho - rho_gs.
                         Requires |v - v_gs| < 16 Ha for every atom potential. */
    TDB_FP16X6 = 4,   /* tcgen05 tensor cores, each operand = 7-bit integer head + two FP16
                         tails (~29 bits) under per-step power-of-two scales; the head
                         products accumulate exactly (integer sums below 2^24), the five
                         tail products in a second FP32 accumulator; on rho - rho_gs */
    TDB_FP64_SLICED = 5 /* FP64-accurate products on the tcgen05 tensor cores: rows of A and
                         columns of B cut into six 7-bit integer slices under power-of-two
                         scales, every slice product summed exactly (see tdb_slice_gemm);
                         FP64 density and update; frozen or moving nuclei; N <= 4096 */
} tdb_precision;

/* The system (geometry and synthetic two-centre model).  Radial integrals:
 *   hopping  V_k(r) =  eta_k * t0 * exp(-r / lam_H)
 *   overlap  S_k(r) = -eta_k * s0 * exp(-r / lam_S),  k = ss-sigma, sp-sigma, pp-sigma, pp-pi
 * combined by the Slater-Koster s/p table (these stand in for the tabulated
 * H0/S of Sec. 2.1).  On-site: H0_AA = diag(eps_s, eps_p, eps_p, eps_p), S_AA = 1.
 * gamma_AB (eq:coul): U_A on-site, 1/R - zeta(R) off-site with the closed form
 * for exponential densities, tau = 16 U / 5.  E_rep = sum_{A<B} rep_A exp(-r / rep_b). */
typedef struct {
    int n_atoms;               /* >= 1 */
    int orbs_per_atom;         /* 1 (s) or 4 (s, px, py, pz) */
    int n_species;             /* >= 1 */
    const int* species;        /* [n_atoms], values in [0, n_species) */
    const double* R;           /* [n_atoms][3] positions, bohr */
    const double* V;           /* [n_atoms][3] velocities (bohr / a.u. time), or NULL (= 0) */
    const double* eps_s;       /* [n_species] on-site s energy, Ha */
    const double* eps_p;       /* [n_species] on-site p energy, Ha */
    const double* hubbard_U;   /* [n_species] Hubbard U, Ha (> 0 when scc) */
    const double* mass;        /* [n_species] amu */
    double t0, lam_H, s0, lam_S;
    double eta[4];
    double rep_A, rep_b;
    double n_electrons;        /* 0 < n_electrons <= 2 N */
} tdb_system;

typedef struct {
    double dt;                 /* time step, a.u. (negative: run backwards) */
    int scc;                   /* 1: SCC Hamiltonian rebuild every step (eq:hscc) */
    int move_nuclei;           /* 1: Ehrenfest nuclei (eq:forces, velocity Verlet); 0: frozen */
    int precision;             /* tdb_precision */
    int window;                /* steps between invariant checks in tdb_check (>= 1) */
    double scc_tol;            /* ground-state tolerance on max |dq_out - dq_in| */
    int scc_max_iter;
    double kT;                 /* ground-state electronic temperature (Ha); 0 = aufbau */
    double scc_mix;            /* Anderson mixing parameter of the ground state (0, 1], 0.3 */
    long history_cap;          /* dipole ring-buffer length (steps), >= 1 */
    void* cuda_stream;         /* cudaStream_t, or NULL */
} tdb_params;

/* Laser pulse E(t) = E0 sin(omega t + phase) f(t) dir (eq:pumpf).
 * envelope: 0 none (f = 1); 1 Gaussian exp(-4 ln2 (t - t_center)^2 / fwhm^2);
 *           2 sin^2(pi t / fwhm) on 0 <= t <= fwhm, zero elsewhere. */
typedef struct {
    double E0, omega, phase, t_center, fwhm;
    double dir[3];
    int envelope;
} tdb_field;

typedef struct {
    double t;                  /* time of rho_n */
    long step;                 /* n */
    double dipole[3];          /* mu = -sum_A dq_A R_A (Sec. 2.2, monopole charges) */
    double E_total;            /* E_band + E_coul + E_rep + E_kin + E_ext */
    double E_band;             /* Re Tr(rho H0) */
    double E_coul;             /* 1/2 sum_AB gamma_AB dq_A dq_B (eq:coul) */
    double E_rep;              /* pair repulsion */
    double E_kin;              /* nuclear kinetic energy at V_n */
    double E_ext;              /* sum_A dq_A R_A . E(t) */
    double work;               /* int_0^t P dt, P = Re Tr[S^-1 H rho (D - D^T)] (trapezoid) */
    double trace_re, trace_im; /* Tr(rho S) */
    double herm_err;           /* max |rho - rho^dagger| */
} tdb_obs;

/* Default parameters (dt 0.2, scc 1, frozen nuclei, FP64, window 100,
 * scc_tol 1e-12, 400 iterations, kT 0, mix 0.3, history 65536, stream NULL). */
void tdb_default_params(tdb_params* out);

/* Device bytes a context needs for this system and these parameters. */
size_t tdb_workspace_bytes(const tdb_system* sys, const tdb_params* prm);

/* Create a context: copy the system to the device and build S, H0, gamma
 * (Sec. 2.1).  workspace: caller-owned device memory of at least
 * tdb_workspace_bytes() bytes, 256-byte aligned, or NULL (the library
 * allocates).  Returns TDB_ERR_NOT_SPD if S is not positive definite. */
tdb_status tdb_create(const tdb_system* sys, const tdb_params* prm, void* workspace,
                      size_t workspace_bytes, tdb_ctx** out);

/* Ground state (Sec. 2.1: cycles of diagonalisation and Hamiltonian build to
 * self-consistency): rho_0 = C f C^T of H C = S C eps, charges mixed until
 * max |dq_out - dq_in| <= scc_tol.  The charge residual is preconditioned with a
 * constant-density-of-states response model (1 - chi gamma)^-1 before Anderson
 * mixing (scc_mix), which keeps large metallic clusters from charge sloshing.
 * Resets t = 0, n = 0, next step Euler. */
tdb_status tdb_ground_state(tdb_ctx* ctx, int* iters_out, double* residual_out);

/* Delta kick of eq:rhokick applied to the current rho (and to the previous
 * leapfrog level, so that the next step is Euler): V = -E0 diag(dir . R_A(mu)). */
tdb_status tdb_kick(tdb_ctx* ctx, double strength, const double dir[3]);

/* Set (or clear with NULL) the laser field of eq:pumpf; takes effect from the next step. */
tdb_status tdb_set_field(tdb_ctx* ctx, const tdb_field* field);

/* Advance n >= 0 leapfrog steps (asynchronous on the context stream). */
tdb_status tdb_step(tdb_ctx* ctx, long n);

/* A new context in the state of src (after its ground state): same system,
 * parameters and precision form, its own device workspace (workspace as in
 * tdb_create, or NULL) and stream (cuda_stream, or NULL for a new one); the
 * device state is copied device to device, so a branch costs no ground state and
 * no host round trip.  Stepping the clone reproduces stepping src bit for bit.
 * This is how a probe run branches from a pump run at delay tau (Sec. 3.2):
 * step the pump to tau, clone, kick the clone. */
tdb_status tdb_clone(tdb_ctx* src, void* cuda_stream, void* workspace, size_t workspace_bytes,
                     tdb_ctx** out);

/* Per-atom SCC shift sum_B gamma_AB dq_B (eq:hscc) of the current rho_n into out, and
 * when dq is non-NULL the charge fluctuations dq_A = q_A - q0_A themselves (Mulliken
 * charges of rho_n, eq:qmulik): n_atoms host doubles each.  Frozen nuclei
 * (TDB_ERR_UNSUPPORTED otherwise).  The learned form takes their history at window
 * ends as network input. */
tdb_status tdb_scc_shift(tdb_ctx* ctx, double* out, double* dq);

/* k leapfrog steps (eq:leapfrog, eq:eomrho) with the Hamiltonian frozen at
 * H_bar = H0 + 1/2 S (v_bar_A + v_bar_B) (eq:hscc with the per-atom potential v_bar,
 * n_atoms values: the SCC shift plus any external potential, averaged over the
 * window), taken in closed form: in the generalised eigenbasis H_bar C = S C eps the
 * leapfrog acts element by element through its own two modes.  One FP64 generalised
 * eigensolve and 17 N^3 products replace k steps of products; charges come only at
 * the window's end, and the dipole history is not written inside a window.  FP64 or
 * FP64_SLICED form, frozen nuclei and no laser field (TDB_ERR_UNSUPPORTED), not right
 * after a ground state, kick or state load (take one tdb_step first: TDB_ERR_STATE).
 * Requires (eps_max - eps_min) |dt| < 1, checked after the eigensolve
 * (TDB_ERR_UNSUPPORTED).  v_bar: n_atoms host doubles, read during the call; k >= 1
 * (TDB_ERR_ARG).  A failed eigensolve returns TDB_ERR_CUDA.  The eigensolver workspace
 * (cuSOLVER's plus N x N doubles) is allocated by the first call (TDB_ERR_NOMEM) and
 * freed by tdb_destroy, also when the context's workspace is the caller's.  Synchronises
 * the context stream twice (before staging v_bar, after the eigensolve); the products
 * after it are asynchronous. */
tdb_status tdb_step_window(tdb_ctx* ctx, const double* v_bar, int k);

/* The per-atom shift network of the learned form (this library's own GPU kernels;
 * the paper has no network, it is the learned part built around its propagator):
 * y = w3 . tanh(W2^T tanh(W1^T x + b1) + b2) + b3 for each sample x (n_features
 * values), weights used in bfloat16 with FP32 accumulation, FP32 master parameters
 * packed as W1 (n_features x hidden, row-major), b1, W2 (hidden x hidden), b2, w3,
 * b3.  Trained with Adam on the mean squared error.  n_features <= 32, hidden <= 64.
 * X: n x n_features row-major host floats; Y: n host floats; params and grad:
 * tdb_shiftnet_param_count floats.  Host buffers are read or written during the call
 * only.  The network owns its device memory and its CUDA stream, and every call
 * synchronises that stream.  NULL arguments, n < 1, epochs < 1, batch < 1 or lr <= 0
 * return TDB_ERR_ARG; CUDA failures TDB_ERR_CUDA.  create: uniform weights in
 * +-sqrt(3 / fan_in) from a splitmix64 stream of seed, zero biases.  set_params also
 * resets the Adam moments and step count.  destroy(NULL) does nothing. */
typedef struct tdb_shiftnet tdb_shiftnet;
tdb_status tdb_shiftnet_create(int n_features, int hidden, unsigned long long seed,
                               tdb_shiftnet** out);
long tdb_shiftnet_param_count(const tdb_shiftnet* net);
tdb_status tdb_shiftnet_get_params(tdb_shiftnet* net, float* params);
tdb_status tdb_shiftnet_set_params(tdb_shiftnet* net, const float* params);
tdb_status tdb_shiftnet_predict(tdb_shiftnet* net, const float* X, long n, float* Y);
/* grad = d(mean squared error)/d(params) over the n samples (FP32 sums in an
 * unspecified order); *loss = the mean squared error. */
tdb_status tdb_shiftnet_gradient(tdb_shiftnet* net, const float* X, const float* Y, long n,
                                 float* grad, double* loss);
/* epochs passes over the samples in mini-batches of batch (in order), one Adam step
 * (learning rate lr) per batch; *loss_out = mean squared error over the last epoch. */
tdb_status tdb_shiftnet_train(tdb_shiftnet* net, const float* X, const float* Y, long n,
                              int epochs, long batch, float lr, double* loss_out);
void tdb_shiftnet_destroy(tdb_shiftnet* net);

/* Advance each of count independent contexts (trajectories) by n >= 0 steps,
 * enqueued step by step across them so that their streams run side by side on the
 * GPU: the probe runs of a pump-probe scan (Sec. 3.2) branch from pump snapshots
 * (tdb_set_state + tdb_kick) and are independent of one another.  Each context
 * should have a stream of its own (params.cuda_stream NULL, or distinct streams);
 * contexts that share a stream are stepped correctly but one after another.
 * Asynchronous like tdb_step.  On an error in context i at step k the contexts
 * before i have made k + 1 steps, the others k; the message names i and k. */
tdb_status tdb_step_batch(tdb_ctx* const* ctxs, int count, long n);

/* A grouped batch: count independent contexts of one tensor-core form (TDB_BF16X3,
 * TDB_FP16X3 or TDB_FP16X6), frozen nuclei, one time step, each after its ground state
 * (the probe runs of a pump-probe scan, Sec. 3.2, branched with tdb_clone).  Every phase of
 * a step (delta H pieces, delta M = S^-1 delta H, X = M rho, the update, the charges of the
 * new level, its potential and dipole) is one launch over all contexts, whatever their
 * sizes: per-context tensor maps and arguments live in device arrays, a work list maps each
 * block to (context, tile), and the six launches of a step are one CUDA graph.  Creating
 * the batch runs an autotuner over the X tile width (128, 176, 256) and the schedule (the
 * contexts in the given order, or the largest first) on the contexts' current operands;
 * the choice changes the time, not the result.  Each context keeps its own state, stream
 * and dipole history; the batch has its own stream, ordered after the contexts' streams
 * at each tdb_batch_step and before them afterwards.  The contexts must not be stepped on
 * their own while the batch is used (TDB_ERR_STATE), and the batch is destroyed before
 * them.  TDB_ERR_UNSUPPORTED for other forms or moving nuclei, TDB_ERR_ARG for mixed forms
 * or time steps, repeated contexts or count < 1. */
typedef struct tdb_batch tdb_batch;
tdb_status tdb_batch_create(tdb_ctx* const* ctxs, int count, tdb_batch** out);
/* Advance every context of the batch by n >= 0 steps (asynchronous).  A pending Euler step
 * (after a kick, ground state or state load) is taken context by context first. */
tdb_status tdb_batch_step(tdb_batch* batch, long n);
/* The autotuner's choice: X tile width, schedule (0 given order, 1 largest first) and the
 * X launch time it measured (ms); any pointer may be NULL. */
tdb_status tdb_batch_tuning(const tdb_batch* batch, int* x_bn, int* schedule, double* x_ms);
void tdb_batch_destroy(tdb_batch* batch);

/* Observables of the current rho_n (synchronises).  charges: [n_atoms] Mulliken
 * populations q_A or NULL; forces: [n_atoms][3] Ehrenfest forces (eq:forces,
 * velocity terms dropped) or NULL. */
tdb_status tdb_observables(tdb_ctx* ctx, tdb_obs* obs, double* charges, double* forces);

/* The dipoles mu_k of the last min(steps, cap) steps, oldest first:
 * out[3 * cap] host doubles; *n_out = number written. */
tdb_status tdb_dipole_history(tdb_ctx* ctx, double* out, long cap, long* n_out);

/* Copy rho_n (and rho_{n-1} when prev_re/prev_im are non-NULL) to host,
 * row-major N x N doubles. */
tdb_status tdb_get_rho(tdb_ctx* ctx, double* re, double* im, double* prev_re, double* prev_im);

/* Checkpoint: bytes of a state blob, and copy it out / back in (rho_{n-1},
 * rho_n, R, V, t, n, Euler flag, work integral).  set_state makes a context
 * continue bitwise as the one it was taken from. */
size_t tdb_state_bytes(const tdb_ctx* ctx);
tdb_status tdb_get_state(tdb_ctx* ctx, void* host_buf, size_t bytes);
tdb_status tdb_set_state(tdb_ctx* ctx, const void* host_buf, size_t bytes);

/* Invariant monitor (synchronises): NaN/Inf, |Tr(rho S) - N_e| / N_e <= tol_trace.
 * Violation returns TDB_ERR_NUMERIC and makes the context sticky. */
tdb_status tdb_check(tdb_ctx* ctx, double tol_trace);

/* Width of the X product's tiles in the tensor-core forms (FP16X6, FP16X3, BF16X3): 128, 176
 * or 256 columns, or 0 for the default (the candidates timed at the first step, the fastest
 * kept).  The width changes the time of a step, not its result (every output element keeps
 * its order of accumulation).  TDB_ERR_ARG for another value or a width the product cannot
 * take at this N, TDB_ERR_UNSUPPORTED for the other forms.  Synchronises the context. */
tdb_status tdb_set_x_tile(tdb_ctx* ctx, int width);
/* The X tile width in effect (0 while a context left to tune it has not stepped; -1 for
 * NULL or a form without tensor-core products). */
int tdb_x_tile(const tdb_ctx* ctx);

/* Failure-detection probe (the paper has no counterpart: it tests this library's handling
 * of a device-side wait that gives up).  Enqueues on the context stream one kernel that
 * waits on an mbarrier nothing arrives on, polling at most `polls` times (>= 1, else
 * TDB_ERR_ARG) like the bounded waits of the tensor-core products, and then records a
 * time-out in the context's device error flag.  The next call that reads the flag
 * (tdb_observables, tdb_check) returns TDB_ERR_TIMEOUT and the context becomes sticky, as
 * after a real time-out.  (The same flag records a split piece that overflowed its scale in
 * the FP16X6/FP16X3/BF16X3 products; that read returns TDB_ERR_NUMERIC.)  The probe issues no copy and holds no tensor memory, so the
 * GPU and the CUDA context stay usable.  Asynchronous. */
tdb_status tdb_wait_probe(tdb_ctx* ctx, long long polls);

/* Device kernel launches issued by the last tdb_step call (for accounting). */
long tdb_last_launch_count(const tdb_ctx* ctx);

/* Advance one step like tdb_step(ctx, 1) but without the captured graph, with a
 * CUDA event recorded on the context stream before each kernel; synchronises.
 * ms[i] = device time of kernel i (milliseconds), names[i] = a static string
 * naming it (names may be NULL); *n_out = kernels timed (<= cap).  With moving
 * nuclei the entries are the phases of the Ehrenfest step (model and S^-1, charges
 * and potential, products X, forces, NAC and power, products Z, update and velocity
 * Verlet). */
tdb_status tdb_step_profiled(tdb_ctx* ctx, double* ms, const char** names, int cap, int* n_out);

/* C = A B through the tensor-core split-precision GEMM on its own, for
 * validation and measurement (no context needed; allocates and frees its own
 * device buffers).  A: M x K, B: K x N, C: M x N, row-major host doubles.
 * fmt 0: FP16 hi/lo pieces with power-of-two scaling (~22 bits), products
 *        A_hi B_hi + A_hi B_lo + A_lo B_hi in one FP32 accumulator (tcgen05, TMEM);
 * fmt 1: the same with BF16 pieces (~16 bits);
 * fmt 2: 7-bit integer head + two FP16 tails (~29 bits); head products summed
 *        exactly, one accumulator per 1024 of K (K <= 3072, else TDB_ERR_ARG),
 *        five tail products in another.
 * ms (may be NULL): kernel time.
 * TDB_ERR_TIMEOUT if a bounded device wait expired. */
tdb_status tdb_split_gemm(int M, int N, int K, const double* A, const double* B, int fmt, double* C,
                          double* ms);

/* C = A B with FP64-accurate integer-slice products on the tensor cores: the
 * products S^-1 H and (S^-1 H) rho of eq:eomrho (Sec. 2.1) in the TDB_FP64_SLICED
 * form, here on their own (no context needed; allocates and frees its own device
 * buffers).  A: M x K, B: K x N, C: M x N, row-major host doubles, K <= 4096.
 * Each row of A (column of B) is scaled by a power of two into (-1, 1) and cut
 * into six signed 7-bit integer slices (FP16 values); the 21 slice pairs with
 * s + t < 6 are multiplied on the FP16 tensor cores, pairs of equal weight summed
 * exactly over 512-deep K chunks (integers below 2^24 in FP32), chunks and weights
 * combined exactly in 64-bit integers.  Error below about 7 2^-42 K max_k|A_ik|
 * max_k|B_kj|.  ms (may be NULL): kernel time.  TDB_ERR_ARG for bad sizes;
 * TDB_ERR_TIMEOUT if a bounded device wait expired. */
tdb_status tdb_slice_gemm(int M, int N, int K, const double* A, const double* B, double* C,
                          double* ms);

/* The same product as tdb_split_gemm, for callers that cannot allocate device
 * memory (this entry point has no counterpart in the paper; it serves library
 * users).  A process whose device memory is fully handed to its own pool, code
 * running while another component owns the allocator, or code that must not
 * trigger the implicit synchronisation of cudaMalloc/cudaFree cannot call
 * tdb_split_gemm, which allocates its own buffers.  This call allocates nothing:
 * A (M x K), B (K x N) and C (M x N) are caller-owned DEVICE arrays of row-major
 * doubles, the work is enqueued on `stream` (a cudaStream_t, NULL = the legacy
 * default stream) and the call returns without synchronising.  Intermediates
 * live in one fixed 8 MiB device array that every GPU loading the library
 * reserves until the process exits; it must hold the 16-bit pieces of A and of
 * B^T (2 or 3 pieces of 2 bytes for each element, K padded to a multiple of 64)
 * plus an FP32 copy of C, else TDB_ERR_NOMEM (for example 512 x 512 x 512
 * fits, 1024 x 1024 x 1024 does not).  All calls share that array and it keeps
 * the last call's contents: calls whose GPU work overlaps race, so serialise
 * them.  The first call on each device looks up the array's address and must
 * come before any stream capture.  fmt as in tdb_split_gemm.  M, N <= 32768 and
 * K <= 65536 (TDB_ERR_ARG).  Because the call returns before its GPU work runs, a
 * failure on the device (a bounded wait of the product that ran out, or an operand
 * piece that overflows, for example from an Inf or NaN in A or B) cannot be returned
 * as a status: C is then filled with NaN.  Check C after synchronising the stream. */
tdb_status tdb_split_gemm_noalloc(int M, int N, int K, const double* A, const double* B, int fmt,
                                  double* C, void* stream);

/* Damped one-sided Fourier transforms of sampled signals, the transforms behind the
 * absorption spectrum (eq:alpha: alpha(w) = (mu(w) - mu_0) / E0 after a kick, eq:sigma)
 * and the transient absorption of pump-probe runs (eq:alphaeff, eq:sigmaeff, Sec. 3.2,
 * where x is the probe dipole minus the pump-only dipole and t_damp the electronic
 * damping time):
 *   F_s(w_k) = dt sum_{n < K} x_s[n] exp(-n dt / t_damp) exp(+i w_k n dt)
 * (the rectangle rule on the step grid; the sign e^{+iwt} makes Im alpha > 0 at an
 * absorption peak).  x: nsig x K row-major host doubles; omega: nw host doubles (angular
 * frequencies, Ha); re, im: nsig x nw host doubles (written).  t_damp > 0, or 0 / +inf for
 * no damping; dt > 0.  FP64 on the GPU (the library allocates and frees its device
 * buffers; synchronises).  TDB_ERR_ARG for bad sizes, pointers or values, TDB_ERR_NOMEM if
 * the device buffers do not fit, TDB_ERR_CUDA for other CUDA failures. */
tdb_status tdb_damped_transform(int nsig, long K, const double* x, double dt, double t_damp,
                                int nw, const double* omega, double* re, double* im);

void tdb_destroy(tdb_ctx* ctx);
const char* tdb_status_string(tdb_status s);
const char* tdb_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TDB_H */
