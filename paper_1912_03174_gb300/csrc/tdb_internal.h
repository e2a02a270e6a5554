// Internal declarations of the tdb library (context layout and kernel launchers).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cusolverDn.h>

#include <string>
#include <vector>

#include "tdb.h"
#include "tdb_oz.h"
#include "tdb_tc.h"

namespace tdb {

constexpr int kTile = 32;          // tile edge of the O(N^2) kernels (update, Mulliken partials)

// Laser field parameters as the kernels read them (eq:pumpf).
struct FieldDev {
    double E0, omega, phase, t_center, fwhm;
    double dir[3];
    int envelope;
    int on;
};

// Device-resident scalars of a trajectory.  Graph-captured kernels read the
// step counter from here, so a replayed graph sees the current step.
struct DevScalars {
    long long step;      // n of the current rho_n
    long long n_base;    // t = t_base + (n - n_base) * dt
    double t_base;
    double dt;
    FieldDev field;
    double E[3];         // field at t_n (written by the potential kernel)
    double mu[3];        // dipole of rho_n
    double e_coul;       // 1/2 dq . gamma dq of rho_n
    double e_ext;        // dq . (R E(t_n))
    long long hist_cap;  // slots of the dipole ring (the requested history length + 1)
    // reduced-precision forms: Tr(rho S) of each master level and the renormalisation
    // factor f - 1 = N_e / Tr(rho S) - 1 that the update applies to it as a base level
    double trace_lvl[2];
    float eps_lvl[2];
    // ground-state constants of the per-level evaluation: N_e - sum_A q_A(rho_ref) and
    // the dipole of rho_ref
    double c0_trace;
    double mu_ref[3];
    double n_e;          // N_e
};

// Per-level evaluation of the reduced-precision forms: the Mulliken charges of a master
// level and what follows from them (SCC potential, dipole, trace), evaluated in FP32-pair
// arithmetic by two kernels: the charges (k_level_dq, from the row partials) and the
// potentials with the level's scalars (k_level_final).
struct LevelArgs {
    int nat, nper, nct, scc;
    const float2* partial;     // [N][nct] Mulliken row partials of the deviation (hi, lo)
    const float2* gam2;        // [nat][nat] gamma as (hi, lo)
    const float2* R2;          // [nat][3] positions as (hi, lo)
    const float* c_res;        // [nat] (gamma dq(rho_ref))_A - v_ref_A: SCC residual of rho_ref
    float2* dq;                // [nat] deviation charges of the level (written by k_level_dq)
    float2* bsum;              // [level_blocks][4] per charge block: sum dq R_x, R_y, R_z, sum dq
    float* dv_f;               // [N] v - v_ref per orbital (written by the final stage)
    tc::DynScales* dyn;        // FP16X6 scales (may be null)
    DevScalars* sc;
    double* hist;
    int* count;                // [2] final-stage arrivals, max |dv| (float bits); zero between evaluations
    float inv_ne;              // 1 / N_e
    int has_scales;            // write s_dh, s_dm from max |dv| (FP16X6)
};

// Moving-nuclei scalars: the work integral of P = Re Tr[S^-1 H rho (D - D^T)].
struct MdScalars {
    double work;      // int_0^{t_{n-1}} P dt (trapezoid), committed
    double P_prev;    // P_{n-1}
    double P_now;     // P of the last evaluated state
    double work_now;  // work including P_now
};

// Parameters of the synthetic two-centre model.
struct ModelParams {
    double t0, lam_H, s0, lam_S;
    double eta[4];
    double rep_A, rep_b;
};

// FP32-pair master of rho - rho_ref (reduced-precision forms), one leapfrog level.
struct MasterPtrs {
    float *re_hi, *re_lo, *im_hi, *im_lo;
};

// A propagation context.  All device pointers point into one workspace.
struct Ctx {
    int nat = 0, nper = 0, N = 0, nspec = 0, nct = 0;
    tdb_params prm{};
    ModelParams mp{};
    double n_electrons = 0;
    std::vector<int> species;
    std::vector<double> R, V, eps_s, eps_p, U, mass;

    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    size_t ws_need = 0;          // bytes of ws the layout uses
    bool own_ws = false;

    // device arrays (FP64)
    double *d_R = nullptr, *d_V = nullptr;           // [nat][3]
    double *d_onsite = nullptr;                     // [N] H0 diagonal
    double *d_U = nullptr, *d_mass = nullptr;        // per atom
    double *d_q0 = nullptr;                          // per atom reference population
    double *S = nullptr, *Sinv = nullptr, *H0 = nullptr, *gamma = nullptr;
    double *rho_re[2] = {nullptr, nullptr}, *rho_im[2] = {nullptr, nullptr};
    double *Xre = nullptr, *Xim = nullptr, *M = nullptr, *Hs = nullptr;
    double *partial = nullptr;                       // [nct][N] Mulliken row partial sums
    double *q = nullptr, *dq = nullptr, *v_orb = nullptr, *v_atom = nullptr, *gdq = nullptr;
    double *v_ref = nullptr;                         // [N] ground-state potential per orbital
    double *hist = nullptr;                          // [cap][3]
    double *obs_blocks = nullptr, *obs_out = nullptr;
    DevScalars* sc = nullptr;

    // reduced-precision operands (TDB_FP32 / TDB_BF16X3)
    double *rho_ref = nullptr;                       // ground-state rho (real)
    float *dv_f = nullptr;                           // [N] v - v_ref per orbital
    float *S_f = nullptr, *Sinv_f = nullptr, *Mgs_f = nullptr, *rref_f = nullptr;
    float *dM_f = nullptr, *M_f = nullptr;           // delta M, M = M_gs + delta M
    float *Xre_f = nullptr, *Xim_f = nullptr;
    // per-level evaluation of the reduced forms (LevelArgs)
    float2 *gam2 = nullptr, *R2 = nullptr, *lv_dq = nullptr, *lv_bsum = nullptr;
    float* c_res = nullptr;
    int* lv_count = nullptr;

    // reduced-precision master (two leapfrog levels) and the FP64 view's state
    MasterPtrs ms[2] = {};
    double* qbase = nullptr;     // Mulliken populations of rho_ref (deviation partials add to it)
    bool view_valid = true;      // FP64 rho_re / rho_im hold the current state

    // tensor-core operands (TDB_BF16X3 / TDB_FP16X3 / TDB_FP16X6): 16-bit pieces
    // (2 or 3 per operand), row stride padded to Np = round_up(N, 64)
    int Np = 0, scheme = 0, npieces = 0;
    uint16_t* pc_sinv[3] = {};   // N x Np     S^-1
    uint16_t* pc_dh[3] = {};     // N x Np     delta H
    uint16_t* pc_am[3] = {};     // N x 2Np    [delta M | M]
    uint16_t* pc_bre[3] = {};    // N x 2Np    [rho_ref | Re(rho - rho_ref)]
    uint16_t* pc_bim[3] = {};    // N x Np     -Im rho
    float* xp[tc::kMaxParts] = {};   // partial products of X (tensor-core forms)
    // FP64_SLICED form: slices of S^-1, H or D, M or Y, Re rho, Im rho
    oz::Sliced oz[5];
    char* oz_raw[5] = {};
    double* oz_colmax = nullptr;
    // moving nuclei, FP32 form: FP32 copies of S^-1, H or D, rho_n; M or Y; X or Z
    float *md_sinv = nullptr, *md_b = nullptr, *md_rre = nullptr, *md_rim = nullptr;
    float *md_m = nullptr, *md_xre = nullptr, *md_xim = nullptr;
    tc::DynScales* dyn = nullptr;
    int* d_err = nullptr;        // bounded-wait time-out / piece overflow flag
    float s_sinv = 1, s_dh = 1, s_m = 1, s_rho = 1, s_ref = 1;   // power-of-two operand scales
    tc::Maps maps_dm{}, maps_x{};
    int x_bn = 0;                // X tile width chosen by tune_x (0: not tuned yet)

    // host-side trajectory state
    int cur = 0;                 // index of rho_n in rho_re/rho_im
    bool have_gs = false, euler_next = true, sticky = false;
    long long n = 0;             // host mirror of the step counter
    long last_launches = 0;
    double spectral_width = 0;   // of S^-1 H at the ground state
    double work = 0;
    tdb_field field{};
    bool field_on = false;

    // pinned host staging for the per-step host<->device traffic (field, observables)
    char* h_pinned = nullptr;
    size_t h_pinned_bytes = 0;

    // moving nuclei (Ehrenfest): per-step buffers
    double *d_Vn = nullptr;                          // V_n (d_V holds V_{n-1/2}, or V_0)
    double *d_F = nullptr;                           // [nat][3] forces F_n
    double *D = nullptr, *Zre = nullptr, *Zim = nullptr, *Wre = nullptr;   // N x N
    double *pw_part = nullptr;                       // work-rate block partials
    MdScalars* md = nullptr;
    double* inv_work = nullptr;                      // cuSOLVER workspace (potrf/potri)
    int inv_lwork = 0;
    int* inv_info = nullptr;

    // closed-form windows (learned form): generalised eigensolver workspace and a scratch
    double* win_work = nullptr;
    int win_lwork = 0;
    int* win_info = nullptr;
    double* win_tmp = nullptr;

    cusolverDnHandle_t solver = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int graph_launches = 0;      // kernels per captured step
};

// ---- kernels (launchers) ----
void launch_build_model(const Ctx& c, const double* R, double* S, double* H0, cudaStream_t st);
void launch_build_gamma(const Ctx& c, const double* R, double* gamma, cudaStream_t st);
void launch_symmetrize_upper_to_lower(int N, double* A, cudaStream_t st);
void launch_transpose(int N, const double* in, double* out, cudaStream_t st);
void launch_mulliken_partials(int N, const double* rho_re, const double* S, double* partial,
                              cudaStream_t st);
// reset0/reset1 (may be null): device doubles zeroed by the kernel
void launch_charges(const Ctx& c, const double* partial, double* q, double* dq, cudaStream_t st,
                    double* reset0 = nullptr, double* reset1 = nullptr,
                    tc::DynScales* dyn = nullptr, int cur = 0, const double* qbase = nullptr);
// max_dv (may be null): atomicMax of |v - v_ref| over atoms
// record = 0: only v_orb, v_atom, gdq (no dipole, history or field record in sc)
void launch_potential(const Ctx& c, const double* gamma, const double* dq, const double* R,
                      DevScalars* sc, double* v_orb, double* v_atom, double* gdq, double* hist,
                      const double* v_ref, float* dv_orb, cudaStream_t st,
                      double* max_dv = nullptr, int record = 1);
void launch_build_hamiltonian(int N, const double* H0, const double* S, const double* v_orb,
                              double* H, cudaStream_t st);
// FP64 leapfrog / Euler update (zre, zim: NAC term of moving nuclei, or null)
void launch_update(const Ctx& c, const double* Xre, const double* Xim, const double* base_re,
                   const double* base_im, double* out_re, double* out_im, double factor,
                   const double* S, double* partial, DevScalars* sc, cudaStream_t st,
                   const double* zre = nullptr, const double* zim = nullptr);
// Operands written by the update for the next step's products.
struct UpdateOperands {
    const double* rho_ref = nullptr;   // deviations are taken from this (real) matrix
    int scheme = 0;                                         // tc::kHiLo / tc::kHead3 pieces
    uint16_t* re[3] = {};                                   // pieces of s (Re rho - rho_ref)
    uint16_t* im[3] = {};                                   // pieces of -s Im rho
    int ld_re = 0, ld_im = 0;
    float scale = 1.f;
    int bf16 = 0;
    tc::DynScales* dyn = nullptr;      // kHead3: s = pscale(max_drho[cur]); tracks the new max
    int cur = 0;
    const float* xre[4] = {};          // X = S^-1 H rho: partial products of Re X ...
    const float* xim[2] = {};          // ... and of Im X, summed in this order
    int nre = 0, nim = 0;
    int base_slot = 0;                 // FP16X6: buffer whose max bounds the update's base
};
void launch_kick_phase(int N, int n_per, const double* R, double strength, const double* dir,
                       const double* Pre, const double* Pim, double* Cre, double* Cim,
                       cudaStream_t st);
void launch_hermitian_half(int N, const double* Tre, const double* Tim, double* out_re,
                           double* out_im, cudaStream_t st);
void launch_obs_reduce(int N, const double* rho_re, const double* rho_im, const double* H0,
                       const double* S, double* block_out, int n_blocks, cudaStream_t st);
void launch_obs_finish(int n_blocks, const double* block_out, double* out4, cudaStream_t st);
void launch_scale_rows_f(int N, const double* in, const double* f, double* out, cudaStream_t st);
// moving nuclei (kern_md.cu)
void launch_forces(const Ctx& c, const double* rre, const double* wre, double* F, cudaStream_t st);
void launch_wre(int N, const double* xre, double* wre, cudaStream_t st);
void launch_build_nac(const Ctx& c, const double* V, double* D, cudaStream_t st);
void launch_power(const Ctx& c, const double* xre, const double* D, double* part, int nb, int first,
                  int commit, cudaStream_t st);
void launch_vel_n(const Ctx& c, const double* F, int first, cudaStream_t st);
void launch_vv(const Ctx& c, const double* F, cudaStream_t st);
// reduced-precision master (kern_step.cu)
// Arguments of one update of the reduced forms (one problem of a grouped launch).
struct UpdateDfArgs {
    int N, nct, out_slot, pad;
    MasterPtrs base, out;
    float fh, fl;
    double factor;
    const float* Sf;
    const float* rgs;
    DevScalars* sc;
    UpdateOperands ops;
    LevelArgs lv;
};
UpdateDfArgs update_df_args(const Ctx& c, const MasterPtrs& base, const MasterPtrs& out,
                            double factor, DevScalars* sc, const UpdateOperands& ops,
                            const LevelArgs& lv);
// Updates of many contexts in one launch: block b runs tile pair work[b].y of args[work[b].x].
void launch_update_df_grouped(const UpdateDfArgs* args, const int2* work, int nwork,
                              cudaStream_t st);
// The update of the reduced forms also renormalises its base level (f = N_e / Tr(rho S))
// and writes the Mulliken row partials of the new level (LevelArgs::partial); the level
// itself is evaluated by launch_level_dq and launch_level_final after it.
void launch_update_df(const Ctx& c, const MasterPtrs& base, const MasterPtrs& out, double factor,
                      DevScalars* sc, const UpdateOperands& ops, const LevelArgs& lv,
                      cudaStream_t st);
// Evaluation of the current level outside a step (after a ground state, kick, field change or
// state load), the two kernels of a step's evaluation; trace_only: only Tr(rho S) and the
// renormalisation factor of level `slot` (partials of that level in lv.partial).
void launch_level(const Ctx& c, const LevelArgs& lv, int slot, int trace_only, cudaStream_t st);
// The level after an update (the new level in slot): charges, then potentials and scalars.
// Atoms per block of the level kernels (64 threads per atom); the potentials kernel has one
// block more (the totals block).
constexpr int kLvAtoms = 4;
__host__ __device__ inline int level_blocks(int nat) { return (nat + kLvAtoms - 1) / kLvAtoms; }
void launch_level_dq(const Ctx& c, const LevelArgs& lv, cudaStream_t st);
void launch_level_final(const Ctx& c, const LevelArgs& lv, int slot, cudaStream_t st);
struct LevelFinalArgs {
    LevelArgs lv;
    int slot, pad;
};
void launch_level_dq_grouped(const LevelFinalArgs* args, const int2* work, int nwork,
                             cudaStream_t st);
void launch_level_final_grouped(const LevelFinalArgs* args, const int2* work, int nwork,
                                cudaStream_t st);
void launch_view_to_master(const Ctx& c, const double* rre, const double* rim, const MasterPtrs& m,
                           cudaStream_t st);
void launch_master_to_view(const Ctx& c, const MasterPtrs& m, double* rre, double* rim,
                           cudaStream_t st);
void launch_master_partials(const Ctx& c, const MasterPtrs& m, float2* partial, cudaStream_t st);
// FP64 populations q_A = qbase_A + sum of the (hi, lo) row partials, dq_A = q_A - q0_A
void launch_charges_df(const Ctx& c, const float2* partial, double* q, double* dq, cudaStream_t st);
void launch_master_absmax(const Ctx& c, const MasterPtrs& m, double* out, cudaStream_t st);
void launch_master_pieces(const Ctx& c, const MasterPtrs& m, const UpdateOperands& ops,
                          const double* mx_exact, const float* dev_scale, cudaStream_t st);
// FP16X6: head pieces of rho - rho_ref (scale from c.dyn->max_drho[slot]) into the B operands
// GEMM: C[M x Ncol] = A[M x K] * B[K x Ncol], row-major, FP64 SIMT.
enum class BKind { Dense = 0, Hamiltonian = 1 };
void gemm_f64(int M, int Ncol, int K, const double* A, int lda, const double* B, int ldb,
              double* C, int ldc, cudaStream_t st);
// C = A * H with H_kj = H0_kj + 1/2 S_kj (v_k + v_j) formed while loading B (eq:hscc).
void gemm_f64_ham(int N, const double* A, const double* H0, const double* S, const double* v_orb,
                  double* C, cudaStream_t st);
// FP32 SIMT: C = A * B (+ Cadd if non-null).
void gemm_f32(int M, int Ncol, int K, const float* A, int lda, const float* B, int ldb, float* C,
              int ldc, cudaStream_t st);

}  // namespace tdb
