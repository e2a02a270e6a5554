// C ABI of the propagator: context lifetime, ground state, kick, field,
// stepping (CUDA graphs), observables and checkpoints.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "tdb_internal.h"

namespace tdb {
void gemm_f32_dham(int N, const float* A, const float* S, const float* dv, float* C, int ldc,
                   const float* Cadd, cudaStream_t st);
void gemm_f32_add(int M, int Ncol, int K, const float* A, int lda, const float* B, int ldb,
                  float* C, int ldc, const float* Cadd, cudaStream_t st);
void launch_f64_to_f32(size_t n, const double* in, float* out, cudaStream_t st);
void launch_f32_to_f64(size_t n, const float* in, double* out, cudaStream_t st);
void launch_ns_update(int N, double* X, const double* Q, cudaStream_t st);
namespace learn {
void launch_window(int N, const double* eps, double dt, int k, double* x0re, double* x0im,
                   double* x1re, double* x1im, cudaStream_t st);
void launch_add_step(DevScalars* sc, int k, cudaStream_t st);
}  // namespace learn
void gemm_f32(int M, int Ncol, int K, const float* A, int lda, const float* B, int ldb, float* C,
              int ldc, cudaStream_t st);
void launch_add_f32_strided(int N, const float* a, const float* b, int ldb, float* out, int ldo,
                            cudaStream_t st);
void launch_small_energies(const Ctx& c, double* out, cudaStream_t st);
void launch_absmax(size_t n, const double* x, double* out, cudaStream_t st,
                   const double* sub = nullptr);
}  // namespace tdb

using namespace tdb;

struct tdb_ctx : public Ctx {};

namespace {
thread_local std::string g_err;
}

namespace tdb {
// message returned by tdb_last_error() on this thread
void set_last_error(const char* msg) { g_err = msg; }
}  // namespace tdb

namespace {

void set_err(const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            set_err("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_));   \
            return TDB_ERR_CUDA;                                                          \
        }                                                                                 \
    } while (0)

#define CKL()                                                                             \
    do {                                                                                  \
        cudaError_t e_ = cudaGetLastError();                                              \
        if (e_ != cudaSuccess) {                                                          \
            set_err("%s:%d kernel launch: %s", __FILE__, __LINE__, cudaGetErrorString(e_)); \
            return TDB_ERR_CUDA;                                                          \
        }                                                                                 \
    } while (0)

#define CKS(call)                                                                         \
    do {                                                                                  \
        cusolverStatus_t s_ = (call);                                                     \
        if (s_ != CUSOLVER_STATUS_SUCCESS) {                                              \
            set_err("%s:%d %s: cusolver status %d", __FILE__, __LINE__, #call, (int)s_);  \
            return TDB_ERR_CUDA;                                                          \
        }                                                                                 \
    } while (0)

#define TRY(x)                         \
    do {                               \
        tdb_status s_ = (x);           \
        if (s_ != TDB_OK) return s_;   \
    } while (0)

constexpr int kObsBlocks = 304;  // 2 x 152 SMs

// Carves named sub-buffers out of one workspace, 256-byte aligned.
struct Carver {
    char* base;
    size_t off = 0;
    template <typename T>
    T* take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

bool tensor(const Ctx& c) {
    return c.prm.precision == TDB_BF16X3 || c.prm.precision == TDB_FP16X3 ||
           c.prm.precision == TDB_FP16X6;
}
// Frozen-nuclei reduced forms (FP32-pair master of rho - rho_ref).
bool mixed(const Ctx& c) {
    return (c.prm.precision == TDB_FP32 || tensor(c)) && !c.prm.move_nuclei;
}
// Moving nuclei with FP32 products (FP64 density, forces and update).
bool md32(const Ctx& c) { return c.prm.move_nuclei && c.prm.precision == TDB_FP32; }
// FP64-accurate integer-slice products (FP64 density and update), any nuclei.
bool sliced(const Ctx& c) { return c.prm.precision == TDB_FP64_SLICED; }
bool head3(const Ctx& c) { return c.prm.precision == TDB_FP16X6; }
// The tensor-core X products (dM rho_ref, M Re(rho - rho_ref), M Im rho) are cut into
// this many K slices with their own FP32 outputs, so that a slice of K <= 1024 keeps one
// exact head accumulator per tile.  (Cutting N = 1024 in two as well spreads the tiles
// more evenly over the SMs, but the update then reads twice the partial products and the
// step is slower.)
int x_split(const Ctx& c) { return c.N > 1024 ? 2 : 1; }
int piece_bf16(const Ctx& c) { return c.prm.precision == TDB_BF16X3 ? 1 : 0; }

// 2^floor(log2(target / m)): the power-of-two scale that maps magnitude m near target
float pow2_scale(double m, double target) {
    if (!(m > 0)) return 1.0f;
    return (float)std::ldexp(1.0, (int)std::floor(std::log2(target / m)));
}

size_t carve(Ctx& c, char* base) {
    Carver k{base};
    const size_t N = c.N, NN = N * N, nat = c.nat;
    c.d_R = k.take<double>(3 * nat);
    c.d_V = k.take<double>(3 * nat);
    c.d_onsite = k.take<double>(N);
    c.d_U = k.take<double>(nat);
    c.d_mass = k.take<double>(nat);
    c.d_q0 = k.take<double>(nat);
    c.S = k.take<double>(NN);
    c.Sinv = k.take<double>(NN);
    c.H0 = k.take<double>(NN);
    c.gamma = k.take<double>(nat * nat);
    for (int i = 0; i < 2; ++i) {
        c.rho_re[i] = k.take<double>(NN);
        c.rho_im[i] = k.take<double>(NN);
    }
    c.Xre = k.take<double>(NN);
    c.Xim = k.take<double>(NN);
    c.M = k.take<double>(NN);
    c.Hs = k.take<double>(NN);
    c.partial = k.take<double>((size_t)c.nct * N);
    c.q = k.take<double>(nat);
    c.dq = k.take<double>(nat);
    c.v_atom = k.take<double>(nat);
    c.gdq = k.take<double>(nat);
    c.v_orb = k.take<double>(N);
    c.v_ref = k.take<double>(N);
    c.hist = k.take<double>(3 * ((size_t)c.prm.history_cap + 1));
    c.obs_blocks = k.take<double>(4 * kObsBlocks);
    c.obs_out = k.take<double>(16 + 2 * N);   // reductions, small energies, eigenvalues, occupations
    c.sc = k.take<DevScalars>(1);
    if (mixed(c)) {
        for (int l = 0; l < 2; ++l) {
            c.ms[l].re_hi = k.take<float>(NN);
            c.ms[l].re_lo = k.take<float>(NN);
            c.ms[l].im_hi = k.take<float>(NN);
            c.ms[l].im_lo = k.take<float>(NN);
        }
        c.qbase = k.take<double>(nat);
        c.rho_ref = k.take<double>(NN);
        c.Mgs_f = k.take<float>(NN);
        c.rref_f = k.take<float>(NN);
        c.gam2 = k.take<float2>(nat * nat);
        c.R2 = k.take<float2>(3 * nat);
        c.lv_dq = k.take<float2>(nat);
        c.lv_bsum = k.take<float2>(4 * (size_t)level_blocks(nat));
        c.c_res = k.take<float>(nat);
        c.lv_count = k.take<int>(2);
    }
    if (mixed(c)) {
        c.dv_f = k.take<float>(N);
        c.S_f = k.take<float>(NN);
    }
    if (sliced(c)) {
        // slices of S^-1 (A), H or D (B), M or Y (A), Re rho and Im rho (B)
        for (int q = 0; q < 5; ++q) c.oz_raw[q] = k.take<char>(oz::sliced_bytes(N, N));
        c.oz_colmax = k.take<double>(N);
    }
    if (md32(c)) {
        c.md_sinv = k.take<float>(NN);
        c.md_b = k.take<float>(NN);
        c.md_rre = k.take<float>(NN);
        c.md_rim = k.take<float>(NN);
        c.md_m = k.take<float>(NN);
        c.md_xre = k.take<float>(NN);
        c.md_xim = k.take<float>(NN);
    }
    if (c.prm.precision == TDB_FP32 && !c.prm.move_nuclei) {
        c.Xre_f = k.take<float>(NN);
        c.Xim_f = k.take<float>(NN);
        c.Sinv_f = k.take<float>(NN);
        c.dM_f = k.take<float>(2 * NN);     // [delta M | M], row stride 2N
        c.M_f = c.dM_f ? c.dM_f + N : nullptr;
    }
    if (tensor(c)) {
        const size_t Np = (N + 63) / 64 * 64;
        c.Np = (int)Np;
        c.scheme = head3(c) ? tc::kHead3 : tc::kHiLo;
        c.npieces = head3(c) ? 3 : 2;
        for (int q = 0; q < c.npieces; ++q) {
            c.pc_sinv[q] = k.take<uint16_t>(N * Np);
            c.pc_dh[q] = k.take<uint16_t>(N * Np);
            c.pc_am[q] = k.take<uint16_t>(2 * N * Np);
            c.pc_bre[q] = k.take<uint16_t>(2 * N * Np);
            c.pc_bim[q] = k.take<uint16_t>(N * Np);
        }
        for (int q = 0; q < 3 * x_split(c); ++q) c.xp[q] = k.take<float>(NN);
        c.dyn = k.take<tc::DynScales>(1);
    }
    if (c.prm.move_nuclei) {
        c.d_Vn = k.take<double>(3 * nat);
        c.d_F = k.take<double>(3 * nat);
        c.D = k.take<double>(NN);
        c.Zre = k.take<double>(NN);
        c.Zim = k.take<double>(NN);
        c.Wre = k.take<double>(NN);
        c.pw_part = k.take<double>(kObsBlocks);
        c.md = k.take<MdScalars>(1);
    }
    c.d_err = k.take<int>(4);
    return k.off + 256;
}

tdb_status validate(const tdb_system* s, const tdb_params* p) {
    if (!s || !p) {
        set_err("NULL system or params");
        return TDB_ERR_ARG;
    }
    if (s->n_atoms < 1 || (s->orbs_per_atom != 1 && s->orbs_per_atom != 4) || s->n_species < 1 ||
        !s->species || !s->R || !s->eps_s || !s->eps_p || !s->hubbard_U || !s->mass) {
        set_err("invalid system (sizes or NULL arrays)");
        return TDB_ERR_ARG;
    }
    const long N = (long)s->n_atoms * s->orbs_per_atom;
    if (N > 32768) {
        set_err("N = %ld exceeds the supported 32768 orbitals", N);
        return TDB_ERR_ARG;
    }
    if (!(s->n_electrons > 0) || s->n_electrons > 2.0 * N) {
        set_err("n_electrons out of range");
        return TDB_ERR_ARG;
    }
    for (int a = 0; a < s->n_atoms; ++a)
        if (s->species[a] < 0 || s->species[a] >= s->n_species) {
            set_err("species[%d] out of range", a);
            return TDB_ERR_ARG;
        }
    if (!(std::isfinite(p->dt)) || p->dt == 0.0 || p->window < 1 || p->history_cap < 1 ||
        p->scc_max_iter < 1 || !(p->scc_mix > 0 && p->scc_mix <= 1) || p->kT < 0 ||
        p->precision < 0 || p->precision > 5) {
        set_err("invalid params");
        return TDB_ERR_ARG;
    }
    if (p->move_nuclei && p->precision != TDB_FP64 && p->precision != TDB_FP32 &&
        p->precision != TDB_FP64_SLICED) {
        set_err("moving nuclei run in the FP64, FP64_SLICED and FP32 forms only in this build");
        return TDB_ERR_UNSUPPORTED;
    }
    if (p->precision == TDB_FP64_SLICED && N > oz::kMaxK) {
        set_err("TDB_FP64_SLICED supports N <= 4096 in this build");
        return TDB_ERR_UNSUPPORTED;
    }
    if (p->precision == TDB_FP16X6 && N > 2048) {
        // the X products are cut into two K slices, and the integer head products of one
        // slice sum exactly only while K * 127^2 < 2^24 (K <= 1040)
        set_err("TDB_FP16X6 supports N <= 2048 in this build");
        return TDB_ERR_UNSUPPORTED;
    }
    return TDB_OK;
}

void fill_host(Ctx& c, const tdb_system* s, const tdb_params* p) {
    c.prm = *p;
    c.nat = s->n_atoms;
    c.nper = s->orbs_per_atom;
    c.N = c.nat * c.nper;
    c.nct = (c.N + kTile - 1) / kTile;
    c.nspec = s->n_species;
    c.n_electrons = s->n_electrons;
    c.species.assign(s->species, s->species + c.nat);
    c.R.assign(s->R, s->R + 3 * c.nat);
    if (s->V)
        c.V.assign(s->V, s->V + 3 * c.nat);
    else
        c.V.assign(3 * c.nat, 0.0);
    c.eps_s.assign(s->eps_s, s->eps_s + c.nspec);
    c.eps_p.assign(s->eps_p, s->eps_p + c.nspec);
    c.U.assign(s->hubbard_U, s->hubbard_U + c.nspec);
    c.mass.assign(s->mass, s->mass + c.nspec);
    c.mp.t0 = s->t0;
    c.mp.lam_H = s->lam_H;
    c.mp.s0 = s->s0;
    c.mp.lam_S = s->lam_S;
    for (int k = 0; k < 4; ++k) c.mp.eta[k] = s->eta[k];
    c.mp.rep_A = s->rep_A;
    c.mp.rep_b = s->rep_b;
}

// Fermi-Dirac (kT > 0) or aufbau occupations, spin-degenerate (max 2 per level).
void occupations(const std::vector<double>& eps, double ne, double kT, std::vector<double>& f) {
    const int N = (int)eps.size();
    f.assign(N, 0.0);
    if (kT <= 0.0) {
        const int k = (int)std::ceil(ne / 2.0);
        const double ef = eps[std::max(k - 1, 0)];
        int below = 0, shell = 0;
        for (int i = 0; i < N; ++i) {
            if (eps[i] < ef - 1e-8)
                ++below;
            else if (std::fabs(eps[i] - ef) <= 1e-8)
                ++shell;
        }
        const double share = (ne - 2.0 * below) / shell;
        for (int i = 0; i < N; ++i) {
            if (eps[i] < ef - 1e-8)
                f[i] = 2.0;
            else if (std::fabs(eps[i] - ef) <= 1e-8)
                f[i] = share;
        }
        return;
    }
    double lo = eps.front() - 50 * kT, hi = eps.back() + 50 * kT;
    auto total = [&](double mu) {
        double s = 0;
        for (int i = 0; i < N; ++i) {
            double x = (eps[i] - mu) / kT;
            x = std::min(700.0, std::max(-700.0, x));
            s += 2.0 / (1.0 + std::exp(x));
        }
        return s;
    };
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (total(mid) > ne)
            hi = mid;
        else
            lo = mid;
    }
    const double mu = 0.5 * (lo + hi);
    for (int i = 0; i < N; ++i) {
        double x = (eps[i] - mu) / kT;
        x = std::min(700.0, std::max(-700.0, x));
        f[i] = 2.0 / (1.0 + std::exp(x));
    }
}

// Charge-sloshing preconditioner of the SCC residual (the paper names no mixer; the
// fixed point does not depend on it).  A potential change dv moves the charges by
// about chi dv; chi is modelled as a constant density of states per atom at the Fermi
// level, c, on the charge-neutral subspace: chi = -c (1 - 11^T / n).  One Newton step
// of dq_out = dq_in + chi gamma dq_in is then x = (1 - chi gamma)^-1 resid.  c sums
// the Fermi-function derivative over the levels at an electronic temperature of at
// least kPrecondKT, so that a gap at the Fermi level does not switch it off.
constexpr double kPrecondKT = 0.02;

void scc_precondition(const std::vector<double>& eps, double ne, double kT,
                      const std::vector<double>& gamma, const std::vector<double>& resid,
                      std::vector<double>& out) {
    const int n = (int)resid.size();
    const double ke = std::max(kT, kPrecondKT);
    std::vector<double> f;
    occupations(eps, ne, ke, f);
    double c = 0.0;
    for (double fi : f) c += fi * (1.0 - 0.5 * fi) / ke;
    c /= n;
    // A = 1 + c (1 - 11^T/n) gamma, solved by Gaussian elimination with partial pivoting
    std::vector<double> colmean(n, 0.0), A((size_t)n * n);
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) colmean[b] += gamma[(size_t)a * n + b] / n;
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b)
            A[(size_t)a * n + b] = (a == b ? 1.0 : 0.0) + c * (gamma[(size_t)a * n + b] - colmean[b]);
    out = resid;
    for (int col = 0; col < n; ++col) {
        int p = col;
        for (int r = col + 1; r < n; ++r)
            if (std::fabs(A[(size_t)r * n + col]) > std::fabs(A[(size_t)p * n + col])) p = r;
        if (p != col) {
            for (int k = 0; k < n; ++k) std::swap(A[(size_t)p * n + k], A[(size_t)col * n + k]);
            std::swap(out[p], out[col]);
        }
        const double d = A[(size_t)col * n + col];
        for (int r = col + 1; r < n; ++r) {
            const double m = A[(size_t)r * n + col] / d;
            if (m == 0.0) continue;
            for (int k = col; k < n; ++k) A[(size_t)r * n + k] -= m * A[(size_t)col * n + k];
            out[r] -= m * out[col];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double v = out[r];
        for (int k = r + 1; k < n; ++k) v -= A[(size_t)r * n + k] * out[k];
        out[r] = v / A[(size_t)r * n + r];
    }
}

// Anderson mixing of the charge fluctuations (history of input/residual pairs).
struct Anderson {
    int hist;
    double beta;
    std::vector<std::vector<double>> xs, fs;
    void next(std::vector<double>& x, const std::vector<double>& f) {
        xs.push_back(x);
        fs.push_back(f);
        if ((int)xs.size() > hist) {
            xs.erase(xs.begin());
            fs.erase(fs.begin());
        }
        const int m = (int)xs.size() - 1, n = (int)x.size();
        if (m < 1) {
            for (int i = 0; i < n; ++i) x[i] += beta * f[i];
            return;
        }
        // least squares: min |f - dF g|, dF[:, j] = f_{j+1} - f_j (normal equations,
        // Tikhonov-guarded)
        std::vector<double> A(m * m, 0.0), b(m, 0.0);
        std::vector<std::vector<double>> dF(m, std::vector<double>(n)), dX(m, std::vector<double>(n));
        for (int j = 0; j < m; ++j)
            for (int i = 0; i < n; ++i) {
                dF[j][i] = fs[j + 1][i] - fs[j][i];
                dX[j][i] = xs[j + 1][i] - xs[j][i];
            }
        for (int a = 0; a < m; ++a) {
            for (int c2 = 0; c2 < m; ++c2) {
                double s = 0;
                for (int i = 0; i < n; ++i) s += dF[a][i] * dF[c2][i];
                A[a * m + c2] = s;
            }
            double s = 0;
            for (int i = 0; i < n; ++i) s += dF[a][i] * f[i];
            b[a] = s;
        }
        double tr = 0;
        for (int a = 0; a < m; ++a) tr += A[a * m + a];
        for (int a = 0; a < m; ++a) A[a * m + a] += 1e-12 * tr + 1e-300;
        // Gaussian elimination with partial pivoting
        std::vector<double> g(b);
        std::vector<int> piv(m);
        for (int col = 0; col < m; ++col) {
            int p = col;
            for (int r = col + 1; r < m; ++r)
                if (std::fabs(A[r * m + col]) > std::fabs(A[p * m + col])) p = r;
            if (p != col) {
                for (int c2 = 0; c2 < m; ++c2) std::swap(A[p * m + c2], A[col * m + c2]);
                std::swap(g[p], g[col]);
            }
            const double d = A[col * m + col];
            for (int r = col + 1; r < m; ++r) {
                const double fct = A[r * m + col] / d;
                for (int c2 = col; c2 < m; ++c2) A[r * m + c2] -= fct * A[col * m + c2];
                g[r] -= fct * g[col];
            }
        }
        for (int col = m - 1; col >= 0; --col) {
            double s = g[col];
            for (int c2 = col + 1; c2 < m; ++c2) s -= A[col * m + c2] * g[c2];
            g[col] = s / A[col * m + col];
        }
        for (int i = 0; i < n; ++i) {
            double corr = 0;
            for (int j = 0; j < m; ++j) corr += (dX[j][i] + beta * dF[j][i]) * g[j];
            x[i] += beta * f[i] - corr;
        }
    }
};

tdb_status upload_field(Ctx& c) {
    // staged through pinned memory; the previous upload has completed when the
    // stream is synchronised by the caller (tdb_set_field synchronises)
    FieldDev& f = *reinterpret_cast<FieldDev*>(c.h_pinned);
    f = FieldDev{};
    if (c.field_on) {
        f.E0 = c.field.E0;
        f.omega = c.field.omega;
        f.phase = c.field.phase;
        f.t_center = c.field.t_center;
        f.fwhm = c.field.fwhm;
        for (int k = 0; k < 3; ++k) f.dir[k] = c.field.dir[k];
        f.envelope = c.field.envelope;
        f.on = 1;
    }
    CK(cudaMemcpyAsync(&c.sc->field, &f, sizeof f, cudaMemcpyHostToDevice, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    return TDB_OK;
}

tdb_status upload_clock(Ctx& c, long long step, long long n_base, double t_base) {
    DevScalars h{};
    CK(cudaMemcpyAsync(&h, c.sc, sizeof h, cudaMemcpyDeviceToHost, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    h.step = step;
    h.n_base = n_base;
    h.t_base = t_base;
    h.dt = c.prm.dt;
    h.hist_cap = c.prm.history_cap + 1;
    CK(cudaMemcpyAsync(c.sc, &h, sizeof h, cudaMemcpyHostToDevice, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    c.n = step;
    return TDB_OK;
}

// Operand pieces written from the master by the reduced forms (tensor-core schemes).
UpdateOperands master_operands(Ctx& c) {
    UpdateOperands ops;
    ops.rho_ref = c.rho_ref;
    ops.scheme = c.scheme;
    ops.bf16 = piece_bf16(c);
    const int np = c.npieces;
    for (int q = 0; q < np; ++q) {
        ops.re[q] = c.pc_bre[q] + c.Np;
        ops.im[q] = c.pc_bim[q];
    }
    ops.ld_re = 2 * c.Np;
    ops.ld_im = c.Np;
    ops.scale = c.s_rho;
    if (head3(c)) ops.dyn = c.dyn;
    return ops;
}

// Arguments of the per-level evaluation of the reduced forms.
LevelArgs level_args(Ctx& c) {
    LevelArgs a{};
    a.nat = c.nat;
    a.nper = c.nper;
    a.nct = c.nct;
    a.scc = c.prm.scc;
    a.partial = reinterpret_cast<const float2*>(c.partial);
    a.gam2 = c.gam2;
    a.R2 = c.R2;
    a.c_res = c.c_res;
    a.dq = c.lv_dq;
    a.bsum = c.lv_bsum;
    a.dv_f = c.dv_f;
    a.dyn = head3(c) ? c.dyn : nullptr;
    a.has_scales = head3(c) ? 1 : 0;
    a.sc = c.sc;
    a.hist = c.hist;
    a.count = c.lv_count;
    a.inv_ne = (float)(1.0 / c.n_electrons);
    return a;
}

// Reduced forms: partials and operands of rho_n from the master, then the evaluation of
// both levels (Tr(rho S) of rho_{n-1}; charges, potential, dipole and trace of rho_n), with
// the kernels a step uses after its update, so that a loaded state continues bit for bit.
// With `restored` (FP16X6 resuming from a checkpoint of the same form) the scales saved
// with the state are kept.
tdb_status derived_from_master(Ctx& c, bool restored = false) {
    float2* part = reinterpret_cast<float2*>(c.partial);
    const LevelArgs lv = level_args(c);
    launch_master_partials(c, c.ms[c.cur ^ 1], part, c.stream);
    launch_level(c, lv, c.cur ^ 1, 1, c.stream);
    launch_master_partials(c, c.ms[c.cur], part, c.stream);
    if (tensor(c)) {
        UpdateOperands ops = master_operands(c);
        if (head3(c) && restored) {
            launch_master_pieces(c, c.ms[c.cur], ops, nullptr, &c.dyn->s_rho, c.stream);
        } else if (head3(c)) {
            // exact maxima of both leapfrog levels, then the pieces of the current one
            for (int l = 0; l < 2; ++l) {
                CK(cudaMemsetAsync(&c.dyn->max_drho[l], 0, sizeof(double), c.stream));
                launch_master_absmax(c, c.ms[l], &c.dyn->max_drho[l], c.stream);
            }
            launch_master_pieces(c, c.ms[c.cur], ops, &c.dyn->max_drho[c.cur], nullptr, c.stream);
            CK(cudaMemsetAsync(&c.dyn->max_drho[2], 0, sizeof(double), c.stream));
        } else {
            launch_master_pieces(c, c.ms[c.cur], ops, nullptr, nullptr, c.stream);
        }
    }
    launch_level(c, lv, c.cur, 0, c.stream);
    CKL();
    return TDB_OK;
}

// After rho_n changes outside a step (ground state, kick, set_state): Mulliken
// partials of rho_n and, for the reduced forms, the master and the operands.
tdb_status refresh_derived(Ctx& c) {
    if (!mixed(c)) {
        launch_mulliken_partials(c.N, c.rho_re[c.cur], c.S, c.partial, c.stream);
        CKL();
        return TDB_OK;
    }
    // the FP64 view is authoritative here: convert both leapfrog levels
    for (int l = 0; l < 2; ++l) launch_view_to_master(c, c.rho_re[l], c.rho_im[l], c.ms[l], c.stream);
    c.view_valid = true;
    return derived_from_master(c);
}

// Reduced forms: bring the FP64 view up to date with the master.
tdb_status materialize(Ctx& c) {
    if (!mixed(c) || c.view_valid) return TDB_OK;
    for (int l = 0; l < 2; ++l) launch_master_to_view(c, c.ms[l], c.rho_re[l], c.rho_im[l], c.stream);
    CKL();
    c.view_valid = true;
    return TDB_OK;
}

// Constants of the reduced forms' per-level evaluation after the ground state: gamma and
// the positions as FP32 pairs, the SCC residual of rho_ref per atom, N_e - sum_A q_A(rho_ref)
// and the dipole of rho_ref (host FP64, once).
tdb_status setup_level_constants(Ctx& c) {
    const int nat = c.nat, N = c.N;
    std::vector<double> g((size_t)nat * nat), qb(nat), vref(N), q0v(nat);
    DevScalars h{};
    CK(cudaMemcpyAsync(g.data(), c.gamma, sizeof(double) * g.size(), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaMemcpyAsync(qb.data(), c.qbase, sizeof(double) * nat, cudaMemcpyDeviceToHost, c.stream));
    CK(cudaMemcpyAsync(vref.data(), c.v_ref, sizeof(double) * N, cudaMemcpyDeviceToHost, c.stream));
    CK(cudaMemcpyAsync(q0v.data(), c.d_q0, sizeof(double) * nat, cudaMemcpyDeviceToHost, c.stream));
    CK(cudaMemcpyAsync(&h, c.sc, sizeof h, cudaMemcpyDeviceToHost, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    auto split = [](double x) {
        const float h = (float)x;
        return make_float2(h, (float)(x - (double)h));
    };
    std::vector<float2> g2(g.size()), r2(3 * (size_t)nat);
    for (size_t i = 0; i < g.size(); ++i) g2[i] = split(g[i]);
    for (int i = 0; i < 3 * nat; ++i) r2[i] = split(c.R[i]);
    std::vector<float> cres(nat);
    double qsum = 0.0, mu[3] = {0.0, 0.0, 0.0};
    for (int A = 0; A < nat; ++A) {
        qsum += qb[A];
        const double dq = qb[A] - q0v[A];
        for (int k = 0; k < 3; ++k) mu[k] -= dq * c.R[3 * A + k];
        double gd = 0.0;
        if (c.prm.scc)
            for (int B = 0; B < nat; ++B) gd += g[(size_t)A * nat + B] * (qb[B] - q0v[B]);
        cres[A] = c.prm.scc ? (float)(gd - vref[(size_t)A * c.nper]) : 0.0f;
    }
    h.c0_trace = c.n_electrons - qsum;
    h.n_e = c.n_electrons;
    for (int k = 0; k < 3; ++k) h.mu_ref[k] = mu[k];
    h.eps_lvl[0] = h.eps_lvl[1] = 0.0f;
    CK(cudaMemcpyAsync(c.gam2, g2.data(), sizeof(float2) * g2.size(), cudaMemcpyHostToDevice, c.stream));
    CK(cudaMemcpyAsync(c.R2, r2.data(), sizeof(float2) * r2.size(), cudaMemcpyHostToDevice, c.stream));
    CK(cudaMemcpyAsync(c.c_res, cres.data(), sizeof(float) * nat, cudaMemcpyHostToDevice, c.stream));
    CK(cudaMemsetAsync(c.lv_count, 0, sizeof(int) * 2, c.stream));
    CK(cudaMemcpyAsync(c.sc, &h, sizeof h, cudaMemcpyHostToDevice, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    return TDB_OK;
}

// Tensor-core form setup after the ground state: scales, constant operands.
tdb_status setup_tensor(Ctx& c) {
    const int N = c.N, b = piece_bf16(c);
    const size_t NN = (size_t)N * N;
    double* dmax = c.obs_out + 8;
    double mx[3];
    const double* srcs[3] = {c.Sinv, c.M, c.rho_ref};
    for (int i = 0; i < 3; ++i) {
        CK(cudaMemsetAsync(dmax, 0, sizeof(double), c.stream));
        launch_absmax(NN, srcs[i], dmax, c.stream);
        CK(cudaMemcpyAsync(&mx[i], dmax, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
        CK(cudaStreamSynchronize(c.stream));
    }
    tc::DynScales d{};
    if (b) {
        c.s_sinv = c.s_dh = c.s_m = c.s_rho = c.s_ref = 1.0f;
    } else if (!head3(c)) {
        c.s_sinv = pow2_scale(mx[0], 2048.0);
        c.s_dh = 4096.0f;                              // |delta H| < 16 Ha
        c.s_m = pow2_scale(std::max(mx[1], 1.0 / 16), 1024.0);
        c.s_rho = c.s_ref = pow2_scale(std::max(mx[2], 0.5), 1024.0);
    } else {
        // integer heads: a matrix bound m maps to (32, 64], leaving 2x to the +-127 clamp
        c.s_sinv = tc::pscale(mx[0]);
        c.s_m = tc::pscale(mx[1] * 1.5);
        c.s_ref = tc::pscale(mx[2]);
        // ||S^-1||_inf bounds |delta M| / max |delta H|
        std::vector<double> h(NN);
        CK(cudaMemcpy(h.data(), c.Sinv, sizeof(double) * NN, cudaMemcpyDeviceToHost));
        double nrm = 0;
        for (int r = 0; r < N; ++r) {
            double sum = 0;
            for (int k = 0; k < N; ++k) sum += std::fabs(h[(size_t)r * N + k]);
            nrm = std::max(nrm, sum);
        }
        d.sinv_norm = nrm;
    }
    d.s_dh = c.s_dh;
    d.s_dm = c.s_m;     // hi/lo schemes: delta M shares the scale of M
    d.s_rho = c.s_rho;
    CK(cudaMemcpyAsync(c.dyn, &d, sizeof d, cudaMemcpyHostToDevice, c.stream));
    tc::launch_split(c.scheme, N, N, c.Sinv, N, c.s_sinv, 1, b, c.pc_sinv, c.Np, c.stream, nullptr,
                     nullptr, c.d_err);
    tc::launch_split(c.scheme, N, N, c.rho_ref, N, c.s_ref, 1, b, c.pc_bre, 2 * c.Np, c.stream,
                     nullptr, nullptr, c.d_err);
    CKL();
    CK(cudaStreamSynchronize(c.stream));
    return TDB_OK;
}

// Width of the X tiles: 128 x 256 tiles read half as much shared memory per MMA as
// 128 x 128 ones (the split products re-read each piece several times, and shared-memory
// bandwidth is what bounds the 128-wide tiles); small systems keep 128.  For
// 768 < N <= 1024 (one K slice) 176-wide tiles give 3 parts x 8 x 6 = 144 CTAs, one wave
// on the 152 SMs (256-wide tiles: 96).
// tune_x replaces this starting guess by the measured fastest width.
int default_xbn(int N) {
    if (N > 768 && N <= 1024) return 176;
    return N >= 512 ? 256 : 128;
}
int xbn(const Ctx& c) { return c.x_bn ? c.x_bn : default_xbn(c.N); }

// Tensor maps of the X product's operands for B tiles of width bn.
bool make_x_maps(const Ctx& c, int bn, tc::Maps& m) {
    const int N = c.N, Np = c.Np, b = piece_bf16(c);
    bool ok = true;
    for (int q = 0; q < c.npieces; ++q)
        ok = ok && tc::make_map(&m.a[q], c.pc_am[q], N, 2 * Np, 2 * Np, b) &&
             tc::make_map(&m.b[0][q], c.pc_bre[q], N, 2 * Np, 2 * Np, b, bn) &&
             tc::make_map(&m.b[1][q], c.pc_bim[q], N, Np, Np, b, bn);
    return ok;
}

tdb_status build_maps(Ctx& c) {
    CK(tc::prepare());
    const int N = c.N, Np = c.Np, b = piece_bf16(c);
    bool ok = true;
    for (int q = 0; q < c.npieces; ++q) {
        ok = ok && tc::make_map(&c.maps_dm.a[q], c.pc_sinv[q], N, N, Np, b) &&
             tc::make_map(&c.maps_dm.b[0][q], c.pc_dh[q], N, N, Np, b, 64);
    }
    ok = ok && make_x_maps(c, xbn(c), c.maps_x);
    if (!ok) {
        set_err("cuTensorMapEncodeTiled failed");
        return TDB_ERR_CUDA;
    }
    return TDB_OK;
}

// S^-1 at the current geometry without synchronising (moving nuclei): Cholesky
// and inverse in the preallocated workspace; a non-positive-definite S shows up as
// NaN through tdb_check.
tdb_status enqueue_inverse(Ctx& c) {
    const int N = c.N;
    CK(cudaMemcpyAsync(c.Sinv, c.S, sizeof(double) * N * N, cudaMemcpyDeviceToDevice, c.stream));
    CKS(cusolverDnDpotrf(c.solver, CUBLAS_FILL_MODE_LOWER, N, c.Sinv, N, c.inv_work, c.inv_lwork,
                         c.inv_info));
    CKS(cusolverDnDpotri(c.solver, CUBLAS_FILL_MODE_LOWER, N, c.Sinv, N, c.inv_work, c.inv_lwork,
                         c.inv_info));
    launch_symmetrize_upper_to_lower(N, c.Sinv, c.stream);
    CKL();
    return TDB_OK;
}

tdb_status oz_product(Ctx& c, int a, int b, double* out);

// S^-1 at a new geometry from the inverse at the previous one (FP64_SLICED form):
// Newton-Schulz steps X <- 2 X - X S X with integer-slice products.  They converge
// quadratically while ||1 - S X|| < 1; between two steps the nuclei move by ~1e-4 bohr,
// so the start is within ~1e-5 and two steps reach the products' precision.
tdb_status ns_inverse(Ctx& c) {
    const int N = c.N;
    oz::slice_rows(c.S, N, 1.0, c.oz[2], c.stream);                 // A = S
    for (int it = 0; it < 2; ++it) {
        oz::slice_rows(c.Sinv, N, 1.0, c.oz[1], c.stream);          // B = X (symmetric)
        TRY(oz_product(c, 2, 1, c.M));                              // P = S X
        oz::slice_rows(c.Sinv, N, 1.0, c.oz[0], c.stream);          // A = X
        oz::slice_cols(c.M, N, c.oz[1], c.oz_colmax, c.stream);     // B = P
        TRY(oz_product(c, 0, 1, c.Hs));                             // Q = X P
        launch_ns_update(N, c.Sinv, c.Hs, c.stream);
    }
    CKL();
    return TDB_OK;
}

// S, H0, gamma and S^-1 at the current device geometry (moving nuclei).  Inside a step
// of the FP64_SLICED form S^-1 follows from the previous one (ns_inverse); otherwise
// (and after a ground state, kick or checkpoint load) it is factorised anew.
tdb_status md_model(Ctx& c, bool in_step = false) {
    launch_build_model(c, c.d_R, c.S, c.H0, c.stream);
    launch_build_gamma(c, c.d_R, c.gamma, c.stream);
    CKL();
    if (in_step && sliced(c)) return ns_inverse(c);
    return enqueue_inverse(c);
}

// Optional per-kernel timing of an enqueued step: an event before each launch.
struct StepTimer {
    std::vector<cudaEvent_t> ev;
    std::vector<const char*> names;
    void mark(cudaStream_t st, const char* name) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        cudaEventRecord(e, st);
        ev.push_back(e);
        names.push_back(name);
    }
    ~StepTimer() {
        for (auto e : ev) cudaEventDestroy(e);
    }
};

#define MARK(name) \
    if (tm) tm->mark(c.stream, name)

// Sliced-form products: out = A B with A, B given through their slices (0: S^-1,
// 1: H or D, 2: M or Y, 3: Re rho, 4: Im rho).
tdb_status oz_product(Ctx& c, int a, int b, double* out) {
    oz::Part part;
    part.b = &c.oz[b];
    part.C = out;
    part.ldc = c.N;
    CK(oz::gemm(c.oz[a], &part, 1, c.d_err, c.stream));
    return TDB_OK;
}
// re = A Re rho, im = A Im rho in one launch
tdb_status oz_product_rho(Ctx& c, int a, double* re, double* im) {
    oz::Part parts[2];
    parts[0].b = &c.oz[3];
    parts[0].C = re;
    parts[0].ldc = c.N;
    parts[1].b = &c.oz[4];
    parts[1].C = im;
    parts[1].ldc = c.N;
    CK(oz::gemm(c.oz[a], parts, 2, c.d_err, c.stream));
    return TDB_OK;
}

// Everything of a moving-nuclei step up to the work rate, for rho_n in buffer cur
// (Sec. 2.3 with the ordering: S_n, S^-1_n; q(rho_n), H_n; X_n; F_n; V_n; D_n; P_n).
// commit = 1 inside a step (the work integral advances), 0 for observables.
tdb_status md_forces(Ctx& c, int cur, bool first, int commit, int* n, StepTimer* tm = nullptr) {
    MARK("md_model_inverse");
    TRY(md_model(c, true));
    MARK("md_charges_potential");
    launch_mulliken_partials(c.N, c.rho_re[cur], c.S, c.partial, c.stream);
    launch_charges(c, c.partial, c.q, c.dq, c.stream);
    launch_potential(c, c.gamma, c.dq, c.d_R, c.sc, c.v_orb, c.v_atom, c.gdq, c.hist, c.v_ref,
                     nullptr, c.stream);
    MARK("md_products_X");
    if (sliced(c)) {
        // M = S^-1 H and X = M rho_n with integer-slice products (S^-1 sliced per step)
        const int N = c.N;
        launch_build_hamiltonian(N, c.H0, c.S, c.v_orb, c.Hs, c.stream);
        oz::slice_rows(c.Sinv, N, 1.0, c.oz[0], c.stream);
        oz::slice_rows(c.Hs, N, 1.0, c.oz[1], c.stream);          // H symmetric
        TRY(oz_product(c, 0, 1, c.M));
        oz::slice_rows(c.M, N, 1.0, c.oz[2], c.stream);
        oz::slice_rows(c.rho_re[cur], N, 1.0, c.oz[3], c.stream);  // Re rho symmetric
        oz::slice_rows(c.rho_im[cur], N, -1.0, c.oz[4], c.stream); // (Im rho)^T = -Im rho
        TRY(oz_product_rho(c, 2, c.Xre, c.Xim));
        if (n) *n += 5;
    } else if (md32(c)) {
        // M = S^-1 H and X = M rho_n with FP32 operands and FFMA accumulation
        const int N = c.N;
        const size_t NN = (size_t)N * N;
        launch_build_hamiltonian(N, c.H0, c.S, c.v_orb, c.Hs, c.stream);
        launch_f64_to_f32(NN, c.Sinv, c.md_sinv, c.stream);
        launch_f64_to_f32(NN, c.Hs, c.md_b, c.stream);
        launch_f64_to_f32(NN, c.rho_re[cur], c.md_rre, c.stream);
        launch_f64_to_f32(NN, c.rho_im[cur], c.md_rim, c.stream);
        gemm_f32(N, N, N, c.md_sinv, N, c.md_b, N, c.md_m, N, c.stream);
        gemm_f32(N, N, N, c.md_m, N, c.md_rre, N, c.md_xre, N, c.stream);
        gemm_f32(N, N, N, c.md_m, N, c.md_rim, N, c.md_xim, N, c.stream);
        launch_f32_to_f64(NN, c.md_xre, c.Xre, c.stream);
        launch_f32_to_f64(NN, c.md_xim, c.Xim, c.stream);
        if (n) *n += 7;
    } else {
        gemm_f64_ham(c.N, c.Sinv, c.H0, c.S, c.v_orb, c.M, c.stream);        // M = S^-1 H
        gemm_f64(c.N, c.N, c.N, c.M, c.N, c.rho_re[cur], c.N, c.Xre, c.N, c.stream);
        gemm_f64(c.N, c.N, c.N, c.M, c.N, c.rho_im[cur], c.N, c.Xim, c.N, c.stream);
    }
    MARK("md_forces");
    launch_wre(c.N, c.Xre, c.Wre, c.stream);
    launch_forces(c, c.rho_re[cur], c.Wre, c.d_F, c.stream);
    launch_vel_n(c, c.d_F, first ? 1 : 0, c.stream);
    MARK("md_nac_power");
    launch_build_nac(c, c.d_Vn, c.D, c.stream);
    launch_power(c, c.Xre, c.D, c.pw_part, kObsBlocks, first ? 1 : 0, commit, c.stream);
    CKL();
    if (n) *n += 16;
    return TDB_OK;
}

// One moving-nuclei step: forces as above, then Z = S^-1 D rho, the update with the
// NAC term, and velocity Verlet for the nuclei.
tdb_status enqueue_step_md(Ctx& c, int cur, bool euler, int* launches, StepTimer* tm = nullptr) {
    const int prv = cur ^ 1;
    int n = 0;
    TRY(md_forces(c, cur, euler, 1, &n, tm));
    MARK("md_products_Z");
    if (sliced(c)) {
        // Y = S^-1 D (D is not symmetric: column slices) and Z = Y rho_n
        oz::slice_cols(c.D, c.N, c.oz[1], c.oz_colmax, c.stream);
        TRY(oz_product(c, 0, 1, c.M));
        oz::slice_rows(c.M, c.N, 1.0, c.oz[2], c.stream);
        TRY(oz_product_rho(c, 2, c.Zre, c.Zim));
        n += 2;
    } else if (md32(c)) {
        // Y = S^-1 D and Z = Y rho_n in FP32 (the FP32 copies of S^-1 and rho_n are current)
        const int N = c.N;
        const size_t NN = (size_t)N * N;
        launch_f64_to_f32(NN, c.D, c.md_b, c.stream);
        gemm_f32(N, N, N, c.md_sinv, N, c.md_b, N, c.md_m, N, c.stream);
        gemm_f32(N, N, N, c.md_m, N, c.md_rre, N, c.md_xre, N, c.stream);
        gemm_f32(N, N, N, c.md_m, N, c.md_rim, N, c.md_xim, N, c.stream);
        launch_f32_to_f64(NN, c.md_xre, c.Zre, c.stream);
        launch_f32_to_f64(NN, c.md_xim, c.Zim, c.stream);
        n += 3;
    } else {
        gemm_f64(c.N, c.N, c.N, c.Sinv, c.N, c.D, c.N, c.M, c.N, c.stream);   // Y = S^-1 D
        gemm_f64(c.N, c.N, c.N, c.M, c.N, c.rho_re[cur], c.N, c.Zre, c.N, c.stream);
        gemm_f64(c.N, c.N, c.N, c.M, c.N, c.rho_im[cur], c.N, c.Zim, c.N, c.stream);
    }
    const double factor = euler ? c.prm.dt : 2.0 * c.prm.dt;
    const double* bre = euler ? c.rho_re[cur] : c.rho_re[prv];
    const double* bim = euler ? c.rho_im[cur] : c.rho_im[prv];
    MARK("md_update_verlet");
    launch_update(c, c.Xre, c.Xim, bre, bim, c.rho_re[prv], c.rho_im[prv], factor, c.S, c.partial,
                  c.sc, c.stream, c.Zre, c.Zim);
    launch_vv(c, c.d_F, c.stream);
    MARK("end");
    CKL();
    if (launches) *launches = n + 5;
    return TDB_OK;
}

// Enqueue one propagation step for rho_n in buffer `cur` (eq:leapfrog, eq:eomrho).
// Parameters of the X product for tiles of width bn; returns the number of parts.
// Parts: X_a = dM rho_ref and X_re = M Re(rho - rho_ref) (the real part of X is their
// sum), then X_im = M Im rho; each cut into x_split K slices.
int x_params(Ctx& c, int bn, tc::GemmParams& x) {
    const int N = c.N, Np = c.Np;
    const bool h3 = head3(c);
    x = tc::GemmParams{};
    x.M = N;
    x.N = N;
    x.idesc = tc::idesc_f16(piece_bf16(c), bn);
    x.bf16 = piece_bf16(c);
    x.err = c.d_err;
    x.max_out = h3 ? c.dyn->max_x : nullptr;
    const int ns = x_split(c);
    const int kc = ((N + ns - 1) / ns + 63) / 64 * 64;
    int nparts = 0;
    for (int prod = 0; prod < 3; ++prod)
        for (int sl = 0; sl < ns; ++sl) {
            const int off = sl * kc, len = std::min(kc, N - off);
            tc::GemmPart& P = x.part[nparts];
            P.k0_a = (prod == 0 ? 0 : Np) + off;
            P.k0_b = (prod == 1 ? Np : 0) + off;
            P.K = len;
            P.mode = 0;
            P.C = c.xp[nparts];
            P.ldc = N;
            P.b_set = prod == 2 ? 1 : 0;
            if (h3) {
                // dM pieces carry s_dm, M pieces s_m; rho_ref pieces s_ref, dRho s_rho
                P.sa = c.s_m;
                P.sa_dev = prod == 0 ? &c.dyn->s_dm : nullptr;
                P.sb = c.s_ref;
                P.sb_dev = prod == 0 ? nullptr : &c.dyn->s_rho;
            } else {
                P.sa = c.s_m;
                P.sb = c.s_rho;
            }
            ++nparts;
        }
    return nparts;
}

// Autotuner of the X product's tile width (tensor-core forms), run once per context
// before the first step is captured: each candidate width times three launches on the
// context's current operands (CUDA events on its stream) and the fastest is kept.  Every
// output element keeps its K order whatever the width, so the choice changes the time,
// not the result.  The launches write only the X partials and the X maxima, which the
// next step overwrites and resets.
tdb_status tune_x(Ctx& c) {
    static const int cand[] = {128, 176, 256};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 0.f;
    int best_bn = 0;
    tdb_status st = TDB_OK;
    for (int bn : cand) {
        tc::Maps m{};
        tc::GemmParams x{};
        if (!make_x_maps(c, bn, m)) continue;   // width not encodable for this size
        const int np = x_params(c, bn, x);
        cudaError_t e = tc::launch(c.scheme, m, x, np, c.stream, bn);   // warm-up
        if (e == cudaErrorInvalidValue) {                               // width not valid here
            cudaGetLastError();
            continue;
        }
        if (e == cudaSuccess) e = cudaEventRecord(e0, c.stream);
        for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = tc::launch(c.scheme, m, x, np, c.stream, bn);
        if (e == cudaSuccess) e = cudaEventRecord(e1, c.stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            set_err("X tile tuning: %s", cudaGetErrorString(e));
            st = TDB_ERR_CUDA;
            break;
        }
        if (!best_bn || ms < best) {
            best = ms;
            best_bn = bn;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != TDB_OK) return st;
    // the timing launches accumulated X maxima: the evaluation of the level had reset them
    if (c.dyn) CK(cudaMemsetAsync(c.dyn->max_x, 0, sizeof(c.dyn->max_x), c.stream));
    if (best_bn) c.x_bn = best_bn;
    if (!make_x_maps(c, xbn(c), c.maps_x)) {
        set_err("cuTensorMapEncodeTiled failed");
        return TDB_ERR_CUDA;
    }
    return TDB_OK;
}

// The four launches of a tensor-form step for rho_n in buffer cur (split of delta H, delta M,
// X, update with the level evaluation), as argument structs: enqueue_step launches them for
// one context, a grouped batch for many at once.
struct TensorStep {
    tc::SplitDhArgs split;
    tc::GemmParams dm;
    tc::GemmParams x;
    int x_parts, x_bn;
    UpdateDfArgs upd;
};

TensorStep tensor_step_args(Ctx& c, int cur, bool euler, int bn) {
    const int N = c.N, Np = c.Np, b = piece_bf16(c), prv = cur ^ 1;
    const bool h3 = head3(c);
    TensorStep ts{};
    ts.split = tc::split_dham_args(c.scheme, N, c.S_f, c.dv_f, c.s_dh, b, c.pc_dh, Np,
                                   h3 ? c.dyn : nullptr, c.d_err);
    // delta M = S^-1 delta H; the epilogue writes the pieces of [delta M | M_gs + delta M]
    tc::GemmParams& g = ts.dm;
    g.M = N;
    g.N = N;
    g.part[0] = {0, 0, N, 1, nullptr, 0, c.s_sinv, 0.f, nullptr, h3 ? &c.dyn->s_dh : nullptr, 0};
    g.part[0].sb = c.s_dh;
    g.idesc = tc::idesc_f16(b, 64);
    g.bf16 = b;
    g.Mgs = c.Mgs_f;
    g.ld_mgs = N;
    for (int q = 0; q < 3; ++q) g.out[q] = c.pc_am[q];
    g.ld_out = 2 * Np;
    g.col_m = Np;
    g.s_m = c.s_m;
    g.s_dm_dev = &c.dyn->s_dm;
    g.err = c.d_err;
    ts.x_bn = bn;
    ts.x_parts = x_params(c, bn, ts.x);
    // the update writes the pieces of rho_{n+1} - rho_ref itself (FP16X6: scaled from a
    // bound on their size) and tracks their maximum
    const int ns = x_split(c);
    UpdateOperands ops = master_operands(c);
    ops.cur = cur;
    ops.base_slot = euler ? cur : prv;
    ops.nre = 2 * ns;
    ops.nim = ns;
    for (int q = 0; q < 2 * ns; ++q) ops.xre[q] = c.xp[q];
    for (int q = 0; q < ns; ++q) ops.xim[q] = c.xp[2 * ns + q];
    const double factor = euler ? c.prm.dt : 2.0 * c.prm.dt;
    ts.upd = update_df_args(c, euler ? c.ms[cur] : c.ms[prv], c.ms[prv], factor, c.sc, ops,
                            level_args(c));
    // each product prefetches into L2 the operands the next kernel reads from DRAM: delta M
    // the B pieces of the X product, X the base level and S of the update
    const size_t NN4 = sizeof(float) * (size_t)N * N;
    L2Prefetch& d = ts.dm.pf;
    d.n = 0;
    for (int q = 0; q < c.npieces; ++q) {
        d.ptr[d.n] = c.pc_bre[q];
        d.bytes[d.n++] = sizeof(uint16_t) * (size_t)N * 2 * Np;
    }
    for (int q = 0; q < c.npieces && d.n < 6; ++q) {
        d.ptr[d.n] = c.pc_bim[q];
        d.bytes[d.n++] = sizeof(uint16_t) * (size_t)N * Np;
    }
    d.parts = ((N + 63) / 64) * ((N + 127) / 128);
    L2Prefetch& x = ts.x.pf;
    const MasterPtrs& bm = ts.upd.base;
    const void* reg[5] = {bm.re_hi, bm.re_lo, bm.im_hi, bm.im_lo, c.S_f};
    x.n = 5;
    for (int r = 0; r < 5; ++r) {
        x.ptr[r] = reg[r];
        x.bytes[r] = NN4;
    }
    x.parts = ((N + bn - 1) / bn) * ((N + 127) / 128) * ts.x_parts;
    return ts;
}

tdb_status enqueue_step(Ctx& c, int cur, bool euler, int* launches, StepTimer* tm = nullptr) {
    const int prv = cur ^ 1;
    const double factor = euler ? c.prm.dt : 2.0 * c.prm.dt;
    const double* bre = euler ? c.rho_re[cur] : c.rho_re[prv];
    const double* bim = euler ? c.rho_im[cur] : c.rho_im[prv];
    int n = 0;
    if (!mixed(c)) {
        // charges and SCC potential of rho_n (the reduced forms evaluate the new level after
        // the update, and the current one after a ground state, kick or state load)
        MARK("charges");
        launch_charges(c, c.partial, c.q, c.dq, c.stream);
        ++n;
        MARK("potential");
        launch_potential(c, c.gamma, c.dq, c.d_R, c.sc, c.v_orb, c.v_atom, c.gdq, c.hist, c.v_ref,
                         nullptr, c.stream);
        ++n;
    }
    if (sliced(c)) {
        const int N = c.N;
        MARK("slice_H");
        launch_build_hamiltonian(N, c.H0, c.S, c.v_orb, c.Hs, c.stream);
        oz::slice_rows(c.Hs, N, 1.0, c.oz[1], c.stream);
        MARK("oz_gemm_M");
        TRY(oz_product(c, 0, 1, c.M));                          // M = S^-1 H
        MARK("slice_M_rho");
        oz::slice_rows(c.M, N, 1.0, c.oz[2], c.stream);
        oz::slice_rows(c.rho_re[cur], N, 1.0, c.oz[3], c.stream);
        oz::slice_rows(c.rho_im[cur], N, -1.0, c.oz[4], c.stream);
        MARK("oz_gemm_X");
        TRY(oz_product_rho(c, 2, c.Xre, c.Xim));                // X = M rho
        n += 7;
        MARK("update");
        launch_update(c, c.Xre, c.Xim, bre, bim, c.rho_re[prv], c.rho_im[prv], factor, c.S,
                      c.partial, c.sc, c.stream);
        ++n;
    } else if (c.prm.precision == TDB_FP64) {
        MARK("gemm_M_f64");
        gemm_f64_ham(c.N, c.Sinv, c.H0, c.S, c.v_orb, c.M, c.stream);  // M = S^-1 H
        MARK("gemm_Xre_f64");
        gemm_f64(c.N, c.N, c.N, c.M, c.N, c.rho_re[cur], c.N, c.Xre, c.N, c.stream);
        MARK("gemm_Xim_f64");
        gemm_f64(c.N, c.N, c.N, c.M, c.N, c.rho_im[cur], c.N, c.Xim, c.N, c.stream);
        n += 3;
        MARK("update");
        launch_update(c, c.Xre, c.Xim, bre, bim, c.rho_re[prv], c.rho_im[prv], factor, c.S,
                      c.partial, c.sc, c.stream);
        ++n;
    } else if (tensor(c)) {
        const TensorStep ts = tensor_step_args(c, cur, euler, xbn(c));
        MARK("split_dH");
        tc::launch_split_dham(c.scheme, ts.split.N, ts.split.S, ts.split.dv, ts.split.scale,
                              ts.split.bf16, ts.split.out, ts.split.ld_out, ts.split.dyn, c.stream,
                              ts.split.err);
        ++n;
        MARK("tc_gemm_dM");
        CK(tc::launch(c.scheme, c.maps_dm, ts.dm, 1, c.stream, 64));
        ++n;
        MARK("tc_gemm_X");
        CK(tc::launch(c.scheme, c.maps_x, ts.x, ts.x_parts, c.stream, ts.x_bn));
        ++n;
        MARK("update");
        launch_update_df(c, ts.upd.base, ts.upd.out, factor, c.sc, ts.upd.ops, ts.upd.lv, c.stream);
        ++n;
        MARK("level_dq");
        launch_level_dq(c, ts.upd.lv, c.stream);
        MARK("level");
        launch_level_final(c, ts.upd.lv, ts.upd.out_slot, c.stream);
        n += 2;
    } else {
        const int N = c.N;
        // delta M = S^-1 delta H (left half of [dM | M]), M = M_gs + delta M (right half)
        MARK("gemm_dM_f32");
        gemm_f32_dham(N, c.Sinv_f, c.S_f, c.dv_f, c.dM_f, 2 * N, nullptr, c.stream);
        ++n;
        MARK("add_M");
        launch_add_f32_strided(N, c.Mgs_f, c.dM_f, 2 * N, c.M_f, 2 * N, c.stream);
        ++n;
        // X_re = dM rho_ref + M Re(rho - rho_ref);  X_im = M Im rho (master hi parts)
        MARK("gemm_Xre_f32");
        gemm_f32_add(N, N, N, c.dM_f, 2 * N, c.rref_f, N, c.Xre_f, N, nullptr, c.stream);
        gemm_f32_add(N, N, N, c.M_f, 2 * N, c.ms[cur].re_hi, N, c.Xre_f, N, c.Xre_f, c.stream);
        MARK("gemm_Xim_f32");
        gemm_f32_add(N, N, N, c.M_f, 2 * N, c.ms[cur].im_hi, N, c.Xim_f, N, nullptr, c.stream);
        n += 3;
        MARK("update");
        UpdateOperands ops;
        ops.cur = cur;
        ops.xre[0] = c.Xre_f;
        ops.xim[0] = c.Xim_f;
        ops.nre = ops.nim = 1;
        ops.base_slot = euler ? cur : prv;
        launch_update_df(c, euler ? c.ms[cur] : c.ms[prv], c.ms[prv], factor, c.sc, ops,
                         level_args(c), c.stream);
        ++n;
        MARK("level_dq");
        launch_level_dq(c, level_args(c), c.stream);
        MARK("level");
        launch_level_final(c, level_args(c), prv, c.stream);
        n += 2;
    }
    MARK("end");
    CKL();
    if (launches) *launches = n;
    return TDB_OK;
}

tdb_status ensure_graph(Ctx& c, int cur) {
    if (c.graph[cur]) return TDB_OK;
    if (tensor(c) && !c.x_bn && !c.graph[cur ^ 1]) TRY(tune_x(c));
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal));
    int nl = 0;
    tdb_status st = enqueue_step(c, cur, false, &nl);
    cudaError_t e = cudaStreamEndCapture(c.stream, &g);
    if (st != TDB_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) {
        set_err("graph capture failed: %s", cudaGetErrorString(e));
        return TDB_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&c.graph[cur], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        set_err("graph instantiate failed: %s", cudaGetErrorString(e));
        return TDB_ERR_CUDA;
    }
    c.graph_launches = nl;
    return TDB_OK;
}

tdb_status build_inverse(Ctx& c) {
    const int N = c.N;
    CK(cudaMemcpyAsync(c.Sinv, c.S, sizeof(double) * N * N, cudaMemcpyDeviceToDevice, c.stream));
    int lwork = 0;
    CKS(cusolverDnDpotrf_bufferSize(c.solver, CUBLAS_FILL_MODE_LOWER, N, c.Sinv, N, &lwork));
    int lwork2 = 0;
    CKS(cusolverDnDpotri_bufferSize(c.solver, CUBLAS_FILL_MODE_LOWER, N, c.Sinv, N, &lwork2));
    lwork = std::max(lwork, lwork2);
    double* work = nullptr;
    int* info = nullptr;
    CK(cudaMalloc(&work, sizeof(double) * std::max(lwork, 1) + 256));
    info = reinterpret_cast<int*>(reinterpret_cast<char*>(work) + sizeof(double) * std::max(lwork, 1));
    tdb_status rc = TDB_OK;
    int h_info = 0;
    if (cusolverDnDpotrf(c.solver, CUBLAS_FILL_MODE_LOWER, N, c.Sinv, N, work, lwork, info) !=
        CUSOLVER_STATUS_SUCCESS) {
        set_err("cusolverDnDpotrf failed");
        rc = TDB_ERR_CUDA;
    }
    if (rc == TDB_OK && cudaMemcpyAsync(&h_info, info, sizeof(int), cudaMemcpyDeviceToHost,
                                        c.stream) == cudaSuccess &&
        cudaStreamSynchronize(c.stream) == cudaSuccess && h_info != 0) {
        set_err("overlap matrix is not positive definite (potrf info %d)", h_info);
        rc = TDB_ERR_NOT_SPD;
    }
    if (rc == TDB_OK &&
        cusolverDnDpotri(c.solver, CUBLAS_FILL_MODE_LOWER, N, c.Sinv, N, work, lwork, info) !=
            CUSOLVER_STATUS_SUCCESS) {
        set_err("cusolverDnDpotri failed");
        rc = TDB_ERR_CUDA;
    }
    if (rc == TDB_OK) {
        // column-major lower == row-major upper
        launch_symmetrize_upper_to_lower(N, c.Sinv, c.stream);
        if (cudaStreamSynchronize(c.stream) != cudaSuccess) rc = TDB_ERR_CUDA;
    }
    cudaFree(work);
    return rc;
}

tdb_status check_ctx(tdb_ctx* c, bool need_gs, bool allow_sticky) {
    if (!c) {
        set_err("NULL context");
        return TDB_ERR_ARG;
    }
    if (c->sticky && !allow_sticky) {
        set_err("context is in an error state (numeric or timeout)");
        return TDB_ERR_STATE;
    }
    if (need_gs && !c->have_gs) {
        set_err("call tdb_ground_state (or tdb_set_state) first");
        return TDB_ERR_STATE;
    }
    return TDB_OK;
}

constexpr unsigned long long kStateMagic = 0x7464625374617465ull;  // "tdbState"

struct StateHeader {
    unsigned long long magic;
    long long N, nat, n, n_base;
    double t_base, work, dt;
    int euler_next, precision;
    double P_prev;   // moving nuclei: work rate of the previous step
};

// TDB_ERR_CUDA with a message when no CUDA device is usable (checked before any
// allocation, so that a host without a GPU gets a clear status, not an allocation one).
tdb_status require_device(const char* who) {
    int ndev = 0;
    const cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        set_err("%s: no usable CUDA device (%s)", who,
                e != cudaSuccess ? cudaGetErrorString(e) : "device count 0");
        return TDB_ERR_CUDA;
    }
    return TDB_OK;
}

}  // namespace

extern "C" {

void tdb_default_params(tdb_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->dt = 0.2;
    p->scc = 1;
    p->move_nuclei = 0;
    p->precision = TDB_FP64;
    p->window = 100;
    p->scc_tol = 1e-12;
    p->scc_max_iter = 400;
    p->kT = 0.0;
    p->scc_mix = 0.3;
    p->history_cap = 65536;
    p->cuda_stream = nullptr;
}

size_t tdb_workspace_bytes(const tdb_system* sys, const tdb_params* prm) {
    if (validate(sys, prm) != TDB_OK) return 0;
    Ctx c;
    fill_host(c, sys, prm);
    return carve(c, nullptr);
}

tdb_status tdb_create(const tdb_system* sys, const tdb_params* prm, void* workspace,
                      size_t workspace_bytes, tdb_ctx** out) {
    if (!out) {
        set_err("NULL out");
        return TDB_ERR_ARG;
    }
    *out = nullptr;
    TRY(validate(sys, prm));
    TRY(require_device("tdb_create"));
    tdb_ctx* c = new (std::nothrow) tdb_ctx();
    if (!c) return TDB_ERR_NOMEM;
    fill_host(*c, sys, prm);
    const size_t need = carve(*c, nullptr);
    c->ws_need = need;
    auto fail = [&](tdb_status s) {
        tdb_destroy(c);
        return s;
    };
    c->h_pinned_bytes = 4096 + sizeof(double) * (size_t)c->N;   // charges, or N doubles for a window
    if (cudaMallocHost(reinterpret_cast<void**>(&c->h_pinned), c->h_pinned_bytes) != cudaSuccess) {
        cudaGetLastError();
        set_err("cudaMallocHost failed");
        return fail(TDB_ERR_NOMEM);
    }
    if (prm->cuda_stream) {
        c->stream = reinterpret_cast<cudaStream_t>(prm->cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            set_err("cudaStreamCreate failed");
            return fail(TDB_ERR_CUDA);
        }
        c->own_stream = true;
    }
    if (workspace) {
        if (workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255)) {
            set_err("workspace too small (%zu < %zu) or not 256-byte aligned", workspace_bytes,
                    need);
            return fail(TDB_ERR_NOMEM);
        }
        c->ws = workspace;
        c->ws_bytes = workspace_bytes;
    } else {
        if (cudaMalloc(&c->ws, need) != cudaSuccess) {
            cudaGetLastError();
            set_err("cudaMalloc of %zu bytes failed", need);
            return fail(TDB_ERR_NOMEM);
        }
        c->own_ws = true;
        c->ws_bytes = need;
    }
    char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(c->ws) + 255) & ~(uintptr_t)255);
    carve(*c, base);
    if (cudaMemsetAsync(c->ws, 0, c->ws_bytes, c->stream) != cudaSuccess) return fail(TDB_ERR_CUDA);
    // per-atom / per-orbital host tables
    std::vector<double> onsite(c->N), Ua(c->nat), ma(c->nat), q0(c->nat, c->n_electrons / c->nat);
    for (int a = 0; a < c->nat; ++a) {
        const int sp = c->species[a];
        for (int i = 0; i < c->nper; ++i) onsite[a * c->nper + i] = i == 0 ? c->eps_s[sp] : c->eps_p[sp];
        Ua[a] = c->U[sp];
        ma[a] = c->mass[sp];
    }
    struct Up {
        double* d;
        const double* h;
        size_t n;
    } ups[] = {{c->d_R, c->R.data(), c->R.size()},       {c->d_V, c->V.data(), c->V.size()},
               {c->d_onsite, onsite.data(), onsite.size()}, {c->d_U, Ua.data(), Ua.size()},
               {c->d_mass, ma.data(), ma.size()},        {c->d_q0, q0.data(), q0.size()}};
    for (auto& u : ups)
        if (cudaMemcpyAsync(u.d, u.h, sizeof(double) * u.n, cudaMemcpyHostToDevice, c->stream) !=
            cudaSuccess)
            return fail(TDB_ERR_CUDA);
    if (upload_clock(*c, 0, 0, 0.0) != TDB_OK) return fail(TDB_ERR_CUDA);
    if (upload_field(*c) != TDB_OK) return fail(TDB_ERR_CUDA);
    launch_build_model(*c, c->d_R, c->S, c->H0, c->stream);
    launch_build_gamma(*c, c->d_R, c->gamma, c->stream);
    if (cudaGetLastError() != cudaSuccess) {
        set_err("model build launch failed");
        return fail(TDB_ERR_CUDA);
    }
    if (cusolverDnCreate(&c->solver) != CUSOLVER_STATUS_SUCCESS ||
        cusolverDnSetStream(c->solver, c->stream) != CUSOLVER_STATUS_SUCCESS) {
        set_err("cusolverDnCreate failed");
        return fail(TDB_ERR_CUDA);
    }
    tdb_status s = build_inverse(*c);
    if (s != TDB_OK) return fail(s);
    if (c->prm.move_nuclei) {
        int l1 = 0, l2 = 0;
        if (cusolverDnDpotrf_bufferSize(c->solver, CUBLAS_FILL_MODE_LOWER, c->N, c->Sinv, c->N, &l1) !=
                CUSOLVER_STATUS_SUCCESS ||
            cusolverDnDpotri_bufferSize(c->solver, CUBLAS_FILL_MODE_LOWER, c->N, c->Sinv, c->N, &l2) !=
                CUSOLVER_STATUS_SUCCESS) {
            set_err("cusolver buffer size query failed");
            return fail(TDB_ERR_CUDA);
        }
        c->inv_lwork = std::max(std::max(l1, l2), 1);
        if (cudaMalloc(&c->inv_work, sizeof(double) * c->inv_lwork + 256) != cudaSuccess) {
            cudaGetLastError();
            set_err("cudaMalloc of the inverse workspace failed");
            return fail(TDB_ERR_NOMEM);
        }
        c->inv_info = reinterpret_cast<int*>(reinterpret_cast<char*>(c->inv_work) +
                                             sizeof(double) * c->inv_lwork);
        if (cudaMemcpyAsync(c->d_Vn, c->d_V, sizeof(double) * 3 * c->nat, cudaMemcpyDeviceToDevice,
                            c->stream) != cudaSuccess)
            return fail(TDB_ERR_CUDA);
    }
    if (mixed(*c)) launch_f64_to_f32((size_t)c->N * c->N, c->S, c->S_f, c->stream);
    if (c->prm.precision == TDB_FP32 && !c->prm.move_nuclei)
        launch_f64_to_f32((size_t)c->N * c->N, c->Sinv, c->Sinv_f, c->stream);
    if (tensor(*c)) {
        s = build_maps(*c);
        if (s != TDB_OK) return fail(s);
    }
    if (sliced(*c)) {
        const int N = c->N;
        bool ok = oz::prepare() == cudaSuccess;
        for (int q = 0; q < 5 && ok; ++q)
            ok = oz::sliced_init(c->oz[q], c->oz_raw[q], N, N, q == 0 || q == 2 ? 128 : 64);
        if (!ok) {
            set_err("integer-slice GEMM setup failed");
            return fail(TDB_ERR_CUDA);
        }
        // frozen nuclei: S^-1 is sliced once
        if (!c->prm.move_nuclei) oz::slice_rows(c->Sinv, N, 1.0, c->oz[0], c->stream);
    }
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
        set_err("setup failed: %s", cudaGetErrorString(cudaGetLastError()));
        return fail(TDB_ERR_CUDA);
    }
    *out = c;
    return TDB_OK;
}

tdb_status tdb_ground_state(tdb_ctx* c, int* iters_out, double* residual_out) {
    TRY(check_ctx(c, false, false));
    const int N = c->N, nat = c->nat;
    double* d_eig = c->obs_out + 16;
    if (c->prm.move_nuclei) {
        TRY(md_model(*c));
        CK(cudaMemsetAsync(c->md, 0, sizeof(MdScalars), c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    double* d_occ = c->obs_out + 16 + N;
    // the ground state is field-free; the field applies from t = 0 on
    const bool saved_on = c->field_on;
    c->field_on = false;
    TRY(upload_field(*c));
    TRY(upload_clock(*c, 0, 0, 0.0));
    int lwork = 0;
    CKS(cusolverDnDsygvd_bufferSize(c->solver, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR,
                                    CUBLAS_FILL_MODE_LOWER, N, c->Hs, N, c->M, N, d_eig, &lwork));
    double* work = nullptr;
    CK(cudaMalloc(&work, sizeof(double) * std::max(lwork, 1) + 256));
    int* info = reinterpret_cast<int*>(reinterpret_cast<char*>(work) + sizeof(double) * std::max(lwork, 1));
    std::vector<double> dq_in(nat, 0.0), dq_out(nat), eig(N), occ(N), resid(nat), pres(nat);
    std::vector<double> h_gamma;
    if (c->prm.scc) {
        h_gamma.resize((size_t)nat * nat);
        CK(cudaMemcpyAsync(h_gamma.data(), c->gamma, sizeof(double) * nat * nat,
                           cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    Anderson mixer{8, c->prm.scc_mix, {}, {}};
    tdb_status rc = TDB_ERR_SCC_NOCONV;
    double res = 0.0;
    int it = 0;
    for (it = 1; it <= c->prm.scc_max_iter; ++it) {
        if (cudaMemcpyAsync(c->dq, dq_in.data(), sizeof(double) * nat, cudaMemcpyHostToDevice,
                            c->stream) != cudaSuccess) {
            rc = TDB_ERR_CUDA;
            break;
        }
        launch_potential(*c, c->gamma, c->dq, c->d_R, c->sc, c->v_orb, c->v_atom, c->gdq, c->hist,
                         c->v_ref, nullptr, c->stream);
        launch_build_hamiltonian(N, c->H0, c->S, c->v_orb, c->Hs, c->stream);
        cudaMemcpyAsync(c->M, c->S, sizeof(double) * N * N, cudaMemcpyDeviceToDevice, c->stream);
        if (cusolverDnDsygvd(c->solver, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR,
                             CUBLAS_FILL_MODE_LOWER, N, c->Hs, N, c->M, N, d_eig, work, lwork,
                             info) != CUSOLVER_STATUS_SUCCESS) {
            set_err("cusolverDnDsygvd failed");
            rc = TDB_ERR_CUDA;
            break;
        }
        int h_info = 0;
        cudaMemcpyAsync(&h_info, info, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
        cudaMemcpyAsync(eig.data(), d_eig, sizeof(double) * N, cudaMemcpyDeviceToHost, c->stream);
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
            set_err("ground state: %s", cudaGetErrorString(cudaGetLastError()));
            rc = TDB_ERR_CUDA;
            break;
        }
        if (h_info != 0) {
            set_err("generalised eigensolver failed (info %d)", h_info);
            rc = h_info > N ? TDB_ERR_NOT_SPD : TDB_ERR_CUDA;
            break;
        }
        occupations(eig, c->n_electrons, c->prm.kT, occ);
        cudaMemcpyAsync(d_occ, occ.data(), sizeof(double) * N, cudaMemcpyHostToDevice, c->stream);
        // rho_0 = sum_i f_i z_i z_i^T: Z (column-major) read row-major is Zr[i][:] = z_i
        launch_transpose(N, c->Hs, c->Xim, c->stream);             // Xim[a][i] = z_i[a]
        launch_scale_rows_f(N, c->Xim, d_occ, c->Xim, c->stream);  // * f_i
        gemm_f64(N, N, N, c->Xim, N, c->Hs, N, c->rho_re[0], N, c->stream);
        cudaMemsetAsync(c->rho_im[0], 0, sizeof(double) * N * N, c->stream);
        launch_mulliken_partials(N, c->rho_re[0], c->S, c->partial, c->stream);
        launch_charges(*c, c->partial, c->q, c->dq, c->stream);
        cudaMemcpyAsync(dq_out.data(), c->dq, sizeof(double) * nat, cudaMemcpyDeviceToHost,
                        c->stream);
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
            set_err("ground state: %s", cudaGetErrorString(cudaGetLastError()));
            rc = TDB_ERR_CUDA;
            break;
        }
        res = 0.0;
        for (int a = 0; a < nat; ++a) {
            resid[a] = dq_out[a] - dq_in[a];
            res = std::max(res, std::fabs(resid[a]));
        }
        if (!std::isfinite(res)) {
            set_err("ground state produced NaN");
            rc = TDB_ERR_NUMERIC;
            break;
        }
        if (!c->prm.scc || res <= c->prm.scc_tol) {
            if (!c->prm.scc) res = 0.0;
            rc = TDB_OK;
            break;
        }
        scc_precondition(eig, c->n_electrons, c->prm.kT, h_gamma, resid, pres);
        mixer.next(dq_in, pres);
    }
    cudaFree(work);
    if (iters_out) *iters_out = std::min(it, c->prm.scc_max_iter);
    if (residual_out) *residual_out = res;
    c->field_on = saved_on;
    TRY(upload_field(*c));
    if (rc != TDB_OK) {
        if (rc == TDB_ERR_SCC_NOCONV) set_err("SCC not converged: residual %.3e", res);
        return rc;
    }
    // rho_0 = Z f Z^T is symmetric only up to rounding; make it exactly symmetric
    launch_hermitian_half(N, c->rho_re[0], c->rho_im[0], c->Xre, c->Xim, c->stream);
    CK(cudaMemcpyAsync(c->rho_re[0], c->Xre, sizeof(double) * N * N, cudaMemcpyDeviceToDevice,
                       c->stream));
    CK(cudaMemcpyAsync(c->rho_im[0], c->Xim, sizeof(double) * N * N, cudaMemcpyDeviceToDevice,
                       c->stream));
    c->spectral_width = eig[N - 1] - eig[0];
    c->cur = 0;
    c->euler_next = true;
    c->have_gs = true;
    c->work = 0.0;
    // ground-state potential and operands of the reduced-precision forms:
    // v_ref = v of the Hamiltonian whose eigenvectors built rho_0
    CK(cudaMemcpyAsync(c->v_ref, c->v_orb, sizeof(double) * N, cudaMemcpyDeviceToDevice, c->stream));
    if (mixed(*c)) {
        const size_t NN = (size_t)N * N;
        CK(cudaMemcpyAsync(c->rho_ref, c->rho_re[0], sizeof(double) * NN,
                           cudaMemcpyDeviceToDevice, c->stream));
        gemm_f64_ham(N, c->Sinv, c->H0, c->S, c->v_ref, c->M, c->stream);  // M_gs
        launch_f64_to_f32(NN, c->M, c->Mgs_f, c->stream);
        launch_f64_to_f32(NN, c->rho_ref, c->rref_f, c->stream);
        // Mulliken populations of rho_ref: the step adds those of rho - rho_ref
        launch_mulliken_partials(N, c->rho_ref, c->S, c->partial, c->stream);
        launch_charges(*c, c->partial, c->qbase, c->dq, c->stream);
        CKL();
        TRY(setup_level_constants(*c));
        if (tensor(*c)) TRY(setup_tensor(*c));
    }
    TRY(upload_clock(*c, 0, 0, 0.0));
    TRY(refresh_derived(*c));
    CK(cudaStreamSynchronize(c->stream));
    return TDB_OK;
}

tdb_status tdb_kick(tdb_ctx* c, double strength, const double dir[3]) {
    TRY(check_ctx(c, true, false));
    if (!dir || !std::isfinite(strength)) {
        set_err("invalid kick");
        return TDB_ERR_ARG;
    }
    const int N = c->N, cur = c->cur;
    TRY(materialize(*c));
    if (c->prm.move_nuclei) TRY(md_model(*c));
    // eq:rhokick: T = e^{iV} rho S e^{-iV} S^-1,  rho(0+) = 1/2 (T + T^dagger)
    gemm_f64(N, N, N, c->rho_re[cur], N, c->S, N, c->Xre, N, c->stream);
    gemm_f64(N, N, N, c->rho_im[cur], N, c->S, N, c->Xim, N, c->stream);
    launch_kick_phase(N, c->nper, c->d_R, strength, dir, c->Xre, c->Xim, c->M, c->Hs, c->stream);
    gemm_f64(N, N, N, c->M, N, c->Sinv, N, c->Xre, N, c->stream);
    gemm_f64(N, N, N, c->Hs, N, c->Sinv, N, c->Xim, N, c->stream);
    launch_hermitian_half(N, c->Xre, c->Xim, c->rho_re[cur], c->rho_im[cur], c->stream);
    CKL();
    c->euler_next = true;
    TRY(refresh_derived(*c));
    CK(cudaStreamSynchronize(c->stream));
    return TDB_OK;
}

tdb_status tdb_set_field(tdb_ctx* c, const tdb_field* f) {
    TRY(check_ctx(c, false, false));
    if (f) {
        if (!std::isfinite(f->E0) || !std::isfinite(f->omega) || f->envelope < 0 ||
            f->envelope > 2 || (f->envelope > 0 && !(f->fwhm > 0))) {
            set_err("invalid field");
            return TDB_ERR_ARG;
        }
        c->field = *f;
        c->field_on = true;
    } else {
        c->field_on = false;
    }
    TRY(upload_field(*c));
    if (mixed(*c) && c->have_gs) {
        // the reduced forms evaluated rho_n's potential with the old field: redo it
        launch_level(*c, level_args(*c), c->cur, 0, c->stream);
        CKL();
    }
    CK(cudaStreamSynchronize(c->stream));
    return TDB_OK;
}

}  // extern "C"

namespace {

// FP64 Mulliken charges and SCC potential of the current rho_n into q, dq, gdq, v_atom,
// v_orb (for observables).  The FP64 forms also record the dipole and field of rho_n; the
// reduced forms keep the record their level evaluation made and change nothing the next
// step reads.
tdb_status fp64_charges_potential(Ctx& c) {
    if (mixed(c)) {
        launch_charges_df(c, reinterpret_cast<const float2*>(c.partial), c.q, c.dq, c.stream);
        launch_potential(c, c.gamma, c.dq, c.d_R, c.sc, c.v_orb, c.v_atom, c.gdq, c.hist, c.v_ref,
                         nullptr, c.stream, nullptr, 0);
    } else {
        launch_charges(c, c.partial, c.q, c.dq, c.stream);
        launch_potential(c, c.gamma, c.dq, c.d_R, c.sc, c.v_orb, c.v_atom, c.gdq, c.hist, c.v_ref,
                         nullptr, c.stream);
    }
    CKL();
    return TDB_OK;
}

// State and stability checks before a context steps.
tdb_status step_checks(tdb_ctx* c) {
    TRY(check_ctx(c, true, false));
    if (std::fabs(c->prm.dt) * c->spectral_width >= 0.9) {
        set_err("dt * spectral width = %.3f >= 0.9: leapfrog unstable",
                std::fabs(c->prm.dt) * c->spectral_width);
        return TDB_ERR_UNSTABLE;
    }
    return TDB_OK;
}

// Enqueue one step of c on its stream: the captured graph of its leapfrog parity, or
// the kernels themselves for an Euler step and for moving nuclei.
tdb_status step_one(tdb_ctx* c, long* launches) {
    int nl = 0;
    if (c->prm.move_nuclei) {
        TRY(enqueue_step_md(*c, c->cur, c->euler_next, &nl));
    } else if (c->euler_next) {
        TRY(enqueue_step(*c, c->cur, true, &nl));
    } else {
        TRY(ensure_graph(*c, c->cur));
        CK(cudaGraphLaunch(c->graph[c->cur], c->stream));
        nl = c->graph_launches;
    }
    *launches += nl;
    c->euler_next = false;
    c->cur ^= 1;
    c->n += 1;
    if (mixed(*c)) c->view_valid = false;
    return TDB_OK;
}

}  // namespace

extern "C" {

tdb_status tdb_step(tdb_ctx* c, long n) {
    TRY(step_checks(c));
    if (n < 0) {
        set_err("negative step count");
        return TDB_ERR_ARG;
    }
    long launches = 0;
    for (long k = 0; k < n; ++k) TRY(step_one(c, &launches));
    c->last_launches = launches;
    return TDB_OK;
}

tdb_status tdb_clone(tdb_ctx* src, void* cuda_stream, void* workspace, size_t workspace_bytes,
                     tdb_ctx** out) {
    TRY(check_ctx(src, true, false));
    if (!out) {
        set_err("NULL out");
        return TDB_ERR_ARG;
    }
    *out = nullptr;
    // the same system and parameters, from the host copies the source keeps
    tdb_system sys{};
    sys.n_atoms = src->nat;
    sys.orbs_per_atom = src->nper;
    sys.n_species = src->nspec;
    sys.species = src->species.data();
    sys.R = src->R.data();
    sys.V = src->V.data();
    sys.eps_s = src->eps_s.data();
    sys.eps_p = src->eps_p.data();
    sys.hubbard_U = src->U.data();
    sys.mass = src->mass.data();
    sys.t0 = src->mp.t0;
    sys.lam_H = src->mp.lam_H;
    sys.s0 = src->mp.s0;
    sys.lam_S = src->mp.lam_S;
    for (int k = 0; k < 4; ++k) sys.eta[k] = src->mp.eta[k];
    sys.rep_A = src->mp.rep_A;
    sys.rep_b = src->mp.rep_b;
    sys.n_electrons = src->n_electrons;
    tdb_params prm = src->prm;
    prm.cuda_stream = cuda_stream;
    TRY(tdb_create(&sys, &prm, workspace, workspace_bytes, out));
    tdb_ctx* c = *out;
    // the device state is the workspace (same layout: no device pointers inside it)
    tdb_status rc = TDB_OK;
    if (c->ws_need != src->ws_need || cudaStreamSynchronize(src->stream) != cudaSuccess ||
        cudaMemcpyAsync(c->ws, src->ws, src->ws_need, cudaMemcpyDeviceToDevice, c->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
        set_err("tdb_clone: copy of the device state failed");
        rc = TDB_ERR_CUDA;
    }
    if (rc != TDB_OK) {
        tdb_destroy(c);
        *out = nullptr;
        return rc;
    }
    // host-side state
    c->R = src->R;
    c->V = src->V;
    c->s_sinv = src->s_sinv;
    c->s_dh = src->s_dh;
    c->s_m = src->s_m;
    c->s_rho = src->s_rho;
    c->s_ref = src->s_ref;
    c->view_valid = src->view_valid;
    c->cur = src->cur;
    c->have_gs = src->have_gs;
    c->euler_next = src->euler_next;
    c->n = src->n;
    c->spectral_width = src->spectral_width;
    c->work = src->work;
    c->field = src->field;
    c->field_on = src->field_on;
    return TDB_OK;
}

tdb_status tdb_scc_shift(tdb_ctx* c, double* out, double* dq) {
    TRY(check_ctx(c, true, true));
    if (!out) {
        set_err("NULL out");
        return TDB_ERR_ARG;
    }
    if (c->prm.move_nuclei) {
        set_err("tdb_scc_shift: frozen nuclei");
        return TDB_ERR_UNSUPPORTED;
    }
    // charges and potential of the current rho_n, as tdb_observables takes them
    TRY(fp64_charges_potential(*c));
    CK(cudaMemcpyAsync(out, c->gdq, sizeof(double) * c->nat, cudaMemcpyDeviceToHost, c->stream));
    if (dq) CK(cudaMemcpyAsync(dq, c->dq, sizeof(double) * c->nat, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return TDB_OK;
}

tdb_status tdb_step_window(tdb_ctx* c, const double* v_bar, int k) {
    TRY(step_checks(c));
    if (!v_bar || k < 1) {
        set_err("tdb_step_window: need v_bar and k >= 1");
        return TDB_ERR_ARG;
    }
    if (c->prm.move_nuclei || (c->prm.precision != TDB_FP64 && c->prm.precision != TDB_FP64_SLICED)) {
        set_err("tdb_step_window: frozen nuclei and an FP64 density (FP64 or FP64_SLICED form)");
        return TDB_ERR_UNSUPPORTED;
    }
    if (c->field_on) {
        set_err("tdb_step_window: no laser field (the window freezes the Hamiltonian)");
        return TDB_ERR_UNSUPPORTED;
    }
    if (c->euler_next) {
        set_err("tdb_step_window: take one tdb_step after a ground state, kick or state load");
        return TDB_ERR_STATE;
    }
    const int N = c->N, cur = c->cur, prv = cur ^ 1;
    double* d_eig = c->obs_out + 16;
    if (!c->win_tmp) {
        int lwork = 0;
        CKS(cusolverDnDsygvd_bufferSize(c->solver, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR,
                                        CUBLAS_FILL_MODE_LOWER, N, c->Hs, N, c->M, N, d_eig, &lwork));
        c->win_lwork = std::max(lwork, 1);
        if (cudaMalloc(&c->win_work, sizeof(double) * c->win_lwork + 256) != cudaSuccess ||
            cudaMalloc(&c->win_tmp, sizeof(double) * N * N) != cudaSuccess) {
            cudaGetLastError();
            set_err("tdb_step_window: workspace allocation failed");
            return TDB_ERR_NOMEM;
        }
        c->win_info = reinterpret_cast<int*>(reinterpret_cast<char*>(c->win_work) +
                                             sizeof(double) * c->win_lwork);
    }
    // H_bar = H0 + 1/2 S (v_bar_mu + v_bar_nu), v_bar per atom repeated over its orbitals
    double* hv = reinterpret_cast<double*>(c->h_pinned + 4096);
    if (c->h_pinned_bytes < 4096 + sizeof(double) * (size_t)N) {
        set_err("tdb_step_window: staging buffer too small");
        return TDB_ERR_STATE;
    }
    CK(cudaStreamSynchronize(c->stream));
    for (int a = 0; a < c->nat; ++a)
        for (int o = 0; o < c->nper; ++o) hv[a * c->nper + o] = v_bar[a];
    CK(cudaMemcpyAsync(c->v_orb, hv, sizeof(double) * N, cudaMemcpyHostToDevice, c->stream));
    launch_build_hamiltonian(N, c->H0, c->S, c->v_orb, c->Hs, c->stream);
    CK(cudaMemcpyAsync(c->M, c->S, sizeof(double) * N * N, cudaMemcpyDeviceToDevice, c->stream));
    CKS(cusolverDnDsygvd(c->solver, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR,
                         CUBLAS_FILL_MODE_LOWER, N, c->Hs, N, c->M, N, d_eig, c->win_work,
                         c->win_lwork, c->win_info));
    {
        // the generalised eigensolve must succeed and the leapfrog's own modes need
        // |(eps_a - eps_b) dt| < 1 (beyond it the leapfrog itself is unstable)
        int* hinfo = reinterpret_cast<int*>(c->h_pinned + 192);
        CK(cudaMemcpyAsync(hinfo, c->win_info, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaMemcpyAsync(hv, d_eig, sizeof(double) * N, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        if (*hinfo != 0) {
            set_err("tdb_step_window: generalised eigensolve failed (info %d)", *hinfo);
            return TDB_ERR_CUDA;
        }
        const double spread = (hv[N - 1] - hv[0]) * std::fabs(c->prm.dt);
        if (!(spread < 1.0)) {
            set_err("tdb_step_window: (eps_max - eps_min) |dt| = %g, needs < 1", spread);
            return TDB_ERR_UNSUPPORTED;
        }
    }
    // Hs read row-major is Z = C^T (columns of C are the eigenvectors, C^T S C = 1)
    double* Z = c->Hs;
    double* Cm = c->M;          // C
    double* lev[4] = {c->rho_re[prv], c->rho_im[prv], c->rho_re[cur], c->rho_im[cur]};
    launch_transpose(N, Z, Cm, c->stream);
    if (sliced(*c)) {
        // Integer-slice products, each with P^T or C as its A operand: with T = P^T rho,
        // rho P = +-T^T and rho~ = P^T (+-T^T); with U = C rho~, rho = C (+-U^T), the sign
        // + for the symmetric real part and - for the antisymmetric imaginary part, and a
        // transposed B operand is the row slicing of the matrix itself.
        cudaStream_t st = c->stream;
        double* Tre = c->Xre;
        double* Tim = c->Xim;
        oz::slice_rows(Z, N, 1.0, c->oz[2], st);
        oz::slice_rows(c->S, N, 1.0, c->oz[1], st);
        TRY(oz_product(*c, 2, 1, Tre));                          // P^T = C^T S
        oz::slice_rows(Tre, N, 1.0, c->oz[2], st);
        auto two_sided = [&](double* re, double* im) -> tdb_status {
            oz::slice_rows(re, N, 1.0, c->oz[3], st);
            oz::slice_rows(im, N, -1.0, c->oz[4], st);
            TRY(oz_product_rho(*c, 2, Tre, Tim));
            oz::slice_rows(Tre, N, 1.0, c->oz[3], st);
            oz::slice_rows(Tim, N, -1.0, c->oz[4], st);
            return oz_product_rho(*c, 2, re, im);
        };
        for (int l = 0; l < 4; l += 2) TRY(two_sided(lev[l], lev[l + 1]));   // rho~ = P^T rho P
        learn::launch_window(N, d_eig, c->prm.dt, k, lev[0], lev[1], lev[2], lev[3], st);
        oz::slice_rows(Cm, N, 1.0, c->oz[2], st);
        for (int l = 0; l < 4; l += 2) TRY(two_sided(lev[l], lev[l + 1]));   // rho = C rho~ C^T
    } else {
        double* Pt = c->Xre;        // P^T = C^T S = Z S
        double* P = c->Xim;         // P = S C
        gemm_f64(N, N, N, Z, N, c->S, N, Pt, N, c->stream);
        launch_transpose(N, Pt, P, c->stream);
        for (double* x : lev) {   // rho~ = P^T rho P
            gemm_f64(N, N, N, Pt, N, x, N, c->win_tmp, N, c->stream);
            gemm_f64(N, N, N, c->win_tmp, N, P, N, x, N, c->stream);
        }
        learn::launch_window(N, d_eig, c->prm.dt, k, lev[0], lev[1], lev[2], lev[3], c->stream);
        for (double* x : lev) {   // rho = C rho~ C^T
            gemm_f64(N, N, N, Cm, N, x, N, c->win_tmp, N, c->stream);
            gemm_f64(N, N, N, c->win_tmp, N, Z, N, x, N, c->stream);
        }
    }
    // exactly Hermitian levels, then the Mulliken partials of the new rho_n
    for (int l : {prv, cur}) {
        launch_hermitian_half(N, c->rho_re[l], c->rho_im[l], c->Xre, c->Xim, c->stream);
        CK(cudaMemcpyAsync(c->rho_re[l], c->Xre, sizeof(double) * N * N, cudaMemcpyDeviceToDevice,
                           c->stream));
        CK(cudaMemcpyAsync(c->rho_im[l], c->Xim, sizeof(double) * N * N, cudaMemcpyDeviceToDevice,
                           c->stream));
    }
    launch_mulliken_partials(N, c->rho_re[cur], c->S, c->partial, c->stream);
    learn::launch_add_step(c->sc, k, c->stream);
    CKL();
    c->n += k;
    c->last_launches = 0;
    return TDB_OK;
}

tdb_status tdb_step_batch(tdb_ctx* const* ctxs, int count, long n) {
    if (!ctxs || count < 1 || n < 0) {
        set_err("tdb_step_batch: need count >= 1 contexts and n >= 0");
        return TDB_ERR_ARG;
    }
    for (int i = 0; i < count; ++i) {
        const tdb_status st = step_checks(ctxs[i]);
        if (st != TDB_OK) {
            set_err("tdb_step_batch: context %d: %s", i, g_err.c_str());
            return st;
        }
    }
    std::vector<long> launches(count, 0);
    // step by step across the contexts, so that their streams run side by side
    for (long k = 0; k < n; ++k)
        for (int i = 0; i < count; ++i) {
            const tdb_status st = step_one(ctxs[i], &launches[i]);
            if (st != TDB_OK) {
                set_err("tdb_step_batch: context %d, step %ld: %s", i, k, g_err.c_str());
                return st;
            }
        }
    for (int i = 0; i < count; ++i) ctxs[i]->last_launches = launches[i];
    return TDB_OK;
}

tdb_status tdb_observables(tdb_ctx* c, tdb_obs* o, double* charges, double* forces) {
    TRY(check_ctx(c, true, true));
    if (!o) {
        set_err("NULL obs");
        return TDB_ERR_ARG;
    }
    if (forces && !c->prm.move_nuclei) {
        set_err("forces are evaluated for moving nuclei (move_nuclei = 1)");
        return TDB_ERR_UNSUPPORTED;
    }
    const int cur = c->cur;
    {
        int* he = reinterpret_cast<int*>(c->h_pinned + 128);
        CK(cudaMemcpyAsync(he, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        if (*he != 0 && !c->sticky) {
            c->sticky = true;
            // codes 1-3: a bounded wait of a tensor-core product (producer, MMA, epilogue),
            // 5: the wait probe; 4: a value outside the range of its split pieces at the
            // scale of the step
            if (*he == 4) {
                set_err("a split piece overflowed its scale (device code 4)");
                return TDB_ERR_NUMERIC;
            }
            set_err("a bounded device-side wait timed out (code %d)", *he);
            return TDB_ERR_TIMEOUT;
        }
    }
    if (c->prm.move_nuclei) {
        TRY(md_forces(*c, cur, c->euler_next, 0, nullptr));
    } else {
        TRY(fp64_charges_potential(*c));
    }
    TRY(materialize(*c));
    launch_obs_reduce(c->N, c->rho_re[cur], c->rho_im[cur], c->H0, c->S, c->obs_blocks, kObsBlocks,
                      c->stream);
    launch_obs_finish(kObsBlocks, c->obs_blocks, c->obs_out, c->stream);
    launch_small_energies(*c, c->obs_out + 4, c->stream);
    CKL();
    double* red = reinterpret_cast<double*>(c->h_pinned + 256);
    DevScalars* hs = reinterpret_cast<DevScalars*>(c->h_pinned + 512);
    double* hq = reinterpret_cast<double*>(c->h_pinned + 4096);
    static_assert(sizeof(DevScalars) <= 4096 - 512, "staging layout");
    CK(cudaMemcpyAsync(red, c->obs_out, 8 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(hs, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream));
    if (charges)
        CK(cudaMemcpyAsync(hq, c->q, sizeof(double) * c->nat, cudaMemcpyDeviceToHost, c->stream));
    MdScalars hm{};
    if (c->prm.move_nuclei) {
        CK(cudaMemcpyAsync(&hm, c->md, sizeof hm, cudaMemcpyDeviceToHost, c->stream));
        if (forces)
            CK(cudaMemcpyAsync(forces, c->d_F, sizeof(double) * 3 * c->nat, cudaMemcpyDeviceToHost,
                               c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    if (charges) std::memcpy(charges, hq, sizeof(double) * c->nat);
    const DevScalars h = *hs;
    std::memset(o, 0, sizeof *o);
    o->step = (long)h.step;
    o->t = h.t_base + (double)(h.step - h.n_base) * h.dt;
    for (int k = 0; k < 3; ++k) o->dipole[k] = h.mu[k];
    o->E_band = red[0];
    o->trace_re = red[1];
    o->trace_im = red[2];
    o->herm_err = red[3];
    o->E_coul = c->prm.scc ? red[4] : 0.0;
    o->E_rep = red[5];
    o->E_kin = red[6];
    o->E_ext = h.e_ext;
    o->work = c->prm.move_nuclei ? hm.work_now : c->work;
    o->E_total = o->E_band + o->E_coul + o->E_rep + o->E_kin + o->E_ext;
    return TDB_OK;
}

tdb_status tdb_dipole_history(tdb_ctx* c, double* out, long cap, long* n_out) {
    TRY(check_ctx(c, true, true));
    if (!out || cap < 1 || !n_out) {
        set_err("invalid history request");
        return TDB_ERR_ARG;
    }
    const long long cap_h = c->prm.history_cap;
    const long long hc = cap_h + 1;   // ring slots (one more than the history length)
    const long long avail = std::min<long long>(std::max<long long>(c->n, 0), cap_h);
    const long long m = std::min<long long>(avail, cap);
    // steps n-m .. n-1 (n counted from the last ground state / set_state): at most two
    // contiguous runs of the ring
    long long k0 = (c->n - m) % hc;
    if (k0 < 0) k0 += hc;
    const long long first = std::min(m, hc - k0);
    if (first > 0)
        CK(cudaMemcpyAsync(out, c->hist + 3 * k0, sizeof(double) * 3 * first, cudaMemcpyDeviceToHost,
                           c->stream));
    if (m > first)
        CK(cudaMemcpyAsync(out + 3 * first, c->hist, sizeof(double) * 3 * (m - first),
                           cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *n_out = (long)m;
    return TDB_OK;
}

tdb_status tdb_get_rho(tdb_ctx* c, double* re, double* im, double* prev_re, double* prev_im) {
    TRY(check_ctx(c, true, true));
    TRY(materialize(*c));
    const size_t b = sizeof(double) * c->N * c->N;
    if (re) CK(cudaMemcpyAsync(re, c->rho_re[c->cur], b, cudaMemcpyDeviceToHost, c->stream));
    if (im) CK(cudaMemcpyAsync(im, c->rho_im[c->cur], b, cudaMemcpyDeviceToHost, c->stream));
    if (prev_re)
        CK(cudaMemcpyAsync(prev_re, c->rho_re[c->cur ^ 1], b, cudaMemcpyDeviceToHost, c->stream));
    if (prev_im)
        CK(cudaMemcpyAsync(prev_im, c->rho_im[c->cur ^ 1], b, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return TDB_OK;
}

// Reduced forms append their FP32-pair master (both leapfrog levels) and the scale
// bookkeeping after the FP64 views, so that a resume in the same form is bitwise.
size_t master_bytes(const tdb_ctx* c) {
    if (!mixed(*c)) return 0;
    return 8 * sizeof(float) * (size_t)c->N * c->N + sizeof(tc::DynScales);
}

size_t tdb_state_bytes(const tdb_ctx* c) {
    if (!c) return 0;
    return sizeof(StateHeader) + 4 * sizeof(double) * (size_t)c->N * c->N +
           6 * sizeof(double) * c->nat + master_bytes(c);
}

tdb_status tdb_get_state(tdb_ctx* c, void* buf, size_t bytes) {
    TRY(check_ctx(c, true, true));
    if (!buf || bytes < tdb_state_bytes(c)) {
        set_err("state buffer too small");
        return TDB_ERR_ARG;
    }
    TRY(materialize(*c));
    DevScalars h{};
    CK(cudaMemcpyAsync(&h, c->sc, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    MdScalars hm{};
    if (c->prm.move_nuclei) {
        CK(cudaMemcpyAsync(&hm, c->md, sizeof hm, cudaMemcpyDeviceToHost, c->stream));
        // positions R_n and velocities V_{n-1/2} (V_0 before the first step) live on the device
        CK(cudaMemcpyAsync(c->R.data(), c->d_R, sizeof(double) * 3 * c->nat, cudaMemcpyDeviceToHost,
                           c->stream));
        CK(cudaMemcpyAsync(c->V.data(), c->d_V, sizeof(double) * 3 * c->nat, cudaMemcpyDeviceToHost,
                           c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    StateHeader hd{kStateMagic, c->N, c->nat, h.step, h.n_base, h.t_base,
                   c->prm.move_nuclei ? hm.work : c->work, c->prm.dt, c->euler_next ? 1 : 0,
                   c->prm.precision, hm.P_prev};
    char* p = static_cast<char*>(buf);
    std::memcpy(p, &hd, sizeof hd);
    p += sizeof hd;
    const size_t b = sizeof(double) * c->N * c->N;
    const int cur = c->cur, prv = cur ^ 1;
    double* dst[4] = {reinterpret_cast<double*>(p), reinterpret_cast<double*>(p + b),
                      reinterpret_cast<double*>(p + 2 * b), reinterpret_cast<double*>(p + 3 * b)};
    CK(cudaMemcpyAsync(dst[0], c->rho_re[prv], b, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(dst[1], c->rho_im[prv], b, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(dst[2], c->rho_re[cur], b, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(dst[3], c->rho_im[cur], b, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    p += 4 * b;
    std::memcpy(p, c->R.data(), sizeof(double) * 3 * c->nat);
    std::memcpy(p + sizeof(double) * 3 * c->nat, c->V.data(), sizeof(double) * 3 * c->nat);
    p += 6 * sizeof(double) * c->nat;
    if (mixed(*c)) {
        const size_t fb = sizeof(float) * c->N * c->N;
        for (int l : {prv, cur}) {
            const MasterPtrs& m = c->ms[l];
            for (const float* src : {m.re_hi, m.re_lo, m.im_hi, m.im_lo}) {
                CK(cudaMemcpyAsync(p, src, fb, cudaMemcpyDeviceToHost, c->stream));
                p += fb;
            }
        }
        tc::DynScales d{};
        if (head3(*c)) CK(cudaMemcpyAsync(&d, c->dyn, sizeof d, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        // the maxima of the two levels are stored in (previous, current) order, like the
        // matrices, so that the blob does not depend on which buffer holds which level
        if (cur == 0) std::swap(d.max_drho[0], d.max_drho[1]);
        std::memcpy(p, &d, sizeof d);
    }
    return TDB_OK;
}

tdb_status tdb_set_state(tdb_ctx* c, const void* buf, size_t bytes) {
    TRY(check_ctx(c, false, false));
    if (!buf || bytes < tdb_state_bytes(c)) {
        set_err("state buffer too small");
        return TDB_ERR_ARG;
    }
    StateHeader hd;
    const char* p = static_cast<const char*>(buf);
    std::memcpy(&hd, p, sizeof hd);
    if (hd.magic != kStateMagic || hd.N != c->N || hd.nat != c->nat) {
        set_err("state blob does not match this context");
        return TDB_ERR_ARG;
    }
    if (!c->have_gs && mixed(*c)) {
        set_err("reduced-precision forms need tdb_ground_state before tdb_set_state");
        return TDB_ERR_STATE;
    }
    p += sizeof hd;
    const size_t b = sizeof(double) * c->N * c->N;
    const int cur = c->cur, prv = cur ^ 1;
    CK(cudaMemcpyAsync(c->rho_re[prv], p, b, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->rho_im[prv], p + b, b, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->rho_re[cur], p + 2 * b, b, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->rho_im[cur], p + 3 * b, b, cudaMemcpyHostToDevice, c->stream));
    if (c->prm.move_nuclei) {
        const char* q = p + 4 * b;
        std::memcpy(c->R.data(), q, sizeof(double) * 3 * c->nat);
        std::memcpy(c->V.data(), q + sizeof(double) * 3 * c->nat, sizeof(double) * 3 * c->nat);
        CK(cudaMemcpyAsync(c->d_R, c->R.data(), sizeof(double) * 3 * c->nat, cudaMemcpyHostToDevice,
                           c->stream));
        CK(cudaMemcpyAsync(c->d_V, c->V.data(), sizeof(double) * 3 * c->nat, cudaMemcpyHostToDevice,
                           c->stream));
        CK(cudaMemcpyAsync(c->d_Vn, c->V.data(), sizeof(double) * 3 * c->nat, cudaMemcpyHostToDevice,
                           c->stream));
        MdScalars hm{hd.work, hd.P_prev, 0.0, hd.work};
        CK(cudaMemcpyAsync(c->md, &hm, sizeof hm, cudaMemcpyHostToDevice, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        TRY(md_model(*c));
    }
    CK(cudaStreamSynchronize(c->stream));
    c->euler_next = hd.euler_next != 0;
    c->work = hd.work;
    c->have_gs = true;
    if (mixed(*c) && hd.precision == c->prm.precision) {
        // same reduced form: the master and the scales continue where they were
        const char* q = p + 4 * b + 6 * sizeof(double) * c->nat;
        const size_t fb = sizeof(float) * c->N * c->N;
        for (int l : {prv, cur}) {
            const MasterPtrs& m = c->ms[l];
            for (float* dst : {m.re_hi, m.re_lo, m.im_hi, m.im_lo}) {
                CK(cudaMemcpyAsync(dst, q, fb, cudaMemcpyHostToDevice, c->stream));
                q += fb;
            }
        }
        if (head3(*c)) {
            tc::DynScales d;
            std::memcpy(&d, q, sizeof d);
            if (cur == 0) std::swap(d.max_drho[0], d.max_drho[1]);
            CK(cudaMemcpyAsync(c->dyn, &d, sizeof d, cudaMemcpyHostToDevice, c->stream));
            CK(cudaStreamSynchronize(c->stream));
        }
        c->view_valid = true;
        TRY(upload_clock(*c, hd.n, hd.n_base, hd.t_base));
        TRY(derived_from_master(*c, true));
        CK(cudaStreamSynchronize(c->stream));
    } else {
        TRY(upload_clock(*c, hd.n, hd.n_base, hd.t_base));
        TRY(refresh_derived(*c));
        CK(cudaStreamSynchronize(c->stream));
    }
    return TDB_OK;
}

tdb_status tdb_check(tdb_ctx* c, double tol_trace) {
    TRY(check_ctx(c, true, false));
    tdb_obs o;
    TRY(tdb_observables(c, &o, nullptr, nullptr));
    const double rel = std::fabs(o.trace_re - c->n_electrons) / c->n_electrons;
    if (!std::isfinite(o.trace_re) || !std::isfinite(o.E_band) || !std::isfinite(o.dipole[0]) ||
        !std::isfinite(o.herm_err) || rel > tol_trace) {
        set_err("invariant violated: |Tr(rho S) - Ne|/Ne = %.3e (tol %.3e)", rel, tol_trace);
        c->sticky = true;
        return TDB_ERR_NUMERIC;
    }
    return TDB_OK;
}

long tdb_last_launch_count(const tdb_ctx* c) { return c ? c->last_launches : 0; }

tdb_status tdb_wait_probe(tdb_ctx* c, long long polls) {
    TRY(check_ctx(c, false, false));
    if (polls < 1) {
        set_err("tdb_wait_probe: polls must be >= 1");
        return TDB_ERR_ARG;
    }
    tc::launch_wait_probe(polls, c->d_err, c->stream);
    CKL();
    return TDB_OK;
}

tdb_status tdb_set_x_tile(tdb_ctx* c, int width) {
    TRY(check_ctx(c, false, false));
    if (!tensor(*c)) {
        set_err("tdb_set_x_tile: the form has no tensor-core products");
        return TDB_ERR_UNSUPPORTED;
    }
    if (width != 0 && width != 128 && width != 176 && width != 256) {
        set_err("tdb_set_x_tile: width must be 0, 128, 176 or 256");
        return TDB_ERR_ARG;
    }
    CK(cudaStreamSynchronize(c->stream));
    const int bn = width ? width : 0;
    tc::Maps m{};
    tc::GemmParams x{};
    const int probe = bn ? bn : default_xbn(c->N);
    if (!make_x_maps(*c, probe, m) || !tc::launchable(c->scheme, x, x_params(*c, probe, x), probe)) {
        set_err("tdb_set_x_tile: width %d cannot be used at N = %d", probe, c->N);
        return TDB_ERR_ARG;
    }
    for (int g = 0; g < 2; ++g)
        if (c->graph[g]) {
            cudaGraphExecDestroy(c->graph[g]);
            c->graph[g] = nullptr;
        }
    c->x_bn = bn;
    c->maps_x = m;
    return TDB_OK;
}

int tdb_x_tile(const tdb_ctx* c) {
    if (!c || !tensor(*c)) return -1;
    return c->x_bn;
}

tdb_status tdb_step_profiled(tdb_ctx* c, double* ms, const char** names, int cap, int* n_out) {
    TRY(check_ctx(c, true, false));
    if (!ms || !n_out || cap < 1) {
        set_err("invalid profiling buffers");
        return TDB_ERR_ARG;
    }
    if (std::fabs(c->prm.dt) * c->spectral_width >= 0.9) {
        set_err("dt * spectral width >= 0.9: leapfrog unstable");
        return TDB_ERR_UNSTABLE;
    }
    StepTimer tm;
    int nl = 0;
    if (c->prm.move_nuclei) {
        TRY(enqueue_step_md(*c, c->cur, c->euler_next, &nl, &tm));
    } else {
        TRY(enqueue_step(*c, c->cur, c->euler_next, &nl, &tm));
    }
    CK(cudaStreamSynchronize(c->stream));
    const int k = std::min<int>(cap, (int)tm.ev.size() - 1);
    for (int i = 0; i < k; ++i) {
        float f = 0.f;
        CK(cudaEventElapsedTime(&f, tm.ev[i], tm.ev[i + 1]));
        ms[i] = f;
        if (names) names[i] = tm.names[i];
    }
    *n_out = k;
    if (mixed(*c)) c->view_valid = false;
    c->euler_next = false;
    c->cur ^= 1;
    c->n += 1;
    c->last_launches = nl;
    return TDB_OK;
}

void tdb_destroy(tdb_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (auto& g : c->graph)
        if (g) cudaGraphExecDestroy(g);
    if (c->solver) cusolverDnDestroy(c->solver);
    if (c->own_ws && c->ws) cudaFree(c->ws);
    if (c->inv_work) cudaFree(c->inv_work);
    if (c->win_work) cudaFree(c->win_work);
    if (c->win_tmp) cudaFree(c->win_tmp);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    delete c;
}

const char* tdb_status_string(tdb_status s) {
    switch (s) {
        case TDB_OK: return "ok";
        case TDB_ERR_ARG: return "invalid argument";
        case TDB_ERR_STATE: return "call out of order";
        case TDB_ERR_CUDA: return "CUDA error";
        case TDB_ERR_NOT_SPD: return "overlap not positive definite";
        case TDB_ERR_SCC_NOCONV: return "SCC not converged";
        case TDB_ERR_UNSTABLE: return "time step unstable";
        case TDB_ERR_NUMERIC: return "numerical invariant violated";
        case TDB_ERR_TIMEOUT: return "device wait timed out";
        case TDB_ERR_NOMEM: return "out of device memory";
        case TDB_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char* tdb_last_error(void) { return g_err.c_str(); }

}  // extern "C"

// ---------------------------------------------------------------------------
// Grouped batches: many independent contexts of one tensor-core form advanced together,
// every phase of a step one launch over all of them (the probe runs of a pump-probe scan,
// Sec. 3.2, are independent trajectories of uneven size).
// ---------------------------------------------------------------------------

struct tdb_batch {
    std::vector<tdb_ctx*> ctxs;
    std::vector<int> off;              // parity of each context against ctxs[0]
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    int scheme = 0, x_bn = 128, schedule = 0;
    float tuned_ms = 0.f;
    char* dmem = nullptr;              // argument arrays and work lists (one allocation)
    tc::SplitDhArgs* d_split[2] = {};
    tc::GroupedGemm* d_dm[2] = {};
    tc::GroupedGemm* d_x[2] = {};
    UpdateDfArgs* d_upd[2] = {};
    LevelFinalArgs* d_fin[2] = {};
    int2 *w_split = nullptr, *w_dm = nullptr, *w_x = nullptr, *w_upd = nullptr, *w_ldq = nullptr,
         *w_fin = nullptr;
    int n_split = 0, n_dm = 0, n_x = 0, n_upd = 0, n_ldq = 0, n_fin = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
};

namespace {

int cdiv(int a, int b) { return (a + b - 1) / b; }

// Work list of a grouped launch: every block of every problem, problem by problem in the
// schedule's order (0: as given; 1: largest N first).
std::vector<int2> work_list(const tdb_batch& b, const std::vector<int>& blocks, int schedule) {
    std::vector<int> order(b.ctxs.size());
    for (size_t p = 0; p < order.size(); ++p) order[p] = (int)p;
    if (schedule == 1)
        std::stable_sort(order.begin(), order.end(),
                         [&](int x, int y) { return b.ctxs[x]->N > b.ctxs[y]->N; });
    std::vector<int2> w;
    for (int p : order)
        for (int k = 0; k < blocks[p]; ++k) w.push_back(make_int2(p, k));
    return w;
}

tc::GroupedGemm grouped(const tc::Maps& m, const tc::GemmParams& p, int N, int bn, int nparts) {
    tc::GroupedGemm g{};
    g.maps = m;
    g.p = p;
    g.tiles_x = cdiv(N, bn);
    g.tiles_y = cdiv(N, 128);
    g.nparts = nparts;
    return g;
}

// Argument arrays of both parities and the work lists for X tile width bn and a schedule,
// uploaded into b.dmem (allocated here).
tdb_status batch_layout(tdb_batch& b, int bn, int schedule) {
    const int P = (int)b.ctxs.size();
    std::vector<tc::SplitDhArgs> split[2];
    std::vector<tc::GroupedGemm> dm[2], xg[2];
    std::vector<UpdateDfArgs> upd[2];
    std::vector<LevelFinalArgs> fin[2];
    std::vector<int> nb_split(P), nb_dm(P), nb_x(P), nb_upd(P), nb_ldq(P), nb_fin(P);
    for (int g = 0; g < 2; ++g)
        for (int p = 0; p < P; ++p) {
            Ctx& c = *b.ctxs[p];
            const TensorStep ts = tensor_step_args(c, g ^ b.off[p], false, bn);
            tc::Maps mx{};
            if (!make_x_maps(c, bn, mx)) {
                set_err("grouped batch: cuTensorMapEncodeTiled failed");
                return TDB_ERR_CUDA;
            }
            split[g].push_back(ts.split);
            dm[g].push_back(grouped(c.maps_dm, ts.dm, c.N, 64, 1));
            xg[g].push_back(grouped(mx, ts.x, c.N, bn, ts.x_parts));
            upd[g].push_back(ts.upd);
            LevelFinalArgs f{};
            f.lv = ts.upd.lv;
            f.slot = ts.upd.out_slot;
            fin[g].push_back(f);
            nb_ldq[p] = level_blocks(c.nat);
            nb_fin[p] = level_blocks(c.nat) + 1;
            nb_split[p] = tc::split_dham_blocks(c.N);
            nb_dm[p] = dm[g].back().tiles_x * dm[g].back().tiles_y;
            nb_x[p] = xg[g].back().tiles_x * xg[g].back().tiles_y * ts.x_parts;
            nb_upd[p] = c.nct * (c.nct + 1) / 2;
        }
    const std::vector<int2> ws = work_list(b, nb_split, schedule), wd = work_list(b, nb_dm, schedule),
                            wx = work_list(b, nb_x, schedule), wu = work_list(b, nb_upd, schedule),
                            wq = work_list(b, nb_ldq, schedule), wf = work_list(b, nb_fin, schedule);
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t s_split = up(sizeof(tc::SplitDhArgs) * P), s_gg = up(sizeof(tc::GroupedGemm) * P),
                 s_upd = up(sizeof(UpdateDfArgs) * P), s_fin = up(sizeof(LevelFinalArgs) * P);
    const size_t total = 2 * (s_split + 2 * s_gg + s_upd + s_fin) +
                         up(sizeof(int2) * ws.size()) + up(sizeof(int2) * wd.size()) +
                         up(sizeof(int2) * wx.size()) + up(sizeof(int2) * wu.size()) +
                         up(sizeof(int2) * wq.size()) + up(sizeof(int2) * wf.size());
    if (b.dmem) {
        CK(cudaStreamSynchronize(b.stream));
        cudaFree(b.dmem);
        b.dmem = nullptr;
    }
    if (cudaMalloc(&b.dmem, total) != cudaSuccess) {
        cudaGetLastError();
        set_err("grouped batch: device allocation of %zu bytes failed", total);
        return TDB_ERR_NOMEM;
    }
    std::vector<char> h(total);
    size_t o = 0;
    auto put = [&](const void* src, size_t n, size_t span) {
        std::memcpy(h.data() + o, src, n);
        char* d = b.dmem + o;
        o += span;
        return d;
    };
    for (int g = 0; g < 2; ++g) {
        b.d_split[g] = reinterpret_cast<tc::SplitDhArgs*>(put(split[g].data(), sizeof(tc::SplitDhArgs) * P, s_split));
        b.d_dm[g] = reinterpret_cast<tc::GroupedGemm*>(put(dm[g].data(), sizeof(tc::GroupedGemm) * P, s_gg));
        b.d_x[g] = reinterpret_cast<tc::GroupedGemm*>(put(xg[g].data(), sizeof(tc::GroupedGemm) * P, s_gg));
        b.d_upd[g] = reinterpret_cast<UpdateDfArgs*>(put(upd[g].data(), sizeof(UpdateDfArgs) * P, s_upd));
        b.d_fin[g] = reinterpret_cast<LevelFinalArgs*>(put(fin[g].data(), sizeof(LevelFinalArgs) * P, s_fin));
    }
    b.w_split = reinterpret_cast<int2*>(put(ws.data(), sizeof(int2) * ws.size(), up(sizeof(int2) * ws.size())));
    b.w_dm = reinterpret_cast<int2*>(put(wd.data(), sizeof(int2) * wd.size(), up(sizeof(int2) * wd.size())));
    b.w_x = reinterpret_cast<int2*>(put(wx.data(), sizeof(int2) * wx.size(), up(sizeof(int2) * wx.size())));
    b.w_upd = reinterpret_cast<int2*>(put(wu.data(), sizeof(int2) * wu.size(), up(sizeof(int2) * wu.size())));
    b.w_ldq = reinterpret_cast<int2*>(put(wq.data(), sizeof(int2) * wq.size(), up(sizeof(int2) * wq.size())));
    b.w_fin = reinterpret_cast<int2*>(put(wf.data(), sizeof(int2) * wf.size(), up(sizeof(int2) * wf.size())));
    b.n_ldq = (int)wq.size();
    b.n_fin = (int)wf.size();
    b.n_split = (int)ws.size();
    b.n_dm = (int)wd.size();
    b.n_x = (int)wx.size();
    b.n_upd = (int)wu.size();
    CK(cudaMemcpyAsync(b.dmem, h.data(), total, cudaMemcpyHostToDevice, b.stream));
    CK(cudaStreamSynchronize(b.stream));
    b.x_bn = bn;
    b.schedule = schedule;
    return TDB_OK;
}

// One grouped step of global parity g: six launches over all contexts.
tdb_status batch_enqueue(tdb_batch& b, int g) {
    tc::launch_split_dham_grouped(b.scheme, b.d_split[g], b.w_split, b.n_split, b.stream);
    CK(tc::launch_grouped(b.scheme, b.d_dm[g], b.w_dm, b.n_dm, b.stream, 64));
    CK(tc::launch_grouped(b.scheme, b.d_x[g], b.w_x, b.n_x, b.stream, b.x_bn));
    launch_update_df_grouped(b.d_upd[g], b.w_upd, b.n_upd, b.stream);
    launch_level_dq_grouped(b.d_fin[g], b.w_ldq, b.n_ldq, b.stream);
    launch_level_final_grouped(b.d_fin[g], b.w_fin, b.n_fin, b.stream);
    CKL();
    return TDB_OK;
}

void batch_free_graphs(tdb_batch& b) {
    for (auto& gr : b.graph)
        if (gr) {
            cudaGraphExecDestroy(gr);
            gr = nullptr;
        }
}

// Autotuner of the grouped X product: every (tile width, schedule) pair times three
// launches on the contexts' current operands; the fastest is kept.  Every output element
// keeps its K order whatever the width and order, so the choice changes the time only.
// The timing launches accumulate X maxima, which are reset afterwards (as after tune_x).
tdb_status batch_tune(tdb_batch& b) {
    static const int cand[] = {128, 176, 256};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 0.f;
    int best_bn = 0, best_s = 0;
    tdb_status st = TDB_OK;
    for (int bn : cand) {
        bool valid = true;
        for (tdb_ctx* c : b.ctxs) {
            tc::Maps m{};
            valid = valid && make_x_maps(*c, bn, m);   // width not encodable for this size
        }
        if (!valid) continue;
        for (int sched = 0; sched < 2; ++sched) {
            st = batch_layout(b, bn, sched);
            if (st != TDB_OK) break;
            cudaError_t e = tc::launch_grouped(b.scheme, b.d_x[0], b.w_x, b.n_x, b.stream, bn);
            if (e == cudaSuccess) e = cudaEventRecord(e0, b.stream);
            for (int r = 0; r < 3 && e == cudaSuccess; ++r)
                e = tc::launch_grouped(b.scheme, b.d_x[0], b.w_x, b.n_x, b.stream, bn);
            if (e == cudaSuccess) e = cudaEventRecord(e1, b.stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                set_err("grouped batch tuning: %s", cudaGetErrorString(e));
                st = TDB_ERR_CUDA;
                break;
            }
            if (!best_bn || ms < best) {
                best = ms;
                best_bn = bn;
                best_s = sched;
            }
        }
        if (st != TDB_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != TDB_OK) return st;
    for (tdb_ctx* c : b.ctxs)
        if (c->dyn) CK(cudaMemsetAsync(c->dyn->max_x, 0, sizeof(c->dyn->max_x), b.stream));
    b.tuned_ms = best / 3.f;
    return batch_layout(b, best_bn ? best_bn : 128, best_s);
}

tdb_status batch_capture(tdb_batch& b) {
    batch_free_graphs(b);
    for (int g = 0; g < 2; ++g) {
        cudaGraph_t gr = nullptr;
        CK(cudaStreamBeginCapture(b.stream, cudaStreamCaptureModeThreadLocal));
        const tdb_status st = batch_enqueue(b, g);
        const cudaError_t e = cudaStreamEndCapture(b.stream, &gr);
        if (st != TDB_OK || e != cudaSuccess) {
            if (gr) cudaGraphDestroy(gr);
            if (st == TDB_OK) set_err("grouped batch: graph capture failed: %s", cudaGetErrorString(e));
            return st != TDB_OK ? st : TDB_ERR_CUDA;
        }
        const cudaError_t ei = cudaGraphInstantiate(&b.graph[g], gr, 0);
        cudaGraphDestroy(gr);
        if (ei != cudaSuccess) {
            set_err("grouped batch: graph instantiate failed: %s", cudaGetErrorString(ei));
            return TDB_ERR_CUDA;
        }
    }
    return TDB_OK;
}

}  // namespace

extern "C" {

void tdb_batch_destroy(tdb_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_free_graphs(*b);
    if (b->dmem) cudaFree(b->dmem);
    if (b->ev) cudaEventDestroy(b->ev);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

tdb_status tdb_batch_create(tdb_ctx* const* ctxs, int count, tdb_batch** out) {
    if (!ctxs || count < 1 || !out) {
        set_err("tdb_batch_create: need count >= 1 contexts and an output pointer");
        return TDB_ERR_ARG;
    }
    *out = nullptr;
    for (int i = 0; i < count; ++i) {
        TRY(step_checks(ctxs[i]));
        tdb_ctx* c = ctxs[i];
        if (!tensor(*c) || c->prm.move_nuclei) {
            set_err("tdb_batch_create: context %d is not a frozen-nuclei tensor-core form", i);
            return TDB_ERR_UNSUPPORTED;
        }
        if (c->prm.precision != ctxs[0]->prm.precision || c->prm.dt != ctxs[0]->prm.dt) {
            set_err("tdb_batch_create: context %d differs in form or time step from context 0", i);
            return TDB_ERR_ARG;
        }
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == c) {
                set_err("tdb_batch_create: context %d appears twice", i);
                return TDB_ERR_ARG;
            }
    }
    tdb_batch* b = new tdb_batch;
    b->ctxs.assign(ctxs, ctxs + count);
    b->scheme = ctxs[0]->scheme;
    tdb_status st = TDB_OK;
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        set_err("tdb_batch_create: stream or event creation failed");
        st = TDB_ERR_CUDA;
    }
    if (st == TDB_OK && tc::prepare() != cudaSuccess) {
        cudaGetLastError();
        set_err("tdb_batch_create: kernel attributes");
        st = TDB_ERR_CUDA;
    }
    for (int i = 0; i < count && st == TDB_OK; ++i) {
        if (cudaStreamSynchronize(ctxs[i]->stream) != cudaSuccess) st = TDB_ERR_CUDA;
        b->off.push_back(ctxs[i]->cur ^ ctxs[0]->cur);
    }
    if (st == TDB_OK) st = batch_tune(*b);
    if (st == TDB_OK) st = batch_capture(*b);
    if (st != TDB_OK) {
        tdb_batch_destroy(b);
        return st;
    }
    *out = b;
    return TDB_OK;
}

tdb_status tdb_batch_tuning(const tdb_batch* b, int* x_bn, int* schedule, double* x_ms) {
    if (!b) {
        set_err("NULL batch");
        return TDB_ERR_ARG;
    }
    if (x_bn) *x_bn = b->x_bn;
    if (schedule) *schedule = b->schedule;
    if (x_ms) *x_ms = b->tuned_ms;
    return TDB_OK;
}

tdb_status tdb_batch_step(tdb_batch* b, long n) {
    if (!b || n < 0) {
        set_err("tdb_batch_step: NULL batch or n < 0");
        return TDB_ERR_ARG;
    }
    const int P = (int)b->ctxs.size();
    for (int i = 0; i < P; ++i) {
        TRY(step_checks(b->ctxs[i]));
        if ((b->ctxs[i]->cur ^ b->ctxs[0]->cur) != b->off[i]) {
            set_err("tdb_batch_step: context %d was stepped on its own since the batch was made", i);
            return TDB_ERR_STATE;
        }
    }
    long k = 0;
    // an Euler step (after a kick, ground state or state load) is taken context by context
    bool euler = false;
    for (tdb_ctx* c : b->ctxs) euler = euler || c->euler_next;
    if (euler && n > 0) {
        for (int i = 0; i < P; ++i) {
            long l = 0;
            TRY(step_one(b->ctxs[i], &l));
            b->ctxs[i]->last_launches = l;
        }
        k = 1;
    }
    if (k >= n) return TDB_OK;
    // the batch stream follows every context's stream, and they follow it
    for (tdb_ctx* c : b->ctxs) {
        CK(cudaEventRecord(b->ev, c->stream));
        CK(cudaStreamWaitEvent(b->stream, b->ev, 0));
    }
    for (; k < n; ++k) {
        CK(cudaGraphLaunch(b->graph[b->ctxs[0]->cur], b->stream));
        for (tdb_ctx* c : b->ctxs) {
            c->cur ^= 1;
            c->n += 1;
            c->view_valid = false;
            c->last_launches = 6;
        }
    }
    CK(cudaEventRecord(b->ev, b->stream));
    for (tdb_ctx* c : b->ctxs) CK(cudaStreamWaitEvent(c->stream, b->ev, 0));
    return TDB_OK;
}

}  // extern "C"
