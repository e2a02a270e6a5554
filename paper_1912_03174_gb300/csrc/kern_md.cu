// Moving nuclei (Ehrenfest dynamics): forces (eq:forces), the non-adiabatic
// coupling matrix D (eq:nac, eq:onsite), the work rate P and velocity Verlet
// (Sec. 2.3).  FP64 throughout.  Gradients of the two-centre blocks are
// recomputed from the geometry where they are used and never stored.
#include <cmath>

#include "tdb_internal.h"

namespace tdb {

namespace {

__device__ __forceinline__ double warp_sum_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Radial integrals and their r-derivatives (hopping if h, else overlap).
__device__ __forceinline__ void radial(const ModelParams& mp, double r, bool h, double K[4],
                                       double dK[4]) {
    const double e = h ? exp(-r / mp.lam_H) : exp(-r / mp.lam_S);
    const double lam = h ? mp.lam_H : mp.lam_S;
    for (int k = 0; k < 4; ++k) {
        K[k] = h ? mp.eta[k] * mp.t0 * e : -mp.eta[k] * mp.s0 * e;
        dK[k] = -K[k] / lam;
    }
}

// Gradient with respect to d = R_B - R_A of element (i, j) of the Slater-Koster
// s/p block (ss = K0, s-a = c_a K1, a-s = -c_a K1, a-b = c_a c_b (K2 - K3) + d_ab K3),
// using dr/dd_g = c_g and dc_a/dd_g = (d_ag - c_a c_g) / r.
__device__ __forceinline__ void block_grad(int i, int j, const double c[3], double r,
                                           const double K[4], const double dK[4], double g[3]) {
    if (i == 0 && j == 0) {
        for (int q = 0; q < 3; ++q) g[q] = dK[0] * c[q];
    } else if (i == 0 || j == 0) {
        const int a = (i == 0 ? j : i) - 1;
        const double sg = i == 0 ? 1.0 : -1.0;
        for (int q = 0; q < 3; ++q)
            g[q] = sg * (((a == q ? 1.0 : 0.0) - c[a] * c[q]) / r * K[1] + c[a] * dK[1] * c[q]);
    } else {
        const int a = i - 1, b = j - 1;
        const double dd = K[2] - K[3], ddk = dK[2] - dK[3];
        for (int q = 0; q < 3; ++q) {
            const double dca = ((a == q ? 1.0 : 0.0) - c[a] * c[q]) / r;
            const double dcb = ((b == q ? 1.0 : 0.0) - c[b] * c[q]) / r;
            g[q] = (dca * c[b] + c[a] * dcb) * dd + c[a] * c[b] * ddk * c[q] +
                   (a == b ? dK[3] * c[q] : 0.0);
        }
    }
}

// d gamma_AB / dR for exponents ta, tb (tau = 16 U / 5): derivative of
// 1/R - zeta(R), with the equal-exponent form below a 3e-4 relative gap.
__device__ double gamma_dR(double ta, double tb, double R) {
    const double tmax = ta > tb ? ta : tb;
    double dz;
    if (fabs(ta - tb) < 3e-4 * tmax) {
        const double t = 0.5 * (ta + tb);
        const double e = exp(-t * R);
        const double poly = 1.0 / R + 11.0 * t / 16.0 + 3.0 * t * t * R / 16.0 + t * t * t * R * R / 48.0;
        const double dpoly = -1.0 / (R * R) + 3.0 * t * t / 16.0 + t * t * t * R / 24.0;
        dz = e * (dpoly - t * poly);
    } else {
        dz = 0.0;
        for (int s = 0; s < 2; ++s) {
            const double a = s ? tb : ta, b = s ? ta : tb;
            const double a2 = a * a, b2 = b * b, d = a2 - b2;
            const double c1 = b2 * b2 * a / (2.0 * d * d);
            const double c2 = (b2 * b2 * b2 - 3.0 * a2 * b2 * b2) / (d * d * d);
            dz += exp(-a * R) * (-a * (c1 - c2 / R) + c2 / (R * R));
        }
    }
    return -1.0 / (R * R) - dz;
}

// Gradient with respect to d = R_B - R_A of the weighted block sum sum_ij w_ij T_ij(d) of a
// two-centre s/p block (T_00 = K0, T_0a = c_a K1, T_a0 = -c_a K1, T_ab = c_a c_b (K2 - K3)
// + delta_ab K3, c = d / r), contracted before differentiating: with p_a = w_0a - w_a0 and
// M_ab = w_ab the sum is w_00 K0 + (p.c) K1 + (c.Mc) (K2 - K3) + tr(M) K3, and with
// dc_a/dd_q = (delta_aq - c_a c_q) / r and dr/dd = c its gradient is
//   c [w_00 K0' + (p.c) K1' + (c.Mc)(K2' - K3') + tr(M) K3' - ((p.c) K1 + 2 (c.Mc)(K2 - K3)) / r]
//   + [p K1 + (M + M^T) c (K2 - K3)] / r.
// nper = 1 (s only): w_00 K0' c.
__device__ __forceinline__ void block_sum_grad(int nper, const double (&w)[16], const double c[3],
                                               double r, const double K[4], const double dK[4],
                                               double g[3]) {
    if (nper == 1) {
        for (int q = 0; q < 3; ++q) g[q] = w[0] * dK[0] * c[q];
        return;
    }
    const double p[3] = {w[1] - w[4], w[2] - w[8], w[3] - w[12]};
    double Mc[3], MTc[3];
    for (int a = 0; a < 3; ++a) {
        Mc[a] = w[4 * (a + 1) + 1] * c[0] + w[4 * (a + 1) + 2] * c[1] + w[4 * (a + 1) + 3] * c[2];
        MTc[a] = w[4 + a + 1] * c[0] + w[8 + a + 1] * c[1] + w[12 + a + 1] * c[2];
    }
    const double pc = p[0] * c[0] + p[1] * c[1] + p[2] * c[2];
    const double cMc = c[0] * Mc[0] + c[1] * Mc[1] + c[2] * Mc[2];
    const double tr = w[5] + w[10] + w[15];
    const double d23 = K[2] - K[3];
    const double inv_r = 1.0 / r;
    const double par = w[0] * dK[0] + pc * dK[1] + cMc * (dK[2] - dK[3]) + tr * dK[3] -
                       (pc * K[1] + 2.0 * cMc * d23) * inv_r;
    for (int q = 0; q < 3; ++q)
        g[q] = par * c[q] + (p[q] * K[1] + (Mc[q] + MTc[q]) * d23) * inv_r;
}

// One block per atom A, its threads over the partners B: F_A = sum over B != A of the pair
// terms of eq:forces (energy-weighted form of the S-derivative terms, velocity terms
// dropped):
//   sum over the (A, B) block of 2 Re rho_ij dH_ij/dR_B + (Re rho_ij (v_A + v_B) - 2 Re W_ij)
//   dS_ij/dR_B, plus -dq_A dq_B dgamma/dR_A + rep_A/rep_b e^{-r/rep_b} u, and -dq_A E(t);
// W = 1/2 (X + X^dagger), X = S^-1 H rho.  The block sums are differentiated in contracted
// form (block_sum_grad); FP64.
__global__ void __launch_bounds__(128)
    k_forces(int nat, int nper, int scc, const double* __restrict__ R,
             const double* __restrict__ rre, const double* __restrict__ wre,
             const double* __restrict__ v_atom, const double* __restrict__ dq,
             const double* __restrict__ U, ModelParams mp, const DevScalars* __restrict__ sc,
             double* __restrict__ F) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int A = blockIdx.x;
    const int N = nat * nper;
    const double RA[3] = {R[3 * A], R[3 * A + 1], R[3 * A + 2]};
    const double vA = v_atom[A], dqA = dq[A], tA = 3.2 * U[A];
    double f[3] = {0.0, 0.0, 0.0};
    for (int B = threadIdx.x; B < nat; B += blockDim.x) {
        if (B == A) continue;
        const double d[3] = {R[3 * B] - RA[0], R[3 * B + 1] - RA[1], R[3 * B + 2] - RA[2]};
        const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        const double inv_r = 1.0 / r;
        const double c[3] = {d[0] * inv_r, d[1] * inv_r, d[2] * inv_r};
        const double eh = exp(-r / mp.lam_H), es = exp(-r / mp.lam_S);
        double KH[4], dKH[4], KS[4], dKS[4];
        for (int k = 0; k < 4; ++k) {
            KH[k] = mp.eta[k] * mp.t0 * eh;
            dKH[k] = -KH[k] / mp.lam_H;
            KS[k] = -mp.eta[k] * mp.s0 * es;
            dKS[k] = -KS[k] / mp.lam_S;
        }
        const double vv = vA + v_atom[B];
        double wh[16], ws[16];
        for (int i = 0; i < nper; ++i) {
            const size_t row = (size_t)(A * nper + i) * N + (size_t)B * nper;
            for (int j = 0; j < nper; ++j) {
                const double pr = rre[row + j], w = wre[row + j];
                wh[4 * i + j] = 2.0 * pr;
                ws[4 * i + j] = pr * vv - 2.0 * w;
            }
        }
        double gh[3], gs[3];
        block_sum_grad(nper, wh, c, r, KH, dKH, gh);
        block_sum_grad(nper, ws, c, r, KS, dKS, gs);
        for (int q = 0; q < 3; ++q) f[q] += gh[q] + gs[q];
        // u = (R_A - R_B) / r = -c
        if (scc) {
            const double g = gamma_dR(tA, 3.2 * U[B], r);
            const double s = dqA * dq[B] * g;
            for (int q = 0; q < 3; ++q) f[q] += s * c[q];
        }
        if (mp.rep_A != 0.0) {
            const double e = mp.rep_A / mp.rep_b * exp(-r / mp.rep_b);
            for (int q = 0; q < 3; ++q) f[q] -= e * c[q];
        }
    }
    for (int q = 0; q < 3; ++q) f[q] = warp_sum_d(f[q]);
    __shared__ double red[3][4];
    if (lane == 0)
        for (int q = 0; q < 3; ++q) red[q][warp] = f[q];
    __syncthreads();
    if (threadIdx.x < 3) {
        const int q = threadIdx.x;
        F[3 * A + q] = ((red[q][0] + red[q][1]) + (red[q][2] + red[q][3])) - dqA * sc->E[q];
    }
}

// Re W = 1/2 (Re X + Re X^T) through a shared-memory tile transpose.
__global__ void k_wre(int N, const double* __restrict__ xre, double* __restrict__ wre) {
    __shared__ double t[kTile][kTile + 1];
    const int bx = blockIdx.x * kTile, by = blockIdx.y * kTile;
    for (int y = threadIdx.y; y < kTile; y += blockDim.y) {
        const int r = bx + y, c = by + threadIdx.x;   // transposed tile
        t[y][threadIdx.x] = (r < N && c < N) ? xre[(size_t)r * N + c] : 0.0;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < kTile; y += blockDim.y) {
        const int r = by + y, c = bx + threadIdx.x;
        if (r < N && c < N) wre[(size_t)r * N + c] = 0.5 * (xre[(size_t)r * N + c] + t[threadIdx.x][y]);
    }
}

// D_mu_nu = Rdot_B . grad_B S_mu_nu for mu in A, nu in B != A; on-site blocks 0.
__global__ void k_build_nac(int nat, int nper, const double* __restrict__ R,
                            const double* __restrict__ V, ModelParams mp, double* __restrict__ D) {
    const int B = blockIdx.x * blockDim.x + threadIdx.x;
    const int A = blockIdx.y * blockDim.y + threadIdx.y;
    if (A >= nat || B >= nat) return;
    const int N = nat * nper;
    if (A == B) {
        for (int i = 0; i < nper; ++i)
            for (int j = 0; j < nper; ++j) D[(size_t)(A * nper + i) * N + B * nper + j] = 0.0;
        return;
    }
    const double d[3] = {R[3 * B] - R[3 * A], R[3 * B + 1] - R[3 * A + 1], R[3 * B + 2] - R[3 * A + 2]};
    const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    const double c[3] = {d[0] / r, d[1] / r, d[2] / r};
    double KS[4], dKS[4];
    radial(mp, r, false, KS, dKS);
    for (int i = 0; i < nper; ++i)
        for (int j = 0; j < nper; ++j) {
            double g[3];
            block_grad(i, j, c, r, KS, dKS, g);
            D[(size_t)(A * nper + i) * N + B * nper + j] =
                V[3 * B] * g[0] + V[3 * B + 1] * g[1] + V[3 * B + 2] * g[2];
        }
}

// Per block: sum_ij Re X_ij (D_ji - D_ij)  (P = Re Tr[S^-1 H rho (D - D^T)]).
__global__ void k_power(int N, const double* __restrict__ xre, const double* __restrict__ D,
                        double* __restrict__ out) {
    double s = 0.0;
    const size_t NN = (size_t)N * N;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < NN;
         i += (size_t)gridDim.x * blockDim.x) {
        const size_t r = i / N, c = i % N;
        s += xre[i] * (D[c * N + r] - D[i]);
    }
    __shared__ double red[32];
    s = warp_sum_d(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
        out[blockIdx.x] = t;
    }
}

// Sum the block partials into P_n; work_n = work_{n-1} + dt/2 (P_n + P_{n-1}) (none at
// the first step).  commit = 0: only report (observables of the current state).
__global__ void k_power_finish(int nb, const double* __restrict__ part, MdScalars* __restrict__ md,
                               double dt, int first, int commit) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double p = 0.0;
    for (int k = 0; k < nb; ++k) p += part[k];
    const double w = first ? md->work : md->work + 0.5 * dt * (p + md->P_prev);
    md->P_now = p;
    md->work_now = w;
    if (commit) {
        md->work = w;
        md->P_prev = p;
    }
}

// V_n = V_{n-1/2} + F_n dt / 2m (V_0 itself at the first step), into Vn.
__global__ void k_vel_n(int nat, const double* __restrict__ Vh, const double* __restrict__ F,
                        const double* __restrict__ mass, double dt, int first,
                        double* __restrict__ Vn) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * nat) return;
    const double m = mass[i / 3] * 1822.888486;
    Vn[i] = first ? Vh[i] : Vh[i] + F[i] * dt / (2.0 * m);
}

// V_{n+1/2} = V_n + F_n dt / 2m;  R_{n+1} = R_n + dt V_{n+1/2}.
__global__ void k_vv(int nat, const double* __restrict__ Vn, const double* __restrict__ F,
                     const double* __restrict__ mass, double dt, double* __restrict__ Vh,
                     double* __restrict__ R) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * nat) return;
    const double m = mass[i / 3] * 1822.888486;
    const double vh = Vn[i] + F[i] * dt / (2.0 * m);
    Vh[i] = vh;
    R[i] += dt * vh;
}

}  // namespace

void launch_forces(const Ctx& c, const double* rre, const double* wre, double* F, cudaStream_t st) {
    k_forces<<<c.nat, 128, 0, st>>>(c.nat, c.nper, c.prm.scc, c.d_R, rre, wre, c.v_atom, c.dq,
                                    c.d_U, c.mp, c.sc, F);
}

void launch_wre(int N, const double* xre, double* wre, cudaStream_t st) {
    dim3 b(kTile, 8), g((N + kTile - 1) / kTile, (N + kTile - 1) / kTile);
    k_wre<<<g, b, 0, st>>>(N, xre, wre);
}

void launch_build_nac(const Ctx& c, const double* V, double* D, cudaStream_t st) {
    dim3 b(32, 8), g((c.nat + 31) / 32, (c.nat + 7) / 8);
    k_build_nac<<<g, b, 0, st>>>(c.nat, c.nper, c.d_R, V, c.mp, D);
}

void launch_power(const Ctx& c, const double* xre, const double* D, double* part, int nb,
                  int first, int commit, cudaStream_t st) {
    k_power<<<nb, 256, 0, st>>>(c.N, xre, D, part);
    k_power_finish<<<1, 32, 0, st>>>(nb, part, c.md, c.prm.dt, first, commit);
}

void launch_vel_n(const Ctx& c, const double* F, int first, cudaStream_t st) {
    k_vel_n<<<(3 * c.nat + 255) / 256, 256, 0, st>>>(c.nat, c.d_V, F, c.d_mass, c.prm.dt, first,
                                                      c.d_Vn);
}

void launch_vv(const Ctx& c, const double* F, cudaStream_t st) {
    k_vv<<<(3 * c.nat + 255) / 256, 256, 0, st>>>(c.nat, c.d_Vn, F, c.d_mass, c.prm.dt, c.d_V,
                                                   c.d_R);
}

}  // namespace tdb
