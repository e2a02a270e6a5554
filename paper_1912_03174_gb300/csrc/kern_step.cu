// O(N^2) kernels of the propagation step and of the setup: model build
// (S, H0, gamma), Mulliken charges, SCC potential, leapfrog update, kick
// helpers and observable reductions.  All arithmetic is FP64.
#include <cmath>

#include <cuda_fp16.h>

#include "pdl.cuh"
#include "tdb_internal.h"

namespace tdb {

namespace {

// E(t) of eq:pumpf: E0 sin(omega t + phase) f(t) dir.
__device__ void field_at(const FieldDev& f, double t, double E[3]) {
    if (!f.on) {
        E[0] = E[1] = E[2] = 0.0;
        return;
    }
    double env = 1.0;
    if (f.envelope == 1) {
        const double x = t - f.t_center;
        env = exp(-x * x * 4.0 * 0.69314718055994530942 / (f.fwhm * f.fwhm));
    } else if (f.envelope == 2) {
        if (t >= 0.0 && t <= f.fwhm) {
            const double s = sin(3.14159265358979323846 * t / f.fwhm);
            env = s * s;
        } else {
            env = 0.0;
        }
    }
    const double a = f.E0 * sin(f.omega * t + f.phase) * env;
    E[0] = a * f.dir[0];
    E[1] = a * f.dir[1];
    E[2] = a * f.dir[2];
}

__device__ __forceinline__ uint16_t to16(float x, int bf16) {
    if (bf16) return __bfloat16_as_ushort(__float2bfloat16_rn(x));
    return __half_as_ushort(__float2half_rn(x));
}
__device__ __forceinline__ float from16(uint16_t x, int bf16) {
    if (bf16) return __bfloat162float(__ushort_as_bfloat16(x));
    return __half2float(__ushort_as_half(x));
}

// head (integer, |h| <= 127) + two FP16 tails of a scaled FP32 value (exact split)
__device__ __forceinline__ void split_head3(float x, uint16_t (&q)[3]) {
    const float h = fminf(fmaxf(rintf(x), -127.f), 127.f);
    const float r = x - h;
    const __half rh = __float2half_rn(r);
    q[0] = __half_as_ushort(__float2half_rn(h));
    q[1] = __half_as_ushort(rh);
    q[2] = __half_as_ushort(__float2half_rn(r - __half2float(rh)));
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One thread per (A, B) atom pair writes the nper x nper blocks of S and H0.
// Off-site: Slater-Koster s/p table with direction cosines c of R_B - R_A:
//   ss = K0, s-a = c_a K1, a-s = -c_a K1, a-b = c_a c_b (K2 - K3) + delta_ab K3,
// with hopping K = eta t0 exp(-r/lam_H) and overlap K = -eta s0 exp(-r/lam_S).
__global__ void k_build_model(int nat, int nper, const double* __restrict__ R,
                              const double* __restrict__ onsite, ModelParams mp,
                              double* __restrict__ S, double* __restrict__ H0) {
    const int B = blockIdx.x * blockDim.x + threadIdx.x;
    const int A = blockIdx.y * blockDim.y + threadIdx.y;
    if (A >= nat || B >= nat) return;
    const int N = nat * nper;
    double hb[4][4], sb[4][4];
    if (A == B) {
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) {
                sb[i][j] = (i == j) ? 1.0 : 0.0;
                hb[i][j] = (i == j && i < nper) ? onsite[A * nper + i] : 0.0;
            }
    } else {
        const double dx = R[3 * B] - R[3 * A], dy = R[3 * B + 1] - R[3 * A + 1],
                     dz = R[3 * B + 2] - R[3 * A + 2];
        const double r = sqrt(dx * dx + dy * dy + dz * dz);
        const double c[3] = {dx / r, dy / r, dz / r};
        const double eh = exp(-r / mp.lam_H), es = exp(-r / mp.lam_S);
        double kh[4], ks[4];
        for (int k = 0; k < 4; ++k) {
            kh[k] = mp.eta[k] * mp.t0 * eh;
            ks[k] = -mp.eta[k] * mp.s0 * es;
        }
        hb[0][0] = kh[0];
        sb[0][0] = ks[0];
        for (int a = 0; a < 3; ++a) {
            hb[0][1 + a] = c[a] * kh[1];
            sb[0][1 + a] = c[a] * ks[1];
            hb[1 + a][0] = -c[a] * kh[1];
            sb[1 + a][0] = -c[a] * ks[1];
            for (int b = 0; b < 3; ++b) {
                const double cc = c[a] * c[b];
                hb[1 + a][1 + b] = cc * (kh[2] - kh[3]) + (a == b ? kh[3] : 0.0);
                sb[1 + a][1 + b] = cc * (ks[2] - ks[3]) + (a == b ? ks[3] : 0.0);
            }
        }
    }
    for (int i = 0; i < nper; ++i) {
        const size_t row = (size_t)(A * nper + i) * N + (size_t)B * nper;
        for (int j = 0; j < nper; ++j) {
            S[row + j] = sb[i][j];
            H0[row + j] = hb[i][j];
        }
    }
}

// Short-range part zeta(R) of gamma for exponents ta, tb (tau = 16 U / 5):
// Coulomb integral of two normalised exp(-tau r) densities is 1/R - zeta(R).
__device__ double gamma_short(double ta, double tb, double R) {
    const double tmax = ta > tb ? ta : tb;
    if (fabs(ta - tb) < 3e-4 * tmax) {
        const double t = 0.5 * (ta + tb);
        return exp(-t * R) * (1.0 / R + 11.0 * t / 16.0 + 3.0 * t * t * R / 16.0 +
                              t * t * t * R * R / 48.0);
    }
    double z = 0.0;
    for (int s = 0; s < 2; ++s) {
        const double a = s ? tb : ta, b = s ? ta : tb;
        const double a2 = a * a, b2 = b * b, d = a2 - b2;
        const double b4 = b2 * b2;
        z += exp(-a * R) * (b4 * a / (2.0 * d * d) - (b4 * b2 - 3.0 * a2 * b4) / (d * d * d * R));
    }
    return z;
}

__global__ void k_build_gamma(int nat, const double* __restrict__ R, const double* __restrict__ U,
                              double* __restrict__ G) {
    const int B = blockIdx.x * blockDim.x + threadIdx.x;
    const int A = blockIdx.y * blockDim.y + threadIdx.y;
    if (A >= nat || B >= nat) return;
    double g;
    if (A == B) {
        g = U[A];
    } else {
        const double dx = R[3 * B] - R[3 * A], dy = R[3 * B + 1] - R[3 * A + 1],
                     dz = R[3 * B + 2] - R[3 * A + 2];
        const double r = sqrt(dx * dx + dy * dy + dz * dz);
        g = 1.0 / r - gamma_short(3.2 * U[A], 3.2 * U[B], r);
    }
    G[(size_t)A * nat + B] = g;
}

// Row-major upper triangle -> lower triangle (after a column-major lower potri).
__global__ void k_sym_upper_to_lower(int N, double* A) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y * blockDim.y + threadIdx.y;
    if (r < N && c < N && r > c) A[(size_t)r * N + c] = A[(size_t)c * N + r];
}

__global__ void k_transpose(int N, const double* __restrict__ in, double* __restrict__ out) {
    __shared__ double t[kTile][kTile + 1];
    const int bx = blockIdx.x * kTile, by = blockIdx.y * kTile;
    for (int y = threadIdx.y; y < kTile; y += blockDim.y) {
        const int r = by + y, c = bx + threadIdx.x;
        if (r < N && c < N) t[y][threadIdx.x] = in[(size_t)r * N + c];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < kTile; y += blockDim.y) {
        const int r = bx + y, c = by + threadIdx.x;
        if (r < N && c < N) out[(size_t)r * N + c] = t[threadIdx.x][y];
    }
}

// partial[row][ct] = sum over the 32 columns of tile ct of Re rho[row][col] * S[row][col]
// (eq:qmulik: q_A = sum_{nu in A} Re (rho S)_{nu nu}; S is symmetric).  Summed in
// column order, exactly as the update kernel sums them, so a state loaded from a
// checkpoint continues bitwise.
__global__ void k_mulliken_partials(int N, int nct, const double* __restrict__ rre,
                                    const double* __restrict__ S, double* __restrict__ partial) {
    __shared__ double pv_s[kTile][kTile + 1];
    const int ct = blockIdx.x;
    const int col = ct * kTile + threadIdx.x;
    for (int y = threadIdx.y; y < kTile; y += blockDim.y) {
        const int row = blockIdx.y * kTile + y;
        double v = 0.0;
        if (row < N && col < N) v = rre[(size_t)row * N + col] * S[(size_t)row * N + col];
        pv_s[y][threadIdx.x] = v;
    }
    __syncthreads();
    if (threadIdx.y == 0) {
        const int row = blockIdx.y * kTile + threadIdx.x;
        double sum = 0.0;
#pragma unroll 8
        for (int k = 0; k < kTile; ++k) sum += pv_s[threadIdx.x][k];
        if (row < N) partial[(size_t)row * nct + ct] = sum;
    }
}

// q_A = sum of the Mulliken row partials of A's orbitals (contiguous in the
// [row][ct] layout): one warp per atom.
__global__ void k_charges(int nat, int nper, int nct, const double* __restrict__ partial,
                          const double* __restrict__ q0, double* __restrict__ q,
                          double* __restrict__ dq, double* reset0, double* reset1,
                          tc::DynScales* __restrict__ dyn, int cur,
                          const double* __restrict__ qbase) {
    const int lane = threadIdx.x & 31;
    const int A = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (reset0) *reset0 = 0.0;
        if (reset1) *reset1 = 0.0;
        if (dyn) {
            // FP16X6 bookkeeping of a step: the maximum of the deviation written by the
            // previous update now describes buffer cur; start this step's maxima
            dyn->max_drho[cur] = dyn->max_drho[2];
            dyn->max_drho[2] = 0.0;
            for (int k = 0; k < tc::kMaxParts; ++k) dyn->max_x[k] = 0.0;
        }
    }
    if (A >= nat) return;
    const double* p = partial + (size_t)A * nper * nct;
    double s = 0.0;
#pragma unroll 4
    for (int i = lane; i < nper * nct; i += 32) s += p[i];
    s = warp_sum(s);
    if (lane == 0) {
        if (qbase) s += qbase[A];   // partials of the deviation rho - rho_ref
        q[A] = s;
        dq[A] = s - q0[A];
    }
}

// Warp per atom A: gdq_A = sum_B gamma_AB dq_B;  v_A = [scc] gdq_A + R_A . E(t_n)
// (eq:hscc, eq:hsccvext with V_ext,A = R_A . E).  Block 0 also records E(t_n),
// the dipole mu = -sum_A dq_A R_A into the history ring, and sum_A dq_A V_ext,A.
__global__ void k_potential(int nat, int nper, int scc, const double* __restrict__ gamma,
                            const double* __restrict__ dq, const double* __restrict__ R,
                            DevScalars* __restrict__ sc, double* __restrict__ v_orb,
                            double* __restrict__ v_atom, double* __restrict__ gdq,
                            double* __restrict__ hist, const double* __restrict__ v_ref,
                            float* __restrict__ dv_f, double* __restrict__ max_dv, int record) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarp = blockDim.x >> 5;
    const long long n = sc->step;
    // the field at t_n, evaluated once per block
    __shared__ double E_sh[3];
    if (threadIdx.x == 0) {
        const double t = sc->t_base + (double)(n - sc->n_base) * sc->dt;
        field_at(sc->field, t, E_sh);
    }
    __syncthreads();
    const double E[3] = {E_sh[0], E_sh[1], E_sh[2]};
    for (int A = blockIdx.x * nwarp + warp; A < nat; A += gridDim.x * nwarp) {
        double s = 0.0;
        if (scc) {
            const double* g = gamma + (size_t)A * nat;
#pragma unroll 8
            for (int B = lane; B < nat; B += 32) s += g[B] * dq[B];
        }
        s = warp_sum(s);
        const double vA = s + R[3 * A] * E[0] + R[3 * A + 1] * E[1] + R[3 * A + 2] * E[2];
        if (lane < nper) {
            const int o = A * nper + lane;
            v_orb[o] = vA;
            if (dv_f) dv_f[o] = (float)(vA - v_ref[o]);
        }
        if (lane == 0) {
            v_atom[A] = vA;
            gdq[A] = s;
            if (max_dv)
                atomicMax(reinterpret_cast<unsigned long long*>(max_dv),
                          (unsigned long long)__double_as_longlong(fabs(vA - v_ref[A * nper])));
        }
    }
    if (blockIdx.x == 0 && record) {
        __shared__ double red[4][32];
        double m0 = 0, m1 = 0, m2 = 0, ee = 0;
        for (int A = threadIdx.x; A < nat; A += blockDim.x) {
            const double d = dq[A];
            m0 -= d * R[3 * A];
            m1 -= d * R[3 * A + 1];
            m2 -= d * R[3 * A + 2];
            ee += d * (R[3 * A] * E[0] + R[3 * A + 1] * E[1] + R[3 * A + 2] * E[2]);
        }
        m0 = warp_sum(m0);
        m1 = warp_sum(m1);
        m2 = warp_sum(m2);
        ee = warp_sum(ee);
        if (lane == 0) {
            red[0][warp] = m0;
            red[1][warp] = m1;
            red[2][warp] = m2;
            red[3][warp] = ee;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0, b = 0, c = 0, e = 0;
            for (int w = 0; w < nwarp; ++w) {
                a += red[0][w];
                b += red[1][w];
                c += red[2][w];
                e += red[3][w];
            }
            sc->mu[0] = a;
            sc->mu[1] = b;
            sc->mu[2] = c;
            sc->e_ext = e;
            sc->E[0] = E[0];
            sc->E[1] = E[1];
            sc->E[2] = E[2];
            const long long slot = n % sc->hist_cap;
            const long long s2 = slot < 0 ? slot + sc->hist_cap : slot;
            hist[3 * s2] = a;
            hist[3 * s2 + 1] = b;
            hist[3 * s2 + 2] = c;
        }
    }
}

__global__ void k_build_hamiltonian(int N, const double* __restrict__ H0,
                                    const double* __restrict__ S, const double* __restrict__ v,
                                    double* __restrict__ H) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y * blockDim.y + threadIdx.y;
    if (r >= N || c >= N) return;
    const size_t i = (size_t)r * N + c;
    H[i] = H0[i] + 0.5 * S[i] * (v[r] + v[c]);
}

// Leapfrog / Euler update of the FP64 form (eq:leapfrog with eq:eomrho):
//   out = base + factor * rhodot,  rhodot = -i (X - X^dagger) - (Z + Z^dagger),
//   X = S^-1 H rho, Z = S^-1 D rho (moving nuclei only).
// Re rhodot_ij = Im X_ij + Im X_ji;  Im rhodot_ij = -(Re X_ij - Re X_ji).
// A block (32 x 8 threads) owns the tile pair (bi, bj), bi <= bj, so both halves
// come out of the same operands and rho stays exactly Hermitian.  The Mulliken
// row partials of the new rho are fused in.
__global__ void __launch_bounds__(256)
    k_update(int N, int nct, const double* __restrict__ Xre, const double* __restrict__ Xim,
             const double* __restrict__ bre, const double* __restrict__ bim,
             double* __restrict__ ore, double* __restrict__ oim, double factor,
             const double* __restrict__ S, double* __restrict__ partial,
             DevScalars* __restrict__ sc, const double* __restrict__ zre,
             const double* __restrict__ zim) {
    const int bi = blockIdx.y, bj = blockIdx.x;
    if (bi > bj) return;
    constexpr int RPT = kTile / 8;   // rows per thread
    __shared__ double xr_ij[kTile][kTile + 1], xi_ij[kTile][kTile + 1];
    __shared__ double xr_ji[kTile][kTile + 1], xi_ji[kTile][kTile + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int y = ty + 8 * k;
        int r = bi * kTile + y, c = bj * kTile + tx;
        double a = 0, b = 0;
        if (r < N && c < N) {
            const size_t i = (size_t)r * N + c;
            a = Xre[i];
            b = Xim[i];
        }
        xr_ij[y][tx] = a;
        xi_ij[y][tx] = b;
        r = bj * kTile + y;
        c = bi * kTile + tx;
        a = 0;
        b = 0;
        if (r < N && c < N) {
            const size_t i = (size_t)r * N + c;
            a = Xre[i];
            b = Xim[i];
        }
        xr_ji[y][tx] = a;
        xi_ji[y][tx] = b;
    }
    __syncthreads();
    __shared__ double pv_s[kTile][kTile + 1];
    for (int half = 0; half < (bi == bj ? 1 : 2); ++half) {
        const int ti = half ? bj : bi, tj = half ? bi : bj;
        double b_re[RPT], b_im[RPT], s_v[RPT];
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int r = ti * kTile + ty + 8 * k, c = tj * kTile + tx;
            b_re[k] = b_im[k] = s_v[k] = 0.0;
            if (r < N && c < N) {
                const size_t i = (size_t)r * N + c;
                b_re[k] = bre[i];
                b_im[k] = bim[i];
                s_v[k] = S[i];
            }
        }
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int y = ty + 8 * k;
            const int r = ti * kTile + y, c = tj * kTile + tx;
            double pv = 0.0;
            if (r < N && c < N) {
                double x_ij_re, x_ij_im, x_ji_re, x_ji_im;
                if (!half) {
                    x_ij_re = xr_ij[y][tx];
                    x_ij_im = xi_ij[y][tx];
                    x_ji_re = xr_ji[tx][y];
                    x_ji_im = xi_ji[tx][y];
                } else {
                    x_ij_re = xr_ji[y][tx];
                    x_ij_im = xi_ji[y][tx];
                    x_ji_re = xr_ij[tx][y];
                    x_ji_im = xi_ij[tx][y];
                }
                // the (j,i) element repeats these operations on the swapped operands
                double dre = x_ij_im + x_ji_im;
                double dim = -(x_ij_re - x_ji_re);
                const size_t i = (size_t)r * N + c;
                if (zre) {
                    const size_t j = (size_t)c * N + r;
                    dre -= zre[i] + zre[j];
                    dim -= zim[i] - zim[j];
                }
                const double nre = b_re[k] + factor * dre;
                const double nim = b_im[k] + factor * dim;
                ore[i] = nre;
                oim[i] = nim;
                pv = nre * s_v[k];
            }
            pv_s[y][tx] = pv;
        }
        // Mulliken row partials: thread (tx, ty == 0) sums row tx of this tile
        __syncthreads();
        if (ty == 0) {
            const int r = ti * kTile + tx;
            double sum = 0.0;
#pragma unroll 8
            for (int k = 0; k < kTile; ++k) sum += pv_s[tx][k];
            if (r < N) partial[(size_t)r * nct + tj] = sum;
        }
        __syncthreads();
    }
    if (bi == 0 && bj == 0 && threadIdx.x == 0 && threadIdx.y == 0) sc->step += 1;
}

// C = diag(p) P diag(conj p), p_mu = exp(-i E0 dir . R_A(mu)): the phase factors of
// eq:rhokick with V = -E0 diag(dir . R).
__global__ void k_kick_phase(int N, int nper, const double* __restrict__ R, double E0, double d0,
                             double d1, double d2, const double* __restrict__ Pre,
                             const double* __restrict__ Pim, double* __restrict__ Cre,
                             double* __restrict__ Cim) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y * blockDim.y + threadIdx.y;
    if (r >= N || c >= N) return;
    const int A = r / nper, B = c / nper;
    const double xa = d0 * R[3 * A] + d1 * R[3 * A + 1] + d2 * R[3 * A + 2];
    const double xb = d0 * R[3 * B] + d1 * R[3 * B + 1] + d2 * R[3 * B + 2];
    // p_r conj(p_c) = exp(-i E0 (x_a - x_b))
    double sn, cs;
    sincos(-E0 * (xa - xb), &sn, &cs);
    const size_t i = (size_t)r * N + c;
    const double pr = Pre[i], pi = Pim[i];
    Cre[i] = cs * pr - sn * pi;
    Cim[i] = cs * pi + sn * pr;
}

// out = 1/2 (T + T^dagger)
__global__ void k_hermitian_half(int N, const double* __restrict__ Tre,
                                 const double* __restrict__ Tim, double* __restrict__ ore,
                                 double* __restrict__ oim) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y * blockDim.y + threadIdx.y;
    if (r >= N || c >= N) return;
    const size_t i = (size_t)r * N + c, j = (size_t)c * N + r;
    ore[i] = 0.5 * (Tre[i] + Tre[j]);
    oim[i] = 0.5 * (Tim[i] - Tim[j]);
}

// Per block: sum Re rho * H0, sum Re rho * S, sum Im rho * S, max |rho_ij - conj rho_ji|.
__global__ void k_obs_reduce(int N, const double* __restrict__ rre, const double* __restrict__ rim,
                             const double* __restrict__ H0, const double* __restrict__ S,
                             double* __restrict__ out) {
    double a = 0, b = 0, c = 0, m = 0;
    const size_t NN = (size_t)N * N;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < NN;
         i += (size_t)gridDim.x * blockDim.x) {
        const size_t r = i / N, col = i % N, j = col * N + r;
        const double re = rre[i], im = rim[i];
        a += re * H0[i];
        b += re * S[i];
        c += im * S[i];
        const double e1 = fabs(re - rre[j]), e2 = fabs(im + rim[j]);
        m = fmax(m, fmax(e1, e2));
    }
    __shared__ double red[4][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) {
        red[0][w] = a;
        red[1][w] = b;
        red[2][w] = c;
        red[3][w] = m;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0, s1 = 0, s2 = 0, mx = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            s0 += red[0][k];
            s1 += red[1][k];
            s2 += red[2][k];
            mx = fmax(mx, red[3][k]);
        }
        out[4 * blockIdx.x] = s0;
        out[4 * blockIdx.x + 1] = s1;
        out[4 * blockIdx.x + 2] = s2;
        out[4 * blockIdx.x + 3] = mx;
    }
}

__global__ void k_obs_finish(int nb, const double* __restrict__ in, double* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s0 = 0, s1 = 0, s2 = 0, mx = 0;
    for (int k = 0; k < nb; ++k) {
        s0 += in[4 * k];
        s1 += in[4 * k + 1];
        s2 += in[4 * k + 2];
        mx = fmax(mx, in[4 * k + 3]);
    }
    out[0] = s0;
    out[1] = s1;
    out[2] = s2;
    out[3] = mx;
}

// out[m][k] = in[m][k] * f[k]
__global__ void k_scale_cols(int N, const double* __restrict__ in, const double* __restrict__ f,
                             double* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y * blockDim.y + threadIdx.y;
    if (r >= N || c >= N) return;
    out[(size_t)r * N + c] = in[(size_t)r * N + c] * f[c];
}

inline dim3 grid2(int nx, int ny, dim3 b) {
    return dim3((nx + b.x - 1) / b.x, (ny + b.y - 1) / b.y);
}

}  // namespace

void launch_build_model(const Ctx& c, const double* R, double* S, double* H0, cudaStream_t st) {
    dim3 b(32, 8);
    k_build_model<<<grid2(c.nat, c.nat, b), b, 0, st>>>(c.nat, c.nper, R, c.d_onsite, c.mp, S, H0);
}

void launch_build_gamma(const Ctx& c, const double* R, double* gamma, cudaStream_t st) {
    dim3 b(32, 8);
    k_build_gamma<<<grid2(c.nat, c.nat, b), b, 0, st>>>(c.nat, R, c.d_U, gamma);
}

void launch_symmetrize_upper_to_lower(int N, double* A, cudaStream_t st) {
    dim3 b(32, 8);
    k_sym_upper_to_lower<<<grid2(N, N, b), b, 0, st>>>(N, A);
}

void launch_transpose(int N, const double* in, double* out, cudaStream_t st) {
    dim3 b(kTile, 8);
    dim3 g((N + kTile - 1) / kTile, (N + kTile - 1) / kTile);
    k_transpose<<<g, b, 0, st>>>(N, in, out);
}

void launch_mulliken_partials(int N, const double* rho_re, const double* S, double* partial,
                              cudaStream_t st) {
    const int nct = (N + kTile - 1) / kTile;
    dim3 b(kTile, 8);
    k_mulliken_partials<<<dim3(nct, nct), b, 0, st>>>(N, nct, rho_re, S, partial);
}

void launch_charges(const Ctx& c, const double* partial, double* q, double* dq, cudaStream_t st,
                    double* reset0, double* reset1, tc::DynScales* dyn, int cur,
                    const double* qbase) {
    k_charges<<<(c.nat + 7) / 8, 256, 0, st>>>(c.nat, c.nper, c.nct, partial, c.d_q0, q, dq,
                                               reset0, reset1, dyn, cur, qbase);
}

void launch_potential(const Ctx& c, const double* gamma, const double* dq, const double* R,
                      DevScalars* sc, double* v_orb, double* v_atom, double* gdq, double* hist,
                      const double* v_ref, float* dv_orb, cudaStream_t st, double* max_dv,
                      int record) {
    const int warps = 8;
    const int blocks = (c.nat + warps - 1) / warps;
    k_potential<<<blocks, warps * 32, 0, st>>>(c.nat, c.nper, c.prm.scc, gamma, dq, R, sc, v_orb,
                                               v_atom, gdq, hist, v_ref, dv_orb, max_dv, record);
}

void launch_build_hamiltonian(int N, const double* H0, const double* S, const double* v_orb,
                              double* H, cudaStream_t st) {
    dim3 b(32, 8);
    k_build_hamiltonian<<<grid2(N, N, b), b, 0, st>>>(N, H0, S, v_orb, H);
}

void launch_update(const Ctx& c, const double* Xre, const double* Xim, const double* base_re,
                   const double* base_im, double* out_re, double* out_im, double factor,
                   const double* S, double* partial, DevScalars* sc, cudaStream_t st,
                   const double* zre, const double* zim) {
    dim3 b(kTile, 8);
    k_update<<<dim3(c.nct, c.nct), b, 0, st>>>(c.N, c.nct, Xre, Xim, base_re, base_im, out_re,
                                               out_im, factor, S, partial, sc, zre, zim);
}

void launch_kick_phase(int N, int n_per, const double* R, double strength, const double* dir,
                       const double* Pre, const double* Pim, double* Cre, double* Cim,
                       cudaStream_t st) {
    dim3 b(32, 8);
    k_kick_phase<<<grid2(N, N, b), b, 0, st>>>(N, n_per, R, strength, dir[0], dir[1], dir[2], Pre,
                                               Pim, Cre, Cim);
}

void launch_hermitian_half(int N, const double* Tre, const double* Tim, double* out_re,
                           double* out_im, cudaStream_t st) {
    dim3 b(32, 8);
    k_hermitian_half<<<grid2(N, N, b), b, 0, st>>>(N, Tre, Tim, out_re, out_im);
}

void launch_obs_reduce(int N, const double* rho_re, const double* rho_im, const double* H0,
                       const double* S, double* block_out, int n_blocks, cudaStream_t st) {
    k_obs_reduce<<<n_blocks, 256, 0, st>>>(N, rho_re, rho_im, H0, S, block_out);
}

void launch_obs_finish(int n_blocks, const double* block_out, double* out4, cudaStream_t st) {
    k_obs_finish<<<1, 32, 0, st>>>(n_blocks, block_out, out4);
}

void launch_scale_rows_f(int N, const double* in, const double* f, double* out, cudaStream_t st) {
    dim3 b(32, 8);
    k_scale_cols<<<grid2(N, N, b), b, 0, st>>>(N, in, f, out);
}

}  // namespace tdb

namespace tdb {

namespace {

__global__ void k_f64_to_f32(size_t n, const double* __restrict__ in, float* __restrict__ out) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

// Newton-Schulz step for the inverse of S: X <- 2 X - 1/2 (Q + Q^T) with Q = X S X and X
// symmetric (the symmetric part keeps the iterate exactly symmetric).
__global__ void k_ns_update(int N, double* __restrict__ X, const double* __restrict__ Q) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y * blockDim.y + threadIdx.y;
    if (r >= N || c >= N) return;
    const size_t i = (size_t)r * N + c, j = (size_t)c * N + r;
    X[i] = 2.0 * X[i] - 0.5 * (Q[i] + Q[j]);
}

__global__ void k_f32_to_f64(size_t n, const float* __restrict__ in, double* __restrict__ out) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        out[i] = (double)in[i];
}

// out[r][c] = a[r][c] + b[r][c] with row strides N (a), ldb (b), ldo (out)
__global__ void k_add_f32(int N, const float* __restrict__ a, const float* __restrict__ b, int ldb,
                          float* __restrict__ out, int ldo) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y * blockDim.y + threadIdx.y;
    if (r >= N || c >= N) return;
    out[(size_t)r * ldo + c] = a[(size_t)r * N + c] + b[(size_t)r * ldb + c];
}

// out[0] = 1/2 sum_A dq_A (gamma dq)_A (eq:coul), out[1] = sum_{A<B} rep_A exp(-r/rep_b),
// out[2] = nuclear kinetic energy (moving nuclei only)
__global__ void k_small_energies(int nat, const double* __restrict__ dq,
                                 const double* __restrict__ gdq, const double* __restrict__ R,
                                 const double* __restrict__ V, const double* __restrict__ mass,
                                 double rep_A, double rep_b, int kinetic,
                                 double* __restrict__ out) {
    double ec = 0, er = 0, ek = 0;
    for (int A = threadIdx.x; A < nat; A += blockDim.x) {
        ec += 0.5 * dq[A] * gdq[A];
        if (kinetic)
            ek += 0.5 * mass[A] * 1822.888486 *
                  (V[3 * A] * V[3 * A] + V[3 * A + 1] * V[3 * A + 1] + V[3 * A + 2] * V[3 * A + 2]);
        if (rep_A != 0.0)
            for (int B = A + 1; B < nat; ++B) {
                const double dx = R[3 * B] - R[3 * A], dy = R[3 * B + 1] - R[3 * A + 1],
                             dz = R[3 * B + 2] - R[3 * A + 2];
                er += rep_A * exp(-sqrt(dx * dx + dy * dy + dz * dz) / rep_b);
            }
    }
    __shared__ double red[3][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    ec = warp_sum(ec);
    er = warp_sum(er);
    ek = warp_sum(ek);
    if (lane == 0) {
        red[0][w] = ec;
        red[1][w] = er;
        red[2][w] = ek;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0, c = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            a += red[0][k];
            b += red[1][k];
            c += red[2][k];
        }
        out[0] = a;
        out[1] = b;
        out[2] = c;
    }
}

// out = max |x| (out must start at 0): non-negative doubles order like their bit patterns
__global__ void k_absmax(size_t n, const double* __restrict__ x, const double* __restrict__ sub,
                         double* __restrict__ out) {
    double m = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        m = fmax(m, fabs(sub ? x[i] - sub[i] : x[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0)
        atomicMax(reinterpret_cast<unsigned long long*>(out), (unsigned long long)__double_as_longlong(m));
}

}  // namespace

void launch_absmax(size_t n, const double* x, double* out, cudaStream_t st, const double* sub) {
    k_absmax<<<608, 256, 0, st>>>(n, x, sub, out);
}

void launch_ns_update(int N, double* X, const double* Q, cudaStream_t st) {
    dim3 b(32, 8);
    k_ns_update<<<grid2(N, N, b), b, 0, st>>>(N, X, Q);
}

void launch_f32_to_f64(size_t n, const float* in, double* out, cudaStream_t st) {
    k_f32_to_f64<<<1216, 256, 0, st>>>(n, in, out);
}

void launch_f64_to_f32(size_t n, const double* in, float* out, cudaStream_t st) {
    k_f64_to_f32<<<1216, 256, 0, st>>>(n, in, out);
}

void launch_add_f32_strided(int N, const float* a, const float* b, int ldb, float* out, int ldo,
                            cudaStream_t st) {
    dim3 bl(32, 8);
    k_add_f32<<<grid2(N, N, bl), bl, 0, st>>>(N, a, b, ldb, out, ldo);
}

void launch_small_energies(const Ctx& c, double* out, cudaStream_t st) {
    k_small_energies<<<1, 256, 0, st>>>(c.nat, c.dq, c.gdq, c.d_R, c.d_Vn, c.d_mass, c.mp.rep_A,
                                        c.mp.rep_b, c.prm.move_nuclei, out);
}

}  // namespace tdb

// ---------------------------------------------------------------------------
// Reduced-precision forms: the density master is rho - rho_ref held as an FP32
// pair (hi + lo, ~48 bits) per element, so the per-step update runs without FP64
// arithmetic (FP64 issues at 1/64 of the FP32 rate on this part).  The FP64
// matrices rho_re / rho_im are a view, materialised for observables, kicks and
// checkpoints.
// ---------------------------------------------------------------------------

namespace tdb {

namespace {

// s + e = a + b exactly (Knuth's two-sum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// (hi, lo) += inc, renormalised
__device__ __forceinline__ void df_add(float& hi, float& lo, float inc) {
    float s, e;
    two_sum(hi, inc, s, e);
    e += lo;
    hi = s + e;
    lo = e - (hi - s);
}

// FP32-pair ("double-float", ~48 bits) sums and products.  FP64 issues at a small fraction
// of the FP32 rate on this part, so the per-step reductions use these.  The sum is
// commutative bit for bit (the rounded sum and its exact error do not depend on the
// order), so butterfly reductions give the same value on every lane.
__device__ __forceinline__ float2 df2_add(float2 a, float2 b) {
    float s, e;
    two_sum(a.x, b.x, s, e);
    e += a.y + b.y;
    const float h = s + e;
    return make_float2(h, e - (h - s));
}
// a * b with the exact product of the high parts (FMA) and the cross terms
__device__ __forceinline__ float2 df2_mul(float2 a, float2 b) {
    const float p = a.x * b.x;
    const float e = fmaf(a.x, b.x, -p) + (a.x * b.y + a.y * b.x);
    return make_float2(p, e);
}
__device__ __forceinline__ float2 df2_shfl_xor(float2 v, int o) {
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}
__device__ __forceinline__ float2 df2_warp_sum(float2 v) {
    for (int o = 16; o > 0; o >>= 1) v = df2_add(v, df2_shfl_xor(v, o));
    return v;
}
__device__ __forceinline__ float2 ldcg2(const float2* p) { return __ldcg(p); }

// Mulliken product of one element of the deviation master with FP32 S: (re_hi + re_lo) S
// as (hi, lo) with the high product exact
__device__ __forceinline__ float2 mulliken_elem(float rh, float rl, float s) {
    const float p = rh * s;
    return make_float2(p, fmaf(rh, s, -p) + rl * s);
}
// Sum of the 32 element values of a tile row (column order fixed: four interleaved
// partial sums, then combined), shared by the update and the master partials.
__device__ __forceinline__ float2 tile_row_sum(const float2* row) {
    float2 a[4] = {row[0], row[1], row[2], row[3]};
#pragma unroll
    for (int k = 4; k < kTile; k += 4)
#pragma unroll
        for (int j = 0; j < 4; ++j) a[j] = df2_add(a[j], row[k + j]);
    return df2_add(df2_add(a[0], a[1]), df2_add(a[2], a[3]));
}

// Power-of-two scale mapping a bound m into (63.5, 127] (FP32 form of tc::pscale; an
// FP32 quotient that rounds up to a power of two gives a scale one step too large, which
// only moves a little more of a value into its FP16 tails: the heads stay within +-127).
__device__ __forceinline__ float pscale_f(float m) {
    if (!(m > 0.f)) return 1099511627776.0f;   // 2^40
    int e;
    frexpf(127.0f / m, &e);
    e -= 1;
    e = min(40, max(-40, e));
    return ldexpf(1.0f, e);
}

// E(t) of eq:pumpf with the phase formed and reduced modulo 2 pi in FP64 and the sine and
// envelope in FP32 (relative error ~1e-7, far below the reduced forms' product error).
__device__ void field_at_f(const FieldDev& f, double t, float E[3]) {
    if (!f.on) {
        E[0] = E[1] = E[2] = 0.f;
        return;
    }
    const double kTwoPi = 6.283185307179586476925;
    float env = 1.f;
    if (f.envelope == 1) {
        const double x = t - f.t_center;
        const double y = x * x * (4.0 * 0.69314718055994530942 / (f.fwhm * f.fwhm));
        const float yf = (float)y;
        env = expf(-yf) * (1.f - (float)(y - (double)yf));
    } else if (f.envelope == 2) {
        if (t >= 0.0 && t <= f.fwhm) {
            const float sv = sinf((float)(3.14159265358979323846 * t / f.fwhm));
            env = sv * sv;
        } else {
            env = 0.f;
        }
    }
    double ph = f.omega * t + f.phase;
    ph -= kTwoPi * rint(ph * (1.0 / kTwoPi));
    const float a = (float)f.E0 * sinf((float)ph) * env;
    E[0] = a * (float)f.dir[0];
    E[1] = a * (float)f.dir[1];
    E[2] = a * (float)f.dir[2];
}

// Counter increment with acquire-release semantics at GPU scope: after a block barrier it
// publishes what the block wrote (release is cumulative over the barrier) and, for the block
// that completes a count, makes what the others published visible (acquire; the barrier
// that follows extends it to the block).  One such atomic per block replaces per-thread
// fences, which serialise across the GPU.
__device__ __forceinline__ int atom_add_acq_rel(int* p, int v) {
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v)
                 : "memory");
    return old;
}

// Evaluation of a level from its Mulliken row partials, in two kernels of one block per
// kLvAtoms atoms (64 threads, two warps, per atom).
//
// Charges (block blk): dq_A = sum of the partials of atom A's rows (thread t of the atom sums
// partials t, t + 64, ... in order; each warp reduces by a butterfly, and the atom's two
// warps are added), into dq[A]; the block's sums of dq_A R_A and dq_A into bsum[blk]
// (dipole and trace parts).
__device__ void level_dq_block(const LevelArgs& a, int blk) {
    __shared__ float2 half_sum[8];
    __shared__ float2 red[kLvAtoms][4];
    __shared__ float2 r_sh[3 * kLvAtoms];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const float2 z = make_float2(0.f, 0.f);
    const int A0 = blk * kLvAtoms;
    const int A = A0 + (warp >> 1), t = (warp & 1) * 32 + lane;
    const int len = a.nper * a.nct;
    if (tid < 3 * kLvAtoms) r_sh[tid] = A0 * 3 + tid < 3 * a.nat ? __ldg(a.R2 + 3 * A0 + tid) : z;
    // the potentials kernel may be scheduled now (it loads its constants, then waits)
    pdl_launch_dependents();
    pdl_wait();
    float2 s = z;
    if (A < a.nat) {
        const float2* p = a.partial + (size_t)A * len;
        for (int k0 = t; k0 < len; k0 += 512) {
            float2 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = k0 + 64 * u < len ? ldcg2(p + k0 + 64 * u) : z;
#pragma unroll
            for (int u = 0; u < 8; ++u) s = df2_add(s, v[u]);
        }
    }
    s = df2_warp_sum(s);
    if (lane == 0) half_sum[warp] = s;
    __syncthreads();
    if (tid < kLvAtoms) {
        const int Aa = A0 + tid;
        float2 m[4] = {z, z, z, z};
        if (Aa < a.nat) {
            const float2 d = df2_add(half_sum[2 * tid], half_sum[2 * tid + 1]);
            a.dq[Aa] = d;
#pragma unroll
            for (int k = 0; k < 3; ++k) m[k] = df2_mul(d, r_sh[3 * tid + k]);
            m[3] = d;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) red[tid][k] = m[k];
    }
    __syncthreads();
    if (tid < 4) {
        float2 x = red[0][tid];
#pragma unroll
        for (int i = 1; i < kLvAtoms; ++i) x = df2_add(x, red[i][tid]);
        a.bsum[4 * blk + tid] = x;
    }
}

// Potentials and the level's scalars.  Blocks 0 .. level_blocks(nat) - 1 (kLvAtoms atoms
// each): dv_A = sum_B gamma_AB dq_B (eq:hscc; thread t of atom A takes B = t, t + 64, ...
// in order, each warp reduces by a butterfly, the atom's two warps are added) + R_A . E(t)
// + the SCC residual of rho_ref, written per orbital (dv_f), and the maximum |dv| over the
// blocks.  Block level_blocks(nat) (the totals block): Tr(rho S) and the renormalisation
// factor of level `slot` from the charge blocks' sums, the dipole mu = mu_ref - sum_A dq_A
// R_A into sc->mu and the history slot of step n_lvl, the field record.  The block that
// arrives last sets the FP16X6 scales of the next products and, with step_end, the step
// counter (to n_lvl) and the FP16X6 maxima (the new level is in `slot`); it resets the
// counters.  trace_only (one block): only Tr(rho S) and f - 1.
__device__ void level_final_block(const LevelArgs& a, int slot, long long n_lvl, bool trace_only,
                                  bool step_end, int blk, int nblk) {
    __shared__ float2 half_sum[8];
    __shared__ float2 tot[4];
    __shared__ float E_sh[3];
    __shared__ float rc_sh[kLvAtoms][4];
    __shared__ float mx_sh;
    __shared__ int last;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    DevScalars* sc = a.sc;
    const float2 z = make_float2(0.f, 0.f);
    const int nab = level_blocks(a.nat);
    // constants first (gamma of this thread's first products, positions, residuals); the
    // charges and scalars of the previous kernels after pdl_wait
    const int A0 = blk * kLvAtoms;
    const int A = A0 + (warp >> 1), t = (warp & 1) * 32 + lane;
    const bool atoms = !trace_only && blk < nab;
    float2 gv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int b = t + 64 * u;
        gv[u] = (atoms && a.scc && A < a.nat && b < a.nat) ? __ldg(a.gam2 + (size_t)A * a.nat + b) : z;
    }
    if (atoms && tid < kLvAtoms) {
        const int Aa = A0 + tid;
        const bool ok = Aa < a.nat;
        rc_sh[tid][0] = ok ? __ldg(&a.R2[3 * Aa].x) : 0.f;
        rc_sh[tid][1] = ok ? __ldg(&a.R2[3 * Aa + 1].x) : 0.f;
        rc_sh[tid][2] = ok ? __ldg(&a.R2[3 * Aa + 2].x) : 0.f;
        rc_sh[tid][3] = ok ? __ldg(a.c_res + Aa) : 0.f;
    }
    pdl_wait();
    if (tid == 0) {
        float E[3] = {0.f, 0.f, 0.f};
        if (!trace_only && sc->field.on) {
            const double t = sc->t_base + (double)(n_lvl - sc->n_base) * sc->dt;
            field_at_f(sc->field, t, E);
        }
        E_sh[0] = E[0];
        E_sh[1] = E[1];
        E_sh[2] = E[2];
        mx_sh = 0.f;
    }
    if (trace_only || blk == nab) {
        // the totals block: sums of the charge blocks' dipole and trace parts (warps 0-3)
        if (warp < 4) {
            float2 s = z;
            for (int r = lane; r < nab; r += 32) s = df2_add(s, ldcg2(a.bsum + 4 * r + warp));
            s = df2_warp_sum(s);
            if (lane == 0) tot[warp] = s;
        }
        __syncthreads();
        if (tid == 0) {
            // Tr(rho S) = N_e - c0 + sum_A dq_A;  f - 1 = (N_e - Tr) / Tr ~ (c0 - sum dq) / N_e
            const float2 d = tot[3];
            const float eps = (((float)sc->c0_trace - d.x) - d.y) * a.inv_ne;
            sc->eps_lvl[slot] = eps;
            sc->trace_lvl[slot] = (sc->n_e - sc->c0_trace) + ((double)d.x + (double)d.y);
        }
        if (trace_only) return;
        if (warp == 1) {
            // dipole (lanes 0-2, one component each) into sc and the history slot of step n_lvl
            const int k = lane < 3 ? lane : 0;
            const double mu = sc->mu_ref[k] - ((double)tot[k].x + (double)tot[k].y);
            const double ek = mu * (double)E_sh[k];
            const double e_ext = -(ek + __shfl_down_sync(0xffffffffu, ek, 1) +
                                   __shfl_down_sync(0xffffffffu, ek, 2));
            if (lane < 3) {
                long long h = n_lvl % sc->hist_cap;
                if (h < 0) h += sc->hist_cap;
                sc->mu[k] = mu;
                sc->E[k] = (double)E_sh[k];
                a.hist[3 * h + k] = mu;
            }
            if (lane == 0) sc->e_ext = e_ext;
        }
    } else {
        float2 acc = z;
        if (a.scc && A < a.nat) {
            const float2* g = a.gam2 + (size_t)A * a.nat;
            for (int b0 = t; b0 < a.nat; b0 += 512) {
                float2 qv[8];
                if (b0 != t)
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int b = b0 + 64 * u;
                        gv[u] = b < a.nat ? __ldg(g + b) : z;
                    }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int b = b0 + 64 * u;
                    qv[u] = b < a.nat ? __ldg(a.dq + b) : z;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) acc = df2_add(acc, df2_mul(gv[u], qv[u]));
            }
        }
        acc = df2_warp_sum(acc);
        if (lane == 0) half_sum[warp] = acc;
        __syncthreads();
        if (warp == 0) {
            float mx = 0.f;
            const int Aa = A0 + lane;
            if (lane < kLvAtoms && Aa < a.nat) {
                const float2 s = df2_add(half_sum[2 * lane], half_sum[2 * lane + 1]);
                const float ext = fmaf(rc_sh[lane][0], E_sh[0],
                                       fmaf(rc_sh[lane][1], E_sh[1], rc_sh[lane][2] * E_sh[2]));
                const float dv = s.x + (s.y + (ext + rc_sh[lane][3]));
                for (int k = 0; k < a.nper; ++k) a.dv_f[Aa * a.nper + k] = dv;
                mx = fabsf(dv);
            }
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (lane == 0) mx_sh = mx;
        }
    }
    // arrival of every block (atom blocks carry their maximum |dv|)
    __syncthreads();
    int* max_bits = a.count + 1;     // max |dv| of this evaluation (float bits, >= 0)
    if (tid == 0) {
        if (blk < nab) atomicMax(max_bits, __float_as_int(mx_sh));
        last = atom_add_acq_rel(a.count, 1) == nblk - 1;
    }
    __syncthreads();
    if (!last || tid != 0) return;
    const float m = __int_as_float(__ldcg(max_bits));
    tc::DynScales* dy = a.dyn;
    if (dy) {
        dy->max_dv = (double)m;
        if (a.has_scales) {
            dy->s_dh = pscale_f(m);
            dy->s_dm = pscale_f(m * (float)dy->sinv_norm);
        }
        for (int k = 0; k < tc::kMaxParts; ++k) dy->max_x[k] = 0.0;
        if (step_end) {
            // the maximum the update's blocks accumulated (atomics, read through L2)
            dy->max_drho[slot] = __ldcg(&dy->max_drho[2]);
            dy->max_drho[2] = 0.0;
        }
    }
    if (step_end) sc->step = n_lvl;
    // the counters, after this thread's read of the maximum
    a.count[0] = 0;
    a.count[1] = 0;
}

// Update of the FP32-pair master (eq:leapfrog, eq:eomrho, frozen nuclei): the same
// tile-pair scheme and operands as k_update, with the increment factor * rhodot formed
// as fh * d + fl * d (factor = fh + fl) so the step length carries no FP32 rounding.
// Every kRenormEvery steps the base level is first renormalised to Tr(rho S) = N_e:
// rho_base <- f rho_base with f = 1 + eps from its trace (Sec. 2.3: the exact leapfrog
// conserves the electron number; the reduced products do not, by ~1e-14 of N_e per step),
// i.e. the deviation gains eps (rho_ref + deviation).  Mulliken row partials of the new
// deviation in FP32-pair arithmetic, from which two small kernels evaluate the new level
// (level_dq_block, level_final_block).
// Steps between renormalisations of a leapfrog level (the reduced forms drift by ~1e-14 of
// N_e per step, so Tr(rho S) stays within ~1e-12 of N_e in between).
constexpr int kRenormEvery = 8;

__device__ __forceinline__ void update_df_block(const UpdateDfArgs& A, int b) {
    const int N = A.N, nct = A.nct;
    const MasterPtrs& base = A.base;
    const MasterPtrs& out = A.out;
    const float fh = A.fh, fl = A.fl;
    const double factor = A.factor;
    const float* __restrict__ Sf = A.Sf;
    const float* __restrict__ rgs = A.rgs;
    DevScalars* __restrict__ sc = A.sc;
    const UpdateOperands& ops = A.ops;
    const LevelArgs& lv = A.lv;
    // one block per tile pair bi <= bj: block b = bj (bj + 1) / 2 + bi
    int bj = (int)((sqrtf(8.0f * (float)b + 1.0f) - 1.0f) * 0.5f);
    while (bj * (bj + 1) / 2 > b) --bj;
    while ((bj + 1) * (bj + 2) / 2 <= b) ++bj;
    const int bi = b - bj * (bj + 1) / 2;
    constexpr int RPT = kTile / 8;
    {
        // every operand line of both halves (rows of 32 floats = one 128-byte line) is
        // requested from DRAM at once; the loads below then hit L2
        const int tid = threadIdx.y * blockDim.x + threadIdx.x;
        const int arr = tid >> 5, row = tid & 31;
        if (arr < 5) {
            const float* p = arr == 0 ? base.re_hi : arr == 1 ? base.re_lo : arr == 2 ? base.im_hi
                             : arr == 3 ? base.im_lo : Sf;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int ti = h ? bj : bi, tj = h ? bi : bj;
                const int r = ti * kTile + row, c = tj * kTile;
                if ((h == 0 || bi != bj) && r < N && c < N)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(p + (size_t)r * N + c));
            }
        }
    }
    // X, the scalars and the outputs belong to the previous kernels from here on
    pdl_wait();
    __shared__ float xr_ij[kTile][kTile + 1], xi_ij[kTile][kTile + 1];
    __shared__ float xr_ji[kTile][kTile + 1], xi_ji[kTile][kTile + 1];
    __shared__ float2 pv_s[kTile][kTile + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    // X = sum of its partial products, in a fixed order (all loads issued first)
    auto load_x = [&](size_t i, float& a, float& b) {
        float t[6];
#pragma unroll
        for (int q = 0; q < 4; ++q) t[q] = q < ops.nre ? ops.xre[q][i] : 0.f;
#pragma unroll
        for (int q = 0; q < 2; ++q) t[4 + q] = q < ops.nim ? ops.xim[q][i] : 0.f;
        a = ((t[0] + t[1]) + t[2]) + t[3];
        b = t[4] + t[5];
    };
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int y = ty + 8 * k;
        int r = bi * kTile + y, c = bj * kTile + tx;
        float a = 0.f, b = 0.f;
        if (r < N && c < N) load_x((size_t)r * N + c, a, b);
        xr_ij[y][tx] = a;
        xi_ij[y][tx] = b;
        r = bj * kTile + y;
        c = bi * kTile + tx;
        a = b = 0.f;
        if (r < N && c < N) load_x((size_t)r * N + c, a, b);
        xr_ji[y][tx] = a;
        xi_ji[y][tx] = b;
    }
    __shared__ float s_bound;
    __shared__ float eps_sh;
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        // both leapfrog chains are renormalised once every kRenormEvery steps
        const long long n = sc->step;
        eps_sh = (n % kRenormEvery) < 2 ? sc->eps_lvl[ops.base_slot] : 0.f;
        if (ops.dyn) {
            // |X| <= the sum of the maxima of its partial products
            const tc::DynScales* d = ops.dyn;
            float mre = 0.f, mim = 0.f;
            for (int q = 0; q < ops.nre; ++q) mre += (float)d->max_x[q];
            for (int q = 0; q < ops.nim; ++q) mim += (float)d->max_x[ops.nre + q];
            s_bound = pscale_f((float)d->max_drho[ops.base_slot] * (1.f + fabsf(eps_sh)) +
                               8.f * fabsf(eps_sh) +
                               fabsf((float)factor) * 2.0f * fmaxf(mre, mim));
        }
    }
    __syncthreads();
    const float op_scale = ops.dyn ? s_bound : ops.scale;
    const float eps = eps_sh;
    float dmax = 0.f;
    for (int half = 0; half < (bi == bj ? 1 : 2); ++half) {
        const int ti = half ? bj : bi, tj = half ? bi : bj;
        float brh[RPT], brl[RPT], bih[RPT], bil[RPT], sv[RPT], gv[RPT];
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int r = ti * kTile + ty + 8 * k, c = tj * kTile + tx;
            brh[k] = brl[k] = bih[k] = bil[k] = sv[k] = gv[k] = 0.f;
            if (r < N && c < N) {
                const size_t i = (size_t)r * N + c;
                brh[k] = base.re_hi[i];
                brl[k] = base.re_lo[i];
                bih[k] = base.im_hi[i];
                bil[k] = base.im_lo[i];
                sv[k] = Sf[i];
                if (eps != 0.f) gv[k] = rgs[i];
            }
        }
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int y = ty + 8 * k;
            const int r = ti * kTile + y, c = tj * kTile + tx;
            float2 pv = make_float2(0.f, 0.f);
            if (r < N && c < N) {
                float x_ij_re, x_ij_im, x_ji_re, x_ji_im;
                if (!half) {
                    x_ij_re = xr_ij[y][tx];
                    x_ij_im = xi_ij[y][tx];
                    x_ji_re = xr_ji[tx][y];
                    x_ji_im = xi_ji[tx][y];
                } else {
                    x_ij_re = xr_ji[y][tx];
                    x_ij_im = xi_ji[y][tx];
                    x_ji_re = xr_ij[tx][y];
                    x_ji_im = xi_ij[tx][y];
                }
                // rhodot = -i (X - X^dagger); the (j,i) element repeats these operations on
                // the swapped operands, so the master stays exactly Hermitian
                const float dre = x_ij_im + x_ji_im;
                const float dim = -(x_ij_re - x_ji_re);
                const float ire = fmaf(fh, dre, fl * dre);
                const float iim = fmaf(fh, dim, fl * dim);
                float rh = brh[k], rl = brl[k], ih = bih[k], il = bil[k];
                if (eps != 0.f) {
                    // renormalised base: f (rho_ref + dev) - rho_ref = dev + eps (rho_ref + dev)
                    df_add(rh, rl, eps * (gv[k] + rh));
                    df_add(ih, il, eps * ih);
                }
                df_add(rh, rl, ire);
                df_add(ih, il, iim);
                const size_t i = (size_t)r * N + c;
                out.re_hi[i] = rh;
                out.re_lo[i] = rl;
                out.im_hi[i] = ih;
                out.im_lo[i] = il;
                pv = mulliken_elem(rh, rl, sv[k]);
                if (ops.dyn) dmax = fmaxf(dmax, fmaxf(fabsf(rh), fabsf(ih)));
                if (ops.re[0]) {
                    // operands of the tensor-core products are K-major: Re rho is symmetric,
                    // the transpose of Im rho is -Im rho
                    const size_t jr = (size_t)r * ops.ld_re + c;
                    const size_t ji = (size_t)r * ops.ld_im + c;
                    if (ops.re[2]) {
                        uint16_t q[3];
                        split_head3(rh * op_scale, q);
                        ops.re[0][jr] = q[0];
                        ops.re[1][jr] = q[1];
                        ops.re[2][jr] = q[2];
                        split_head3(-ih * op_scale, q);
                        ops.im[0][ji] = q[0];
                        ops.im[1][ji] = q[1];
                        ops.im[2][ji] = q[2];
                    } else {
                        const float xa = rh * op_scale;
                        const uint16_t h1 = to16(xa, ops.bf16);
                        ops.re[0][jr] = h1;
                        ops.re[1][jr] = to16(xa - from16(h1, ops.bf16), ops.bf16);
                        const float yb = -ih * op_scale;
                        const uint16_t h2 = to16(yb, ops.bf16);
                        ops.im[0][ji] = h2;
                        ops.im[1][ji] = to16(yb - from16(h2, ops.bf16), ops.bf16);
                    }
                }
            }
            pv_s[y][tx] = pv;
        }
        __syncthreads();
        if (ty == 0) {
            const int r = ti * kTile + tx;
            const float2 sum = tile_row_sum(pv_s[tx]);
            if (r < N) const_cast<float2*>(lv.partial)[(size_t)r * nct + tj] = sum;
        }
        __syncthreads();
    }
    if (ops.dyn) {
        // one atomic per block (the warps' maxima through shared memory)
        __shared__ float wmax[8];
        for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        if (tx == 0) wmax[ty] = dmax;
        __syncthreads();
        if (tx == 0 && ty == 0) {
            for (int w = 1; w < 8; ++w) dmax = fmaxf(dmax, wmax[w]);
            atomicMax(reinterpret_cast<unsigned long long*>(&ops.dyn->max_drho[2]),
                      (unsigned long long)__double_as_longlong((double)dmax));
            if (bi == 0 && bj == 0) ops.dyn->s_rho = op_scale;
        }
    }
}

__global__ void __launch_bounds__(256, 4) k_update_df(UpdateDfArgs a) { update_df_block(a, blockIdx.x); }

__global__ void __launch_bounds__(256, 4)
    k_update_df_grouped(const UpdateDfArgs* __restrict__ args, const int2* __restrict__ work) {
    const int2 w = work[blockIdx.x];
    update_df_block(args[w.x], w.y);
}

// The charges of a level (after an update, or of the current level outside a step).
__global__ void __launch_bounds__(256) k_level_dq(LevelArgs lv) { level_dq_block(lv, blockIdx.x); }

__global__ void __launch_bounds__(256)
    k_level_dq_grouped(const LevelFinalArgs* __restrict__ args, const int2* __restrict__ work) {
    const int2 w = work[blockIdx.x];
    level_dq_block(args[w.x].lv, w.y);
}

// The potentials and scalars of a level after k_level_dq: after an update (step_end, the new
// level n + 1 in slot) or of the current level.
__global__ void __launch_bounds__(256) k_level_final(LevelArgs lv, int slot, int trace_only, int step_end) {
    const long long n_lvl = lv.sc->step + (step_end ? 1 : 0);
    level_final_block(lv, slot, n_lvl, trace_only != 0, step_end != 0, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(256)
    k_level_final_grouped(const LevelFinalArgs* __restrict__ args, const int2* __restrict__ work) {
    const int2 w = work[blockIdx.x];
    const LevelFinalArgs& f = args[w.x];
    const long long n_lvl = f.lv.sc->step + 1;
    level_final_block(f.lv, f.slot, n_lvl, false, true, w.y, level_blocks(f.lv.nat) + 1);
}

// FP64 populations from the (hi, lo) row partials of the deviation: one warp per atom
__global__ void k_charges_df(int nat, int nper, int nct, const float2* __restrict__ partial,
                             const double* __restrict__ qbase, const double* __restrict__ q0,
                             double* __restrict__ q, double* __restrict__ dq) {
    const int lane = threadIdx.x & 31;
    const int A = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (A >= nat) return;
    const float2* p = partial + (size_t)A * nper * nct;
    double s = 0.0;
    for (int i = lane; i < nper * nct; i += 32) s += (double)p[i].x + (double)p[i].y;
    s = warp_sum(s);
    if (lane == 0) {
        s += qbase[A];
        q[A] = s;
        dq[A] = s - q0[A];
    }
}

// master (hi, lo) of rho - rho_ref from the FP64 view
__global__ void k_view_to_master(size_t n, const double* __restrict__ rre,
                                 const double* __restrict__ rim, const double* __restrict__ ref,
                                 MasterPtrs m) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const double d = rre[i] - ref[i];
        const float h = (float)d;
        m.re_hi[i] = h;
        m.re_lo[i] = (float)(d - (double)h);
        const double e = rim[i];
        const float g = (float)e;
        m.im_hi[i] = g;
        m.im_lo[i] = (float)(e - (double)g);
    }
}

// FP64 view rho = rho_ref + hi + lo from the master
__global__ void k_master_to_view(size_t n, MasterPtrs m, const double* __restrict__ ref,
                                 double* __restrict__ rre, double* __restrict__ rim) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        rre[i] = ref[i] + ((double)m.re_hi[i] + (double)m.re_lo[i]);
        rim[i] = (double)m.im_hi[i] + (double)m.im_lo[i];
    }
}

// Mulliken row partials of the deviation held by the master, with the arithmetic of
// k_update_df (exact high products, FP32-pair sums in the same column order)
__global__ void k_master_partials(int N, int nct, MasterPtrs m, const float* __restrict__ Sf,
                                  float2* __restrict__ partial) {
    __shared__ float2 pv_s[kTile][kTile + 1];
    const int ct = blockIdx.x;
    const int col = ct * kTile + threadIdx.x;
    for (int y = threadIdx.y; y < kTile; y += blockDim.y) {
        const int row = blockIdx.y * kTile + y;
        float2 v = make_float2(0.f, 0.f);
        if (row < N && col < N) {
            const size_t i = (size_t)row * N + col;
            v = mulliken_elem(m.re_hi[i], m.re_lo[i], Sf[i]);
        }
        pv_s[y][threadIdx.x] = v;
    }
    __syncthreads();
    if (threadIdx.y == 0) {
        const int row = blockIdx.y * kTile + threadIdx.x;
        const float2 sum = tile_row_sum(pv_s[threadIdx.x]);
        if (row < N) partial[(size_t)row * nct + ct] = sum;
    }
}

// max(|re_hi|, |im_hi|) into out (out must start at 0)
__global__ void k_master_absmax(size_t n, MasterPtrs m, double* __restrict__ out) {
    float mx = 0.f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        mx = fmaxf(mx, fmaxf(fabsf(m.re_hi[i]), fabsf(m.im_hi[i])));
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0)
        atomicMax(reinterpret_cast<unsigned long long*>(out),
                  (unsigned long long)__double_as_longlong((double)mx));
}

// operand pieces of the master deviation (the update's arithmetic); the scale is
// pscale(*mx_exact) (FP16X6, exact maximum), else *dev_scale (FP16X6, restored), else
// the constant ops.scale
__global__ void k_master_pieces(int N, MasterPtrs m, UpdateOperands ops, const double* mx_exact,
                                const float* dev_scale) {
    __shared__ float s_sh;
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        s_sh = mx_exact ? tc::pscale(*mx_exact) : dev_scale ? *dev_scale : ops.scale;
        if (mx_exact && ops.dyn && blockIdx.x == 0 && blockIdx.y == 0) ops.dyn->s_rho = s_sh;
    }
    __syncthreads();
    const float sc = s_sh;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y * blockDim.y + threadIdx.y;
    if (r >= N || c >= N) return;
    const size_t i = (size_t)r * N + c;
    const float rh = m.re_hi[i], ih = m.im_hi[i];
    const size_t jr = (size_t)r * ops.ld_re + c;
    const size_t ji = (size_t)r * ops.ld_im + c;
    if (ops.re[2]) {
        uint16_t q[3];
        split_head3(rh * sc, q);
        ops.re[0][jr] = q[0];
        ops.re[1][jr] = q[1];
        ops.re[2][jr] = q[2];
        split_head3(-ih * sc, q);
        ops.im[0][ji] = q[0];
        ops.im[1][ji] = q[1];
        ops.im[2][ji] = q[2];
    } else {
        const float xa = rh * sc;
        const uint16_t h1 = to16(xa, ops.bf16);
        ops.re[0][jr] = h1;
        ops.re[1][jr] = to16(xa - from16(h1, ops.bf16), ops.bf16);
        const float yb = -ih * sc;
        const uint16_t h2 = to16(yb, ops.bf16);
        ops.im[0][ji] = h2;
        ops.im[1][ji] = to16(yb - from16(h2, ops.bf16), ops.bf16);
    }
}

}  // namespace

UpdateDfArgs update_df_args(const Ctx& c, const MasterPtrs& base, const MasterPtrs& out,
                            double factor, DevScalars* sc, const UpdateOperands& ops,
                            const LevelArgs& lv) {
    UpdateDfArgs a{};
    a.N = c.N;
    a.nct = c.nct;
    a.out_slot = out.re_hi == c.ms[0].re_hi ? 0 : 1;
    a.base = base;
    a.out = out;
    a.fh = (float)factor;
    a.fl = (float)(factor - (double)a.fh);
    a.factor = factor;
    a.Sf = c.S_f;
    a.rgs = c.rref_f;
    a.sc = sc;
    a.ops = ops;
    a.lv = lv;
    return a;
}

void launch_update_df(const Ctx& c, const MasterPtrs& base, const MasterPtrs& out, double factor,
                      DevScalars* sc, const UpdateOperands& ops, const LevelArgs& lv,
                      cudaStream_t st) {
    launch_pdl(k_update_df, dim3(c.nct * (c.nct + 1) / 2), dim3(kTile, 8), 0, st,
               update_df_args(c, base, out, factor, sc, ops, lv));
}

void launch_update_df_grouped(const UpdateDfArgs* args, const int2* work, int nwork,
                              cudaStream_t st) {
    launch_pdl(k_update_df_grouped, dim3(nwork), dim3(kTile, 8), 0, st, args, work);
}

void launch_level(const Ctx& c, const LevelArgs& lv, int slot, int trace_only, cudaStream_t st) {
    k_level_dq<<<level_blocks(c.nat), dim3(kTile, 8), 0, st>>>(lv);
    k_level_final<<<trace_only ? 1 : level_blocks(c.nat) + 1, dim3(kTile, 8), 0, st>>>(
        lv, slot, trace_only, 0);
}

void launch_level_dq(const Ctx& c, const LevelArgs& lv, cudaStream_t st) {
    launch_pdl(k_level_dq, dim3(level_blocks(c.nat)), dim3(kTile, 8), 0, st, lv);
}

void launch_level_dq_grouped(const LevelFinalArgs* args, const int2* work, int nwork,
                             cudaStream_t st) {
    launch_pdl(k_level_dq_grouped, dim3(nwork), dim3(kTile, 8), 0, st, args, work);
}

void launch_level_final(const Ctx& c, const LevelArgs& lv, int slot, cudaStream_t st) {
    launch_pdl(k_level_final, dim3(level_blocks(c.nat) + 1), dim3(kTile, 8), 0, st, lv, slot, 0, 1);
}

void launch_level_final_grouped(const LevelFinalArgs* args, const int2* work, int nwork,
                                cudaStream_t st) {
    launch_pdl(k_level_final_grouped, dim3(nwork), dim3(kTile, 8), 0, st, args, work);
}

void launch_charges_df(const Ctx& c, const float2* partial, double* q, double* dq, cudaStream_t st) {
    k_charges_df<<<(c.nat + 7) / 8, 256, 0, st>>>(c.nat, c.nper, c.nct, partial, c.qbase, c.d_q0, q,
                                                  dq);
}

void launch_view_to_master(const Ctx& c, const double* rre, const double* rim, const MasterPtrs& m,
                           cudaStream_t st) {
    k_view_to_master<<<1216, 256, 0, st>>>((size_t)c.N * c.N, rre, rim, c.rho_ref, m);
}

void launch_master_to_view(const Ctx& c, const MasterPtrs& m, double* rre, double* rim,
                           cudaStream_t st) {
    k_master_to_view<<<1216, 256, 0, st>>>((size_t)c.N * c.N, m, c.rho_ref, rre, rim);
}

void launch_master_partials(const Ctx& c, const MasterPtrs& m, float2* partial, cudaStream_t st) {
    dim3 b(kTile, 8);
    k_master_partials<<<dim3(c.nct, c.nct), b, 0, st>>>(c.N, c.nct, m, c.S_f, partial);
}

void launch_master_absmax(const Ctx& c, const MasterPtrs& m, double* out, cudaStream_t st) {
    k_master_absmax<<<608, 256, 0, st>>>((size_t)c.N * c.N, m, out);
}

void launch_master_pieces(const Ctx& c, const MasterPtrs& m, const UpdateOperands& ops,
                          const double* mx_exact, const float* dev_scale, cudaStream_t st) {
    dim3 b(32, 8);
    k_master_pieces<<<grid2(c.N, c.N, b), b, 0, st>>>(c.N, m, ops, mx_exact, dev_scale);
}

}  // namespace tdb
