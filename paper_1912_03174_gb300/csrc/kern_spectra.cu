// Damped one-sided Fourier transforms of sampled dipole signals: the transforms behind the
// absorption cross section (eq:alpha, eq:sigma, Sec. 2.2) and the transient absorption of
// pump-probe runs (eq:alphaeff, eq:sigmaeff, Sec. 3.2):
//
//   F_s(w) = dt sum_{n < K} x_s[n] exp(-n dt / t_damp) exp(+i w n dt).
//
// FP64.  One thread per frequency and eight signals per block (blockIdx.y): the twiddle of a
// frequency is shared by the eight signals, whose samples are staged through shared memory
// (every thread reads the same address: broadcast).  The twiddle exp((i w - 1/t_damp) n dt)
// is evaluated exactly (sincos, exp) every 32 samples and advanced by the one-step factor in
// between, which keeps its error at a few tens of ulps.
#include <cmath>
#include <vector>

#include "tdb_internal.h"

namespace tdb {
void set_last_error(const char* msg);
}

namespace {

constexpr int kFreqs = 128;   // frequencies (threads) per block
constexpr int kSigs = 8;      // signals per block
constexpr int kSamp = 256;    // samples staged per pass
constexpr int kExact = 32;    // samples between exact twiddles

__global__ void __launch_bounds__(kFreqs)
    k_damped_transform(int nsig, long long K, const double* __restrict__ x, double dt,
                       double inv_td, int nw, const double* __restrict__ omega,
                       double* __restrict__ re, double* __restrict__ im) {
    __shared__ double xs[kSigs][kSamp];
    const int k = blockIdx.x * kFreqs + threadIdx.x;
    const int s0 = blockIdx.y * kSigs;
    const double w = k < nw ? omega[k] : 0.0;
    double sw, cw;
    sincos(w * dt, &sw, &cw);
    const double r1 = exp(-dt * inv_td);
    const double c1 = r1 * cw, s1 = r1 * sw;
    double ar[kSigs], ai[kSigs];
#pragma unroll
    for (int s = 0; s < kSigs; ++s) ar[s] = ai[s] = 0.0;
    for (long long n0 = 0; n0 < K; n0 += kSamp) {
        __syncthreads();
        for (int i = threadIdx.x; i < kSigs * kSamp; i += kFreqs) {
            const int s = i / kSamp;
            const long long n = n0 + i % kSamp;
            xs[s][i % kSamp] = (s0 + s < nsig && n < K) ? x[(size_t)(s0 + s) * K + n] : 0.0;
        }
        __syncthreads();
        const int len = (int)(K - n0 < kSamp ? K - n0 : kSamp);
        for (int b = 0; b < len; b += kExact) {
            const double t = (double)(n0 + b) * dt;
            double sn, cn;
            sincos(w * t, &sn, &cn);
            const double d = exp(-t * inv_td);
            double tr = d * cn, ti = d * sn;
            const int e = len - b < kExact ? len - b : kExact;
            for (int j = 0; j < e; ++j) {
#pragma unroll
                for (int s = 0; s < kSigs; ++s) {
                    const double v = xs[s][b + j];
                    ar[s] = fma(v, tr, ar[s]);
                    ai[s] = fma(v, ti, ai[s]);
                }
                const double nr = tr * c1 - ti * s1;
                ti = fma(tr, s1, ti * c1);
                tr = nr;
            }
        }
    }
    if (k >= nw) return;
#pragma unroll
    for (int s = 0; s < kSigs; ++s)
        if (s0 + s < nsig) {
            re[(size_t)(s0 + s) * nw + k] = dt * ar[s];
            im[(size_t)(s0 + s) * nw + k] = dt * ai[s];
        }
}

tdb_status fail(tdb_status st, const char* msg) {
    tdb::set_last_error(msg);
    return st;
}

}  // namespace

extern "C" tdb_status tdb_damped_transform(int nsig, long K, const double* x, double dt,
                                           double t_damp, int nw, const double* omega, double* re,
                                           double* im) {
    if (nsig < 1 || K < 1 || nw < 1 || !x || !omega || !re || !im || !std::isfinite(dt) ||
        !(dt > 0) || std::isnan(t_damp) || t_damp < 0 || nsig > 65535 * kSigs)
        return fail(TDB_ERR_ARG, "tdb_damped_transform: invalid sizes, pointers, dt or t_damp");
    for (int k = 0; k < nw; ++k)
        if (!std::isfinite(omega[k]))
            return fail(TDB_ERR_ARG, "tdb_damped_transform: non-finite frequency");
    const double inv_td = (t_damp == 0.0 || std::isinf(t_damp)) ? 0.0 : 1.0 / t_damp;
    double *dx = nullptr, *dw = nullptr, *dre = nullptr, *dim = nullptr;
    const size_t nx = (size_t)nsig * (size_t)K, no = (size_t)nsig * (size_t)nw;
    tdb_status rc = TDB_OK;
    cudaStream_t st = nullptr;
    auto ok = [&](cudaError_t e) {
        if (e != cudaSuccess && rc == TDB_OK) rc = e == cudaErrorMemoryAllocation ? TDB_ERR_NOMEM : TDB_ERR_CUDA;
        return e == cudaSuccess;
    };
    ok(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    ok(cudaMalloc(&dx, sizeof(double) * nx));
    ok(cudaMalloc(&dw, sizeof(double) * nw));
    ok(cudaMalloc(&dre, sizeof(double) * no));
    ok(cudaMalloc(&dim, sizeof(double) * no));
    if (rc == TDB_OK) {
        ok(cudaMemcpyAsync(dx, x, sizeof(double) * nx, cudaMemcpyHostToDevice, st));
        ok(cudaMemcpyAsync(dw, omega, sizeof(double) * nw, cudaMemcpyHostToDevice, st));
        dim3 grid((nw + kFreqs - 1) / kFreqs, (nsig + kSigs - 1) / kSigs);
        k_damped_transform<<<grid, kFreqs, 0, st>>>(nsig, (long long)K, dx, dt, inv_td, nw, dw, dre,
                                                    dim);
        ok(cudaGetLastError());
        ok(cudaMemcpyAsync(re, dre, sizeof(double) * no, cudaMemcpyDeviceToHost, st));
        ok(cudaMemcpyAsync(im, dim, sizeof(double) * no, cudaMemcpyDeviceToHost, st));
        ok(cudaStreamSynchronize(st));
    }
    cudaFree(dx);
    cudaFree(dw);
    cudaFree(dre);
    cudaFree(dim);
    if (st) cudaStreamDestroy(st);
    if (rc != TDB_OK) tdb::set_last_error("tdb_damped_transform: a CUDA call failed");
    return rc;
}
