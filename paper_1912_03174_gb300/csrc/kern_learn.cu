// The learned form: the per-atom shift network (forward, backward, Adam) and the
// closed-form leapfrog window with a frozen Hamiltonian.
//
// Network: y = w3 . tanh(W2^T tanh(W1^T x + b1) + b2) + b3 per sample, weights used in
// bfloat16 (rounded from FP32 masters when staged into shared memory), FP32
// accumulation.  Training minimises the mean squared error with Adam; the backward pass
// stages a block of 128 samples' activations in shared memory and forms the weight
// gradients as block-level sums (X^T dz1, h1^T dz2) added to the global gradient.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>

#include "tdb_internal.h"

namespace tdb {
namespace learn {
namespace {

constexpr int kBlockSamples = 128;

__device__ __forceinline__ float bf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Packed parameter offsets (W1 F x H, b1 H, W2 H x H, b2 H, w3 H, b3).
struct Layout {
    int F, H, oW1, ob1, oW2, ob2, ow3, ob3, n;
};
__host__ __device__ inline Layout layout(int F, int H) {
    Layout L;
    L.F = F;
    L.H = H;
    L.oW1 = 0;
    L.ob1 = F * H;
    L.oW2 = L.ob1 + H;
    L.ob2 = L.oW2 + H * H;
    L.ow3 = L.ob2 + H;
    L.ob3 = L.ow3 + H;
    L.n = L.ob3 + 1;
    return L;
}

// Stage the parameters into shared memory, weight matrices rounded to bfloat16.
__device__ void stage(const Layout& L, const float* __restrict__ p, float* s) {
    for (int i = threadIdx.x; i < L.n; i += blockDim.x) {
        const bool weight = i < L.ob1 || (i >= L.oW2 && i < L.ob2) || (i >= L.ow3 && i < L.ob3);
        s[i] = weight ? bf(p[i]) : p[i];
    }
}

__global__ void k_net_forward(int F, int H, const float* __restrict__ params,
                              const float* __restrict__ X, long n, float* __restrict__ Y) {
    extern __shared__ float sp[];
    const Layout L = layout(F, H);
    stage(L, params, sp);
    __syncthreads();
    const long s = static_cast<long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float h1[64];
    const float* x = X + s * F;
    for (int j = 0; j < H; ++j) {
        float z = sp[L.ob1 + j];
        for (int f = 0; f < F; ++f) z = fmaf(x[f], sp[L.oW1 + f * H + j], z);
        h1[j] = tanhf(z);
    }
    float y = sp[L.ob3];
    for (int j = 0; j < H; ++j) {
        float z = sp[L.ob2 + j];
        for (int i = 0; i < H; ++i) z = fmaf(h1[i], sp[L.oW2 + i * H + j], z);
        y = fmaf(tanhf(z), sp[L.ow3 + j], y);
    }
    Y[s] = y;
}

// Gradient of the mean squared error over n samples (scale = 1 / n), added to grad;
// the sum of squared residuals is added to *sse.
__global__ void __launch_bounds__(256)
    k_net_grad(int F, int H, const float* __restrict__ params, const float* __restrict__ X,
               const float* __restrict__ Y, long n, float scale, float* __restrict__ grad,
               double* __restrict__ sse) {
    extern __shared__ float sm[];
    const Layout L = layout(F, H);
    // per-sample rows padded by one float against bank conflicts
    const int FS = F + 1, HS = H + 1;
    float* sp = sm;                                   // parameters
    float* sx = sp + ((L.n + 31) & ~31);              // X block   [128][F + 1]
    float* sh1 = sx + kBlockSamples * FS;             // h1        [128][H + 1]
    float* sd1 = sh1 + kBlockSamples * HS;            // dz1       [128][H + 1]
    float* sd2 = sd1 + kBlockSamples * HS;            // dz2       [128][H + 1]
    float* sb = sd2 + kBlockSamples * HS;             // b1, b2, w3 grads, b3, sse [3H + 2]
    stage(L, params, sp);
    for (int i = threadIdx.x; i < 3 * H + 2; i += blockDim.x) sb[i] = 0.f;
    __syncthreads();
    const long s0 = static_cast<long>(blockIdx.x) * kBlockSamples;
    const int t = threadIdx.x;
    if (t < kBlockSamples) {
        const long s = s0 + t;
        float* xs = sx + t * FS;
        float* h1 = sh1 + t * HS;
        float* d1 = sd1 + t * HS;
        float* d2 = sd2 + t * HS;
        if (s < n) {
            for (int f = 0; f < F; ++f) xs[f] = X[s * F + f];
            for (int j = 0; j < H; ++j) {
                float z = sp[L.ob1 + j];
                for (int f = 0; f < F; ++f) z = fmaf(xs[f], sp[L.oW1 + f * H + j], z);
                h1[j] = tanhf(z);
            }
            // h2 is kept in d2 until dz2 replaces it
            float y = sp[L.ob3];
            for (int j = 0; j < H; ++j) {
                float z = sp[L.ob2 + j];
                for (int i = 0; i < H; ++i) z = fmaf(h1[i], sp[L.oW2 + i * H + j], z);
                d2[j] = tanhf(z);
                y = fmaf(d2[j], sp[L.ow3 + j], y);
            }
            const float r = y - Y[s];
            const float dy = 2.f * r * scale;
            atomicAdd(&sb[3 * H], dy);                 // b3
            atomicAdd(&sb[3 * H + 1], r * r);          // squared residual
            for (int j = 0; j < H; ++j) {
                const float h2 = d2[j];
                atomicAdd(&sb[2 * H + j], h2 * dy);    // w3
                d2[j] = dy * sp[L.ow3 + j] * (1.f - h2 * h2);
                atomicAdd(&sb[H + j], d2[j]);          // b2
            }
            for (int i = 0; i < H; ++i) {
                float g = 0.f;
                for (int j = 0; j < H; ++j) g = fmaf(d2[j], sp[L.oW2 + i * H + j], g);
                d1[i] = g * (1.f - h1[i] * h1[i]);
                atomicAdd(&sb[i], d1[i]);              // b1
            }
        } else {
            for (int f = 0; f < F; ++f) xs[f] = 0.f;
            for (int j = 0; j < H; ++j) h1[j] = d1[j] = d2[j] = 0.f;
        }
    }
    __syncthreads();
    // W1 = X^T dz1 and W2 = h1^T dz2 over the block's samples
    for (int e = t; e < F * H + H * H; e += blockDim.x) {
        float g = 0.f;
        if (e < F * H) {
            const int f = e / H, j = e % H;
            for (int q = 0; q < kBlockSamples; ++q) g = fmaf(sx[q * FS + f], sd1[q * HS + j], g);
            atomicAdd(&grad[L.oW1 + e], g);
        } else {
            const int e2 = e - F * H, i = e2 / H, j = e2 % H;
            for (int q = 0; q < kBlockSamples; ++q) g = fmaf(sh1[q * HS + i], sd2[q * HS + j], g);
            atomicAdd(&grad[L.oW2 + e2], g);
        }
    }
    for (int j = t; j < H; j += blockDim.x) {
        atomicAdd(&grad[L.ob1 + j], sb[j]);
        atomicAdd(&grad[L.ob2 + j], sb[H + j]);
        atomicAdd(&grad[L.ow3 + j], sb[2 * H + j]);
    }
    if (t == 0) {
        atomicAdd(&grad[L.ob3], sb[3 * H]);
        atomicAdd(sse, static_cast<double>(sb[3 * H + 1]));
    }
}

__global__ void k_adam(int n, float* __restrict__ p, const float* __restrict__ g,
                       float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2,
                       float c1, float c2, float eps) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    m[i] = b1 * m[i] + (1.f - b1) * g[i];
    v[i] = b2 * v[i] + (1.f - b2) * g[i] * g[i];
    p[i] -= lr * (m[i] / c1) / (sqrtf(v[i] / c2) + eps);
}

// Closed-form leapfrog window in the eigenbasis: for element (a, b), theta = (e_a - e_b) dt,
// the leapfrog modes are l+ = exp(-i phi), l- = -exp(i phi) with phi = asin(theta);
// (x0, x1) = (x_{n-1}, x_n) -> (x_{n-1+k}, x_{n+k}).
__global__ void k_window(int N, const double* __restrict__ eps, double dt, int k,
                         double* __restrict__ x0re, double* __restrict__ x0im,
                         double* __restrict__ x1re, double* __restrict__ x1im) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    const int a = blockIdx.y * blockDim.y + threadIdx.y;
    if (a >= N || b >= N) return;
    const size_t i = static_cast<size_t>(a) * N + b;
    const double th = (eps[a] - eps[b]) * dt;
    const double c = sqrt(1.0 - th * th);
    const double phi = asin(th);
    // A = (x1 - l- x0) / (2c), l- = (-c, -th);  B = x0 - A
    const double lmr = -c, lmi = -th;
    const double ar = (x1re[i] - (lmr * x0re[i] - lmi * x0im[i])) / (2.0 * c);
    const double ai = (x1im[i] - (lmr * x0im[i] + lmi * x0re[i])) / (2.0 * c);
    const double br = x0re[i] - ar, bi = x0im[i] - ai;
    double out[2][2];
    for (int q = 0; q < 2; ++q) {
        const int m = k + q;
        double sn, cs;
        sincos(m * phi, &sn, &cs);
        const double sg = (m & 1) ? -1.0 : 1.0;
        // l+^m = (cs, -sn), l-^m = sg (cs, sn)
        out[q][0] = (ar * cs + ai * sn) + sg * (br * cs - bi * sn);
        out[q][1] = (ai * cs - ar * sn) + sg * (bi * cs + br * sn);
    }
    x0re[i] = out[0][0];
    x0im[i] = out[0][1];
    x1re[i] = out[1][0];
    x1im[i] = out[1][1];
}

__global__ void k_add_step(DevScalars* sc, int k) {
    if (threadIdx.x == 0 && blockIdx.x == 0) sc->step += k;
}

}  // namespace

int n_params(int F, int H) { return layout(F, H).n; }

size_t grad_smem(int F, int H) {
    const Layout L = layout(F, H);
    return sizeof(float) * (((L.n + 31) & ~31) + kBlockSamples * (F + 1) +
                            3 * kBlockSamples * (H + 1) + 3 * H + 2);
}

// The attributes are set for the largest network (32 features, 64 hidden), so that
// networks of different sizes can live side by side.
cudaError_t prepare(int, int) {
    cudaError_t e = cudaFuncSetAttribute(k_net_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(grad_smem(32, 64)));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_net_forward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(sizeof(float) * layout(32, 64).n));
    return e;
}

void launch_forward(int F, int H, const float* params, const float* X, long n, float* Y,
                    cudaStream_t st) {
    const int blocks = static_cast<int>((n + 127) / 128);
    k_net_forward<<<blocks, 128, sizeof(float) * layout(F, H).n, st>>>(F, H, params, X, n, Y);
}

void launch_grad(int F, int H, const float* params, const float* X, const float* Y, long n,
                 float scale, float* grad, double* sse, cudaStream_t st) {
    const int blocks = static_cast<int>((n + kBlockSamples - 1) / kBlockSamples);
    k_net_grad<<<blocks, 256, grad_smem(F, H), st>>>(F, H, params, X, Y, n, scale, grad, sse);
}

void launch_adam(int n, float* p, const float* g, float* m, float* v, float lr, float b1,
                 float b2, float c1, float c2, float eps, cudaStream_t st) {
    k_adam<<<(n + 255) / 256, 256, 0, st>>>(n, p, g, m, v, lr, b1, b2, c1, c2, eps);
}

void launch_window(int N, const double* eps, double dt, int k, double* x0re, double* x0im,
                   double* x1re, double* x1im, cudaStream_t st) {
    dim3 b(32, 8);
    dim3 g((N + 31) / 32, (N + 7) / 8);
    k_window<<<g, b, 0, st>>>(N, eps, dt, k, x0re, x0im, x1re, x1im);
}

void launch_add_step(DevScalars* sc, int k, cudaStream_t st) { k_add_step<<<1, 32, 0, st>>>(sc, k); }

}  // namespace learn
}  // namespace tdb
