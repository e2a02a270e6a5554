// The learned form: the per-atom shift network (forward, backward, Adam) and the
// closed-form leapfrog window with a frozen Hamiltonian.
//
// Network: y = w3 . tanh(W2^T tanh(W1^T x + b1) + b2) + b3 per sample, weights used in
// bfloat16 (rounded from FP32 masters when staged into shared memory), FP32
// accumulation.  Training minimises the mean squared error with Adam; the backward pass
// keeps a block of 128 samples' activations in shared memory and forms the weight
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
// the sum of squared residuals is added to *sse.  One block takes 128 samples and works
// layer by layer, all threads on each layer's 128 x H outputs (one sample's row is read
// as a broadcast, the weights along consecutive columns); W2 is staged with rows padded
// to H + 1 so that its transposed use in the backward pass is conflict-free too.  The
// weight and bias gradients are the block's column sums, one global atomic per element.
// Rows past n carry x = 0 and dy = 0, so they add nothing.
__global__ void __launch_bounds__(256)
    k_net_grad(int F, int H, const float* __restrict__ params, const float* __restrict__ X,
               const float* __restrict__ Y, long n, float scale, float* __restrict__ grad,
               double* __restrict__ sse) {
    extern __shared__ float sm[];
    const Layout L = layout(F, H);
    const int FS = F + 1, HS = H + 1, t = threadIdx.x, nt = blockDim.x;
    constexpr int S = kBlockSamples;
    float* sW1 = sm;                        // F x H
    float* sb1 = sW1 + F * H;               // H
    float* sW2 = sb1 + H;                   // H x (H + 1)
    float* sb2 = sW2 + H * HS;              // H
    float* sw3 = sb2 + H;                   // H
    float* sx = sw3 + H + 1;                // [S][F + 1]   (b3 sits at sw3[H])
    float* sh1 = sx + S * FS;               // [S][H + 1]
    float* sh2 = sh1 + S * HS;              // [S][H + 1]
    float* sd1 = sh2 + S * HS;              // [S][H + 1]
    float* sd2 = sd1 + S * HS;              // [S][H + 1]
    float* sdy = sd2 + S * HS;              // [S]
    float* sr2 = sdy + S;                   // [S] squared residuals
    for (int i = t; i < F * H; i += nt) sW1[i] = bf(params[L.oW1 + i]);
    for (int i = t; i < H * H; i += nt) sW2[(i / H) * HS + i % H] = bf(params[L.oW2 + i]);
    for (int i = t; i < H; i += nt) {
        sb1[i] = params[L.ob1 + i];
        sb2[i] = params[L.ob2 + i];
        sw3[i] = bf(params[L.ow3 + i]);
    }
    if (t == 0) sw3[H] = params[L.ob3];
    const long s0 = static_cast<long>(blockIdx.x) * S;
    for (int e = t; e < S * F; e += nt) {
        const int q = e / F, f = e % F;
        sx[q * FS + f] = s0 + q < n ? X[(s0 + q) * F + f] : 0.f;
    }
    __syncthreads();
    // h1 = tanh(x W1 + b1)
    for (int e = t; e < S * H; e += nt) {
        const int q = e / H, j = e % H;
        float z = sb1[j];
        for (int f = 0; f < F; ++f) z = fmaf(sx[q * FS + f], sW1[f * H + j], z);
        sh1[q * HS + j] = tanhf(z);
    }
    __syncthreads();
    // h2 = tanh(h1 W2 + b2)
    for (int e = t; e < S * H; e += nt) {
        const int q = e / H, j = e % H;
        float z = sb2[j];
        for (int i = 0; i < H; ++i) z = fmaf(sh1[q * HS + i], sW2[i * HS + j], z);
        sh2[q * HS + j] = tanhf(z);
    }
    __syncthreads();
    // y = h2 w3 + b3, dy = 2 (y - Y) / n
    for (int q = t; q < S; q += nt) {
        float y = sw3[H];
        for (int j = 0; j < H; ++j) y = fmaf(sh2[q * HS + j], sw3[j], y);
        const bool ok = s0 + q < n;
        const float r = ok ? y - Y[s0 + q] : 0.f;
        sdy[q] = 2.f * r * scale;
        sr2[q] = r * r;
    }
    __syncthreads();
    // dz2 = dy w3 (1 - h2^2)
    for (int e = t; e < S * H; e += nt) {
        const int q = e / H, j = e % H;
        const float h2 = sh2[q * HS + j];
        sd2[q * HS + j] = sdy[q] * sw3[j] * (1.f - h2 * h2);
    }
    __syncthreads();
    // dz1 = (dz2 W2^T) (1 - h1^2)
    for (int e = t; e < S * H; e += nt) {
        const int q = e / H, i = e % H;
        float g = 0.f;
        for (int j = 0; j < H; ++j) g = fmaf(sd2[q * HS + j], sW2[i * HS + j], g);
        const float h1 = sh1[q * HS + i];
        sd1[q * HS + i] = g * (1.f - h1 * h1);
    }
    __syncthreads();
    // column sums over the block's samples
    const int nW1 = F * H, nW2 = H * H;
    for (int e = t; e < nW1 + nW2 + 3 * H + 1; e += nt) {
        float g = 0.f;
        int dst;
        if (e < nW1) {
            const int f = e / H, j = e % H;
            for (int q = 0; q < S; ++q) g = fmaf(sx[q * FS + f], sd1[q * HS + j], g);
            dst = L.oW1 + e;
        } else if (e < nW1 + nW2) {
            const int e2 = e - nW1, i = e2 / H, j = e2 % H;
            for (int q = 0; q < S; ++q) g = fmaf(sh1[q * HS + i], sd2[q * HS + j], g);
            dst = L.oW2 + e2;
        } else {
            const int e3 = e - nW1 - nW2, j = e3 % H;
            if (e3 < H) {                       // b1
                for (int q = 0; q < S; ++q) g += sd1[q * HS + j];
                dst = L.ob1 + j;
            } else if (e3 < 2 * H) {            // b2
                for (int q = 0; q < S; ++q) g += sd2[q * HS + j];
                dst = L.ob2 + j;
            } else if (e3 < 3 * H) {            // w3
                for (int q = 0; q < S; ++q) g = fmaf(sh2[q * HS + j], sdy[q], g);
                dst = L.ow3 + j;
            } else {                            // b3
                for (int q = 0; q < S; ++q) g += sdy[q];
                dst = L.ob3;
            }
        }
        atomicAdd(&grad[dst], g);
    }
    if (t < 32) {
        float r2 = 0.f;
        for (int q = t; q < S; q += 32) r2 += sr2[q];
        for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
        if (t == 0) atomicAdd(sse, static_cast<double>(r2));
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
    return sizeof(float) * (F * H + H + H * (H + 1) + 3 * H + 1 + kBlockSamples * (F + 1) +
                            4 * kBlockSamples * (H + 1) + 2 * kBlockSamples);
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
