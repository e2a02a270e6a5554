// SIMT matrix products (row-major C = A B).  FP64 (DFMA) for the FP64 form of
// the propagator and for the setup; FP32 (FFMA) for the TDB_FP32 form.  The
// B operand can be formed while it is loaded (the SCC Hamiltonian of eq:hscc,
// H_kj = H0_kj + 1/2 S_kj (v_k + v_j)), so H is never stored.
#include "tdb_internal.h"

namespace tdb {

namespace {

template <typename T>
struct Dense {
    const T* p;
    int ld;
    __device__ __forceinline__ T operator()(int r, int c) const { return p[(size_t)r * ld + c]; }
};

// H_kj = H0_kj + 1/2 S_kj (v_k + v_j)
struct Ham {
    const double *H0, *S, *v;
    int N;
    __device__ __forceinline__ double operator()(int k, int j) const {
        const size_t i = (size_t)k * N + j;
        return H0[i] + 0.5 * S[i] * (v[k] + v[j]);
    }
};

// delta H_kj = 1/2 S_kj (dv_k + dv_j) in FP32
struct DeltaHamF {
    const float *S, *dv;
    int N;
    __device__ __forceinline__ float operator()(int k, int j) const {
        return 0.5f * S[(size_t)k * N + j] * (dv[k] + dv[j]);
    }
};

// C[BM x BN] tile per block; each thread owns TM x TN outputs strided by the
// thread-grid size, so shared-memory reads of a warp are conflict-free.
template <typename T, int BM, int BN, int BK, int TM, int TN, class LA, class LB>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    k_gemm(int M, int Ncol, int K, LA la, LB lb, T* C, int ldc,
           const T* Cadd) {
    constexpr int TX = BN / TN, TY = BM / TM, NT = TX * TY;
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN];
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
    for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
        for (int e = tid; e < BM * BK; e += NT) {
            const int m = e / BK, k = e % BK;
            const int gm = m0 + m, gk = k0 + k;
            As[k][m] = (gm < M && gk < K) ? la(gm, gk) : T(0);
        }
#pragma unroll
        for (int e = tid; e < BK * BN; e += NT) {
            const int k = e / BN, n = e % BN;
            const int gk = k0 + k, gn = n0 + n;
            Bs[k][n] = (gk < K && gn < Ncol) ? lb(gk, gn) : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + i * TY];
#pragma unroll
            for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + j * TX];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int gm = m0 + ty + i * TY;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int gn = n0 + tx + j * TX;
            if (gn < Ncol) {
                const size_t o = (size_t)gm * ldc + gn;
                C[o] = Cadd ? acc[i][j] + Cadd[o] : acc[i][j];
            }
        }
    }
}

template <class LA, class LB>
void run_f64(int M, int Ncol, int K, LA la, LB lb, double* C, int ldc, const double* Cadd,
             cudaStream_t st) {
    constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;
    dim3 g((Ncol + BN - 1) / BN, (M + BM - 1) / BM);
    k_gemm<double, BM, BN, BK, TM, TN, LA, LB>
        <<<g, (BM / TM) * (BN / TN), 0, st>>>(M, Ncol, K, la, lb, C, ldc, Cadd);
}

template <class LA, class LB>
void run_f32(int M, int Ncol, int K, LA la, LB lb, float* C, int ldc, const float* Cadd,
             cudaStream_t st) {
    constexpr int BM = 128, BN = 128, BK = 8, TM = 8, TN = 8;
    dim3 g((Ncol + BN - 1) / BN, (M + BM - 1) / BM);
    k_gemm<float, BM, BN, BK, TM, TN, LA, LB>
        <<<g, (BM / TM) * (BN / TN), 0, st>>>(M, Ncol, K, la, lb, C, ldc, Cadd);
}

}  // namespace

void gemm_f64(int M, int Ncol, int K, const double* A, int lda, const double* B, int ldb,
              double* C, int ldc, cudaStream_t st) {
    run_f64(M, Ncol, K, Dense<double>{A, lda}, Dense<double>{B, ldb}, C, ldc, nullptr, st);
}

void gemm_f64_ham(int N, const double* A, const double* H0, const double* S, const double* v_orb,
                  double* C, cudaStream_t st) {
    run_f64(N, N, N, Dense<double>{A, N}, Ham{H0, S, v_orb, N}, C, N, nullptr, st);
}

void gemm_f32(int M, int Ncol, int K, const float* A, int lda, const float* B, int ldb, float* C,
              int ldc, cudaStream_t st) {
    run_f32(M, Ncol, K, Dense<float>{A, lda}, Dense<float>{B, ldb}, C, ldc, nullptr, st);
}

// C = A * dH + Cadd, dH_kj = 1/2 S_kj (dv_k + dv_j): delta M = S^-1 delta H, M = M_gs + delta M
void gemm_f32_dham(int N, const float* A, const float* S, const float* dv, float* C, int ldc,
                   const float* Cadd, cudaStream_t st) {
    run_f32(N, N, N, Dense<float>{A, N}, DeltaHamF{S, dv, N}, C, ldc, Cadd, st);
}

// C = A * B + Cadd (FP32; Cadd may be C itself)
void gemm_f32_add(int M, int Ncol, int K, const float* A, int lda, const float* B, int ldb,
                  float* C, int ldc, const float* Cadd, cudaStream_t st) {
    run_f32(M, Ncol, K, Dense<float>{A, lda}, Dense<float>{B, ldb}, C, ldc, Cadd, st);
}

}  // namespace tdb
