// Integer-slice GEMM on the tcgen05 tensor cores (see tdb_oz.h for the arithmetic).
//
// Data path per 128 x 64 output tile: TMA loads the kSlices slices of A and of B^T for
// a 32-deep K block into a 3-stage shared-memory ring; one thread issues the 21 slice
// products (pairs s + t < kSlices) of each 16-deep step as 8 MMAs of N <= 256 into
// kSlices TMEM accumulators, one per weight w = s + t; after every kChunk of K the
// eight drain warps move the (exact, integer-valued) accumulators into 64-bit integer
// sums in registers and hand the TMEM back; the last drain writes FP64 C with the row
// and column scales.  All waits are bounded; a time-out records an error code and the
// kernel frees its TMEM and returns.
#include <cuda.h>
#include <cuda_fp16.h>

#include <cstdint>

#include "tc_ptx.cuh"
#include "tdb_oz.h"
#include "tdb_tc.h"

namespace tdb {
namespace oz {

namespace {
using namespace tc::ptx;

constexpr int BM = 128, BN = 64, BK = 32;
constexpr int kThreads = 384;                 // warps 0-3: TMA, MMA, TMEM; 4-11: drain
constexpr int kChunkKB = kChunk / BK;         // K blocks per exact chunk
constexpr int A_TILE = BM * BK * 2;           // 8 KiB per A slice
constexpr int B_TILE = BN * BK * 2;           // 4 KiB per B slice
constexpr int SB = kSlices * (A_TILE + B_TILE);
constexpr int STAGES = 3;
constexpr int SMEM = STAGES * SB + 1024 + 256;
constexpr uint32_t TMEM_COLS = 512;           // kSlices x BN = 384 used

static_assert(kSlices * BN <= 512, "accumulators must fit in TMEM");
static_assert(SMEM <= 227 * 1024, "shared memory");
static_assert((kSlices) * kChunk * 64 * 64 < (1 << 24), "chunk sums must stay exact in FP32");

struct Maps {
    CUtensorMap a[kSlices];
    CUtensorMap b[2][kSlices];
};

struct Params {
    int M, N, K;
    const int* ea;
    const int* eb[2];
    double* C[2];
    int ldc[2];
    int* err;
    uint32_t idesc[5];   // [nb]: instruction descriptor of an N = 64 nb product
};

// One CTA per 128 x 64 output tile; every CTA issues its own TMA loads of the A and B
// slices it multiplies.
__global__ void __launch_bounds__(kThreads, 1)
    k_oz_gemm(const __grid_constant__ Maps maps, Params p) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* gbase = smem_raw + (base - raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + STAGES * SB);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 2);
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES);
    const uint32_t cfull = smem_u32(bars + 2 * STAGES), cempty = smem_u32(bars + 2 * STAGES + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int z = blockIdx.z;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int nkb = (p.K + BK - 1) / BK;
    const int nchunk = (nkb + kChunkKB - 1) / kChunkKB;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(cfull, 1);
        mbar_init(cempty, 8);   // one arrival per drain warp
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        fence_before();
    }
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // TMA producer: the kSlices slices of A, then of B^T, of one K block per stage
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % STAGES, round = kb / STAGES;
                if (kb >= STAGES && !mbar_wait(empty0 + 8 * s, (round - 1) & 1, p.err, 1)) break;
                const uint32_t st = base + s * SB, fb = full0 + 8 * s;
                mbar_expect_tx(fb, SB);
#pragma unroll
                for (int q = 0; q < kSlices; ++q) {
                    tma_load_2d(st + q * A_TILE, &maps.a[q], kb * BK, m0, fb);
                    tma_load_2d(st + kSlices * A_TILE + q * B_TILE, &maps.b[z][q], kb * BK, n0, fb);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % STAGES, round = kb / STAGES;
                const int c = kb / kChunkKB;
                const bool first = (kb % kChunkKB) == 0;
                // a new chunk overwrites the accumulators once the previous one is drained
                if (first && c > 0 && !mbar_wait(cempty, (c - 1) & 1, p.err, 2)) break;
                if (!mbar_wait(full0 + 8 * s, round & 1, p.err, 2)) break;
                fence_after();
                const uint32_t st = base + s * SB;
#pragma unroll
                for (int k = 0; k < BK / 16; ++k) {
                    uint64_t a[kSlices], b[kSlices];
#pragma unroll
                    for (int q = 0; q < kSlices; ++q) {
                        a[q] = sdesc(st + q * A_TILE + k * 32);
                        b[q] = sdesc(st + kSlices * A_TILE + q * B_TILE + k * 32);
                    }
                    // pair (sa, tb) into the accumulator of weight sa + tb.  The B slices lie
                    // one after another in shared memory and the accumulators by weight in
                    // TMEM, so one MMA of N = 64 nb takes the pairs (sa, tb .. tb + nb - 1)
                    // into the accumulators sa + tb .. sa + tb + nb - 1: 8 MMAs (N <= 256)
                    // instead of 21.  The sa = 0 products of a chunk's first step cover every
                    // accumulator and start them afresh.
#pragma unroll
                    for (int sa = 0; sa < kSlices; ++sa)
#pragma unroll
                        for (int tb = 0; sa + tb < kSlices; tb += 4) {
                            const int nb = kSlices - sa - tb < 4 ? kSlices - sa - tb : 4;
                            mma_f16(tmem + static_cast<uint32_t>((sa + tb) * BN), a[sa], b[tb],
                                    p.idesc[nb], (first && k == 0 && sa == 0) ? 0u : 1u);
                        }
                }
                // free the stage for a refill (none follows the last STAGES blocks, so no
                // arrival is left in flight when the CTA exits)
                if (kb + STAGES < nkb) mma_commit(empty0 + 8 * s);
                if ((kb % kChunkKB) == kChunkKB - 1 || kb == nkb - 1) mma_commit(cfull);
            }
        }
    } else if (warp >= 4) {
        // drain warps: TMEM lane quarter (warp % 4) and 32-column half (warp - 4) / 4
        const int quarter = warp & 3, half = (warp - 4) >> 2;
        const int row = m0 + quarter * 32 + lane;
        const uint32_t lane_off = static_cast<uint32_t>(quarter * 32) << 16;
        long long T[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) T[j] = 0;
        bool ok = true;
        for (int c = 0; c < nchunk && ok; ++c) {
            ok = __all_sync(0xffffffffu, mbar_wait(cfull, c & 1, p.err, 3) ? 1 : 0) != 0;
            if (!ok) break;
            fence_after();
#pragma unroll
            for (int w = 0; w < kSlices; ++w) {
                uint32_t r[32];
                tmem_ld32(tmem + static_cast<uint32_t>(w * BN + half * 32) + lane_off, r);
                tmem_wait_ld();
                // the accumulators hold integers below 2^24: exact in 64-bit integers
                const long long wgt = 1ll << (7 * (kSlices - 1 - w));
#pragma unroll
                for (int j = 0; j < 32; ++j) T[j] += __float2ll_rn(__uint_as_float(r[j])) * wgt;
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(cempty);
        }
        if (ok && row < p.M) {
            const int ea = p.ea[row] - 12 - 7 * (kSlices - 1);
            double* out = p.C[z] + static_cast<size_t>(row) * p.ldc[z];
            const int col0 = n0 + half * 32;
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (col0 + j < p.N)
                    out[col0 + j] = ldexp(static_cast<double>(T[j]), ea + p.eb[z][col0 + j]);
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 2) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS)
                     : "memory");
    }
}

// frexp exponent of a normal m > 0 (m = f 2^e, f in [0.5, 1)) from its bits
__device__ __forceinline__ int exponent_of(double m) {
    return static_cast<int>((__double_as_longlong(m) >> 52) & 0x7ff) - 1022;
}
// 2^k for -1022 <= k <= 1023 from its bits
__device__ __forceinline__ double pow2(int k) {
    return __longlong_as_double(static_cast<long long>(k + 1023) << 52);
}
// Exponent e of a row (column) maximum m and the scale 2^(41 - e) that maps the row onto
// 41-bit integers; maxima below 2^-900 count as zero rows (all slices 0).
__device__ __forceinline__ void row_scale(double m, int& e, double& scale41) {
    if (m < 0x1p-900) {
        e = 0;
        scale41 = 0.0;
    } else {
        e = exponent_of(m);
        scale41 = pow2(41 - e);
    }
}

// Slices of x: v = round(x 2^(41 - e)) (|v| <= 2^41, one rounding), written in balanced
// base-128 digits from the bottom (|d| <= 64 each; the top one is <= 64 because
// |x| 2^-e < 1).  Integer arithmetic only, so the FP64 pipe does one multiply and one
// conversion per value.
__device__ __forceinline__ void put_slices(double x, double scale41, uint16_t* const* s,
                                           size_t o) {
    long long v = __double2ll_rn(x * scale41);
#pragma unroll
    for (int q = kSlices - 1; q > 0; --q) {
        const long long r = ((v + 64) & 127) - 64;
        s[q][o] = __half_as_ushort(__int2half_rn(static_cast<int>(r)));
        v = (v - r) >> 7;
    }
    s[0][o] = __half_as_ushort(__int2half_rn(static_cast<int>(v)));
}

struct SlicePtrs {
    uint16_t* s[kSlices];
    int* e;
    int ld;
};

// One block per row: the row maximum gives the exponent, then the slices.
__global__ void k_slice_rows(const double* __restrict__ A, int lda, int K, double sign,
                             SlicePtrs out) {
    const int row = blockIdx.x;
    const double* a = A + static_cast<size_t>(row) * lda;
    double m = 0.0;
    for (int k = threadIdx.x; k < K; k += blockDim.x) m = fmax(m, fabs(a[k]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    __shared__ double sc_sh;
    if (threadIdx.x == 0) {
        double mm = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = fmax(mm, red[w]);
        int e;
        double sc;
        row_scale(mm, e, sc);
        sc_sh = sign * sc;
        out.e[row] = e;
    }
    __syncthreads();
    const double sc = sc_sh;
    for (int k = threadIdx.x; k < K; k += blockDim.x)
        put_slices(a[k], sc, out.s, static_cast<size_t>(row) * out.ld + k);
}

// Column maxima |B| (colmax starts at zero): 32 columns x 8 row groups per block.
__global__ void k_colmax(const double* __restrict__ B, int ldb, int K, int cols,
                         double* __restrict__ colmax) {
    const int c = blockIdx.x * 32 + threadIdx.x;
    double m = 0.0;
    if (c < cols)
        for (int r = blockIdx.y * 8 + threadIdx.y; r < K; r += gridDim.y * 8)
            m = fmax(m, fabs(B[static_cast<size_t>(r) * ldb + c]));
    __shared__ double red[8][33];
    red[threadIdx.y][threadIdx.x] = m;
    __syncthreads();
    if (threadIdx.y == 0 && c < cols) {
        for (int y = 1; y < 8; ++y) m = fmax(m, red[y][threadIdx.x]);
        atomicMax(reinterpret_cast<unsigned long long*>(colmax + c),
                  static_cast<unsigned long long>(__double_as_longlong(m)));
    }
}

// Slices of B^T through a 32 x 32 shared-memory transpose (coalesced on both sides).
__global__ void k_slice_cols(const double* __restrict__ B, int ldb, int K, int cols,
                             const double* __restrict__ colmax, SlicePtrs out) {
    __shared__ double t[32][33];
    const int k0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = k0 + threadIdx.y + 8 * i, c = c0 + threadIdx.x;
        t[threadIdx.y + 8 * i][threadIdx.x] =
            (r < K && c < cols) ? B[static_cast<size_t>(r) * ldb + c] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int n = c0 + threadIdx.y + 8 * i, k = k0 + threadIdx.x;
        if (n >= cols || k >= K) continue;
        int e;
        double sc;
        row_scale(colmax[n], e, sc);
        if (k == 0) out.e[n] = e;
        put_slices(t[threadIdx.x][threadIdx.y + 8 * i], sc, out.s,
                   static_cast<size_t>(n) * out.ld + k);
    }
}

SlicePtrs ptrs(const Sliced& s) {
    SlicePtrs p;
    for (int q = 0; q < kSlices; ++q) p.s[q] = s.s[q];
    p.e = s.e;
    p.ld = s.ld;
    return p;
}

size_t up256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

}  // namespace

size_t sliced_bytes(int rows, int K) {
    const size_t ld = static_cast<size_t>((K + 63) / 64 * 64);
    return kSlices * up256(2 * ld * rows) + up256(sizeof(int) * rows);
}

bool sliced_init(Sliced& s, void* base, int rows, int K, int box_rows) {
    s.rows = rows;
    s.K = K;
    s.ld = (K + 63) / 64 * 64;
    char* p = static_cast<char*>(base);
    for (int q = 0; q < kSlices; ++q) {
        s.s[q] = reinterpret_cast<uint16_t*>(p);
        p += up256(2 * static_cast<size_t>(s.ld) * rows);
    }
    s.e = reinterpret_cast<int*>(p);
    for (int q = 0; q < kSlices; ++q)
        if (!tc::make_map(&s.map[q], s.s[q], rows, K, s.ld, 0, box_rows)) return false;
    return true;
}

void slice_rows(const double* A, int lda, double sign, Sliced& out, cudaStream_t st) {
    k_slice_rows<<<out.rows, 256, 0, st>>>(A, lda, out.K, sign, ptrs(out));
}

void slice_cols(const double* B, int ldb, Sliced& out, double* colmax, cudaStream_t st) {
    const int cols = out.rows, K = out.K;
    cudaMemsetAsync(colmax, 0, sizeof(double) * cols, st);
    k_colmax<<<dim3((cols + 31) / 32, 16), dim3(32, 8), 0, st>>>(B, ldb, K, cols, colmax);
    k_slice_cols<<<dim3((cols + 31) / 32, (K + 31) / 32), dim3(32, 8), 0, st>>>(B, ldb, K, cols,
                                                                              colmax, ptrs(out));
}

cudaError_t prepare() {
    return cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
}

cudaError_t gemm(const Sliced& a, const Part* parts, int nparts, int* err, cudaStream_t st) {
    if (nparts < 1 || nparts > 2 || a.K < 1 || a.K > kMaxK) return cudaErrorInvalidValue;
    const int N = parts[0].b->rows;
    Maps m;
    Params p{};
    for (int q = 0; q < kSlices; ++q) m.a[q] = a.map[q];
    for (int z = 0; z < nparts; ++z) {
        const Sliced& b = *parts[z].b;
        if (b.K != a.K || b.rows != N) return cudaErrorInvalidValue;
        for (int q = 0; q < kSlices; ++q) m.b[z][q] = b.map[q];
        p.eb[z] = b.e;
        p.C[z] = parts[z].C;
        p.ldc[z] = parts[z].ldc;
    }
    p.M = a.rows;
    p.N = N;
    p.K = a.K;
    p.ea = a.e;
    p.err = err;
    for (int nb = 1; nb <= 4; ++nb) p.idesc[nb] = tc::idesc_f16(0, nb * BN);
    const int ntile = (N + BN - 1) / BN;
    dim3 grid(ntile, (a.rows + BM - 1) / BM, nparts);
    k_oz_gemm<<<grid, kThreads, SMEM, st>>>(m, p);
    return cudaGetLastError();
}

}  // namespace oz
}  // namespace tdb
