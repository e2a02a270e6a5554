// Tensor-core (tcgen05) split-precision GEMM for sm_103a.
//
// Operands are carried as 16-bit pieces (see tdb_tc.h for the two schemes).
// kHiLo evaluates A_hi B_hi + A_hi B_lo + A_lo B_hi into one FP32 TMEM
// accumulator.  The tensor core's FP32 accumulation truncates, which biases
// long sums by ~K 2^-25 relative; kHead3 removes that bias from the dominant
// term: the integer heads' products are summed exactly (integers below 2^24)
// in their own accumulator and only the small tail products (~2^-7 of the
// result) share the second, inexact one.
//
// Data path: TMA (cp.async.bulk.tensor, 64-byte swizzle, K blocks of 32) ->
// shared-memory ring of up to 8 stages (mbarrier full/empty pairs) ->
// tcgen05.mma issued by one thread -> TMEM accumulators (128 lanes x BN
// columns each; kHead3 keeps one head accumulator per 1024 of K plus the tail
// one) -> tcgen05.ld by all 8 warps -> epilogue in registers -> global.  Both
// operands are K-major: A is M x K row-major and B is given as its transpose
// Bt (N x K row-major).
//
// Every mbarrier wait is bounded; on time-out the kernel records an error
// code, lets the issued MMAs drain, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include <cstdint>

#include "pdl.cuh"
#include "tc_ptx.cuh"
#include "tc_split.cuh"
#include "tdb_tc.h"

namespace tdb {
namespace tc {

namespace {
using namespace ptx;

// K blocks of 32 (64 bytes of 16-bit values, one 64-byte swizzle span): smaller stages,
// so more of them fit and the TMA producer can run further ahead of the MMAs.
constexpr int BM = 128, BK = 32;
constexpr int TILE_BYTES = BM * BK * 2;   // 8 KiB per A piece (B pieces: BN * BK * 2)
constexpr int kThreads = 256;             // 8 warps: all of them run the epilogue
constexpr int kHeadKB = kHeadK / BK;      // K blocks per exact head accumulator

template <int SCHEME>
struct Cfg;
template <>
struct Cfg<kHiLo> {
    static constexpr int PIECES = 2;
};
template <>
struct Cfg<kHead3> {
    static constexpr int PIECES = 3;
};

// Accumulators of a K-deep product: kHead3 one exact head accumulator per kHeadK slice
// plus the tail accumulators; kHiLo one.  With 64-wide kHead3 tiles the five tail
// products get one accumulator each (n_tails = 5), so that products sharing an A piece
// run as one MMA over two adjacent B pieces (N = 128) into adjacent accumulators: four
// MMAs per 16-deep step instead of six.
__host__ __device__ inline int n_heads(int scheme, int K) {
    return scheme == kHead3 ? (K + kHeadK - 1) / kHeadK : 0;
}
__host__ __device__ constexpr int n_tails(int scheme, int bn) {
    return scheme == kHead3 && bn == 64 ? 5 : 1;
}
__host__ __device__ inline uint32_t tmem_cols(int scheme, int K, int bn) {
    const uint32_t need = static_cast<uint32_t>((n_heads(scheme, K) + n_tails(scheme, bn)) * bn);
    uint32_t cols = 32;
    while (cols < need) cols <<= 1;
    return cols;
}
template <int S, int BN>
__host__ __device__ constexpr int stage_bytes() {
    return Cfg<S>::PIECES * (TILE_BYTES + BN * BK * 2);
}
// as many ring stages as fit in 227 KiB of shared memory, at most 4 (measured: the 64-wide
// delta-M tiles ran 7% faster with 4 stages than with 6; the wider tiles fit at most 4)
template <int S, int BN>
__host__ __device__ constexpr int stages() {
    return (227 * 1024 - 1024 - 256) / stage_bytes<S, BN>() > 4
               ? 4
               : (227 * 1024 - 1024 - 256) / stage_bytes<S, BN>();
}
template <int S, int BN>
__host__ __device__ constexpr int smem_total() {
    return stages<S, BN>() * stage_bytes<S, BN>() + 1024 + 256;
}

// One 128 x BN output tile (tile column tx, tile row ty) of part tz of a product.  The
// tensor maps may live in kernel parameters or in global memory (grouped launches).
template <int SCHEME, int BN>
__device__ __forceinline__ void gemm_tile(const Maps& maps, const GemmParams& p, int tx, int ty,
                                          int tz) {
    constexpr int PIECES = Cfg<SCHEME>::PIECES, STAGES = stages<SCHEME, BN>();
    constexpr int SB = stage_bytes<SCHEME, BN>();
    constexpr int BTILE = BN * BK * 2;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* gbase = smem_raw + (base - raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + STAGES * SB);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 1);
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES),
                   done = smem_u32(bars + 2 * STAGES);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const GemmPart& P = p.part[tz];
    const int m0 = ty * BM, n0 = tx * BN;
    const int nkb = (P.K + BK - 1) / BK;
    // TMEM columns [h BN, (h + 1) BN): head accumulator of K slice h; then the tail one
    const int nheads = n_heads(SCHEME, P.K);
    const uint32_t ncols = tmem_cols(SCHEME, P.K, BN);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        fence_before();
    }
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    // delta-M epilogue of 64-wide tiles (one 32-column chunk per warp): every thread loads
    // its row's 32 values of M_gs now, so that the loads overlap the products
    float4 mgs_pre[8];
    bool pre = false;
    if (BN == 64 && P.mode == 1) {
        const int row = m0 + (warp & 3) * 32 + lane, col0 = n0 + (warp >> 2) * 32;
        pre = row < p.M && col0 + 32 <= p.N && (p.ld_mgs & 3) == 0;
        if (pre) {
            const float4* mg4 =
                reinterpret_cast<const float4*>(p.Mgs + static_cast<size_t>(row) * p.ld_mgs + col0);
#pragma unroll
            for (int u = 0; u < 8; ++u) mgs_pre[u] = __ldg(mg4 + u);
        }
    }
    // everything above touches only constants and this CTA's own memory: the operands the
    // previous kernel wrote are read from here on
    pdl_wait();
    if (warp == 0 && lane == 0) {
        // TMA producer: A pieces then B pieces of one 64-wide K block per stage
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % STAGES, round = kb / STAGES;
            if (kb >= STAGES && !mbar_wait(empty0 + 8 * s, (round - 1) & 1, p.err, 1)) break;
            const uint32_t st = base + s * SB;
            const uint32_t fb = full0 + 8 * s;
            mbar_expect_tx(fb, SB);
#pragma unroll
            for (int q = 0; q < PIECES; ++q) {
                tma_load_2d(st + q * TILE_BYTES, &maps.a[q], P.k0_a + kb * BK, m0, fb);
                tma_load_2d(st + PIECES * TILE_BYTES + q * BTILE, &maps.b[P.b_set][q],
                            P.k0_b + kb * BK, n0, fb);
            }
        }
    } else if (warp == 1 && lane == 0) {
        const uint32_t tail = tmem + static_cast<uint32_t>(nheads * BN);
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % STAGES, round = kb / STAGES;
            if (!mbar_wait(full0 + 8 * s, round & 1, p.err, 2)) break;
            fence_after();
            const uint32_t st = base + s * SB;
#pragma unroll
            for (int k = 0; k < BK / 16; ++k) {
                uint64_t a[PIECES], b[PIECES];
#pragma unroll
                for (int q = 0; q < PIECES; ++q) {
                    a[q] = sdesc(st + q * TILE_BYTES + k * 32);
                    b[q] = sdesc(st + PIECES * TILE_BYTES + q * BTILE + k * 32);
                }
                const uint32_t accum = (kb | k) != 0;   // 0: the first product overwrites
                if (SCHEME == kHiLo) {
                    mma_f16(tail, a[0], b[0], p.idesc, accum);
                    mma_f16(tail, a[0], b[1], p.idesc, 1);
                    mma_f16(tail, a[1], b[0], p.idesc, 1);
                } else {
                    // exact integer sums, a fresh accumulator every kHeadK of K
                    const uint32_t head = tmem + static_cast<uint32_t>((kb / kHeadKB) * BN);
                    mma_f16(head, a[0], b[0], p.idesc, ((kb % kHeadKB) | k) != 0);
                    if (n_tails(SCHEME, BN) == 5) {
                        // tails [a0 b1 | a0 b2 | a1 b0 | a1 b1 | a2 b0], B pieces adjacent
                        const uint32_t idw = (p.idesc & ~(0x3Fu << 17)) |
                                             (static_cast<uint32_t>(2 * BN >> 3) << 17);
                        mma_f16(tail, a[0], b[1], idw, accum);
                        mma_f16(tail + static_cast<uint32_t>(2 * BN), a[1], b[0], idw, accum);
                        mma_f16(tail + static_cast<uint32_t>(4 * BN), a[2], b[0], p.idesc, accum);
                    } else {
                        mma_f16(tail, a[0], b[1], p.idesc, accum);
                        mma_f16(tail, a[1], b[0], p.idesc, 1);
                        mma_f16(tail, a[1], b[1], p.idesc, 1);
                        mma_f16(tail, a[0], b[PIECES - 1], p.idesc, 1);
                        mma_f16(tail, a[PIECES - 1], b[0], p.idesc, 1);
                    }
                }
            }
            mma_commit(empty0 + 8 * s);
        }
        mma_commit(done);
    } else if (warp >= 2 && p.pf.n > 0) {
        // this CTA's share of the lines to prefetch (CTAs numbered over tiles and parts)
        const int tiles_x = (p.N + BN - 1) / BN, tiles_y = (p.M + BM - 1) / BM;
        l2_prefetch_share(p.pf, ((long long)tz * tiles_y + ty) * tiles_x + tx, threadIdx.x - 64,
                          kThreads - 64);
    }
    __syncwarp();

    // epilogue: warp w reads TMEM lanes (rows) 32 (w % 4) .. + 31 (the lane quarter a warp
    // may access) and every second 32-column chunk starting at chunk w / 4
    const bool ok = __all_sync(0xffffffffu, mbar_wait(done, 0, p.err, 3) ? 1 : 0) != 0;
    fence_after();
    // the products are done: the next kernel may be scheduled while the epilogue runs
    pdl_launch_dependents();
    if (ok) {
        const float sa = P.sa_dev ? *P.sa_dev : P.sa, sb = P.sb_dev ? *P.sb_dev : P.sb;
        const float inv = 1.0f / (sa * sb);
        const int quarter = warp & 3;
        const int row = m0 + quarter * 32 + lane;
        const uint32_t lane_off = static_cast<uint32_t>(quarter * 32) << 16;
        for (int c = warp >> 2; c < (BN + 31) / 32; c += kThreads / 128) {
            // columns of this chunk inside the tile (a 176-wide tile ends in a 16-column
            // chunk; the TMEM columns read past it belong to the next accumulator or to
            // the unused end of the allocation) and inside the matrix
            const int lim = min(min(32, BN - c * 32), p.N - (n0 + c * 32));
            uint32_t r[32];
            tmem_ld32(tmem + lane_off + c * 32, r);
            float v[32];
            if (SCHEME == kHead3) {
                // heads summed first (exact while below 2^24), then the tail
                uint32_t r1[32];
                tmem_ld32(tmem + static_cast<uint32_t>(nheads * BN) + lane_off + c * 32, r1);
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
                for (int h = 1; h < nheads; ++h) {
                    tmem_ld32(tmem + static_cast<uint32_t>(h * BN) + lane_off + c * 32, r);
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] += __uint_as_float(r[j]);
                }
                // separate tail accumulators summed in a fixed order
                for (int t = 1; t < n_tails(SCHEME, BN); ++t) {
                    tmem_ld32(tmem + static_cast<uint32_t>((nheads + t) * BN) + lane_off + c * 32, r);
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        r1[j] = __float_as_uint(__uint_as_float(r1[j]) + __uint_as_float(r[j]));
                }
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = (v[j] + __uint_as_float(r1[j])) * inv;
            } else {
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]) * inv;
            }
            const int col0 = n0 + c * 32;
            if (P.mode == 0 && p.max_out) {
                float m = 0.f;
                if (row < p.M)
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (j < lim) m = fmaxf(m, fabsf(v[j]));
                for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
                if (lane == 0)
                    atomicMax(reinterpret_cast<unsigned long long*>(&p.max_out[tz]),
                              static_cast<unsigned long long>(__double_as_longlong(static_cast<double>(m))));
            }
            if (row >= p.M) continue;
            if (P.mode == 0) {
                float* out = P.C + static_cast<size_t>(row) * P.ldc + col0;
                if (lim == 32 && (P.ldc & 3) == 0) {
#pragma unroll
                    for (int j = 0; j < 32; j += 4)
                        *reinterpret_cast<float4*>(out + j) =
                            make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (j < lim) out[j] = v[j];
                }
            } else {
                // delta M and M = M_gs + delta M, both re-split into A pieces; 16-byte
                // vector loads of M_gs and stores of 8 pieces at a time
                const float s_dm = p.s_dm_dev ? *p.s_dm_dev : 1.0f;
                const float* mg = p.Mgs + static_cast<size_t>(row) * p.ld_mgs + col0;
                const size_t ob = static_cast<size_t>(row) * p.ld_out + col0;
                bool fine = true;
                const bool vec = lim == 32 && (p.ld_mgs & 3) == 0 && (p.ld_out & 7) == 0 &&
                                 (p.col_m & 7) == 0;
                if (vec) {
#pragma unroll
                    for (int j0 = 0; j0 < 32; j0 += 8) {
                        const float4 g0 = pre ? mgs_pre[j0 / 4] : *reinterpret_cast<const float4*>(mg + j0);
                        const float4 g1 =
                            pre ? mgs_pre[j0 / 4 + 1] : *reinterpret_cast<const float4*>(mg + j0 + 4);
                        const float gm[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
                        uint16_t qd[3][8], qm[3][8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            uint16_t q[3];
                            fine &= split_value<SCHEME>(v[j0 + j] * s_dm, p.bf16, q);
#pragma unroll
                            for (int t = 0; t < 3; ++t) qd[t][j] = q[t];
                            fine &= split_value<SCHEME>((gm[j] + v[j0 + j]) * p.s_m, p.bf16, q);
#pragma unroll
                            for (int t = 0; t < 3; ++t) qm[t][j] = q[t];
                        }
#pragma unroll
                        for (int t = 0; t < PIECES; ++t) {
                            uint4 a, b;
                            a.x = qd[t][0] | (uint32_t(qd[t][1]) << 16);
                            a.y = qd[t][2] | (uint32_t(qd[t][3]) << 16);
                            a.z = qd[t][4] | (uint32_t(qd[t][5]) << 16);
                            a.w = qd[t][6] | (uint32_t(qd[t][7]) << 16);
                            b.x = qm[t][0] | (uint32_t(qm[t][1]) << 16);
                            b.y = qm[t][2] | (uint32_t(qm[t][3]) << 16);
                            b.z = qm[t][4] | (uint32_t(qm[t][5]) << 16);
                            b.w = qm[t][6] | (uint32_t(qm[t][7]) << 16);
                            *reinterpret_cast<uint4*>(p.out[t] + ob + j0) = a;
                            *reinterpret_cast<uint4*>(p.out[t] + ob + p.col_m + j0) = b;
                        }
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        if (j >= lim) continue;
                        uint16_t q[3];
                        fine &= split_value<SCHEME>(v[j] * s_dm, p.bf16, q);
#pragma unroll
                        for (int t = 0; t < PIECES; ++t) p.out[t][ob + j] = q[t];
                        fine &= split_value<SCHEME>((mg[j] + v[j]) * p.s_m, p.bf16, q);
#pragma unroll
                        for (int t = 0; t < PIECES; ++t) p.out[t][ob + p.col_m + j] = q[t];
                    }
                }
                if (!fine && p.err) atomicCAS(p.err, 0, 4);
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 2) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(ncols)
                     : "memory");
    }
}

template <int SCHEME, int BN>
__global__ void __launch_bounds__(kThreads, 1)
    k_split_gemm(const __grid_constant__ Maps maps, GemmParams p) {
    gemm_tile<SCHEME, BN>(maps, p, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Many independent products in one launch: block b takes work[b] = (problem, tile index
// within the problem, parts outermost), so the order of the work list is the schedule.
template <int SCHEME, int BN>
__global__ void __launch_bounds__(kThreads, 1)
    k_split_gemm_grouped(const GroupedGemm* __restrict__ g, const int2* __restrict__ work) {
    const int2 w = work[blockIdx.x];
    const GroupedGemm& G = g[w.x];
    const int per = G.tiles_x * G.tiles_y;
    const int tz = w.y / per, r = w.y - tz * per;
    gemm_tile<SCHEME, BN>(G.maps, G.p, r % G.tiles_x, r / G.tiles_x, tz);
}

// ---- splitting kernels (FP64 -> scaled 16-bit pieces) ----

struct Pieces {
    uint16_t* p[3];
};

template <int SCHEME>
__global__ void k_split(int rows, int cols, const double* __restrict__ in,
                        const double* __restrict__ sub, int ld_in, float scale,
                        const float* __restrict__ scale_dev, int sign, int bf16, Pieces out,
                        int ld_out, int* err) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y * blockDim.y + threadIdx.y;
    if (r >= rows || c >= cols) return;
    const size_t i = static_cast<size_t>(r) * ld_in + c;
    const double v = sub ? in[i] - sub[i] : in[i];
    const float s = scale_dev ? *scale_dev : scale;
    uint16_t q[3];
    const bool ok = split_value<SCHEME>(static_cast<float>(sign * v) * s, bf16, q);
    const size_t o = static_cast<size_t>(r) * ld_out + c;
#pragma unroll
    for (int t = 0; t < Cfg<SCHEME>::PIECES; ++t) out.p[t][o] = q[t];
    if (!ok && err) atomicCAS(err, 0, 4);
}

// delta H_kj = 1/2 S_kj (dv_k + dv_j) from FP32 copies of S and dv = v - v_ref; block
// (bx, by) of a grid with gy block rows
template <int SCHEME>
__device__ __forceinline__ void split_dham_block(int N, const float* __restrict__ S,
                                                 const float* __restrict__ dv, float scale_const,
                                                 int bf16, const Pieces& out, int ld_out,
                                                 const DynScales* __restrict__ dyn, int* err,
                                                 int bx, int by, int gy) {
    // FP16X6: the delta-M product may be scheduled now (its CTAs set up their barriers and
    // tensor memory and load M_gs while this kernel runs, then wait for it).  Its CTAs cannot
    // share an SM with this kernel's, so they start as SMs drain; the smaller two-piece CTAs
    // can, and slowed the split (measured: FP16X6 +1.6%, BF16X3 -7% steps/s)
    if (SCHEME == kHead3) pdl_launch_dependents();
    const int c = bx * blockDim.x + threadIdx.x;
    const int r = by * blockDim.y + threadIdx.y;
    // FP16X6: the scale of this step, pscale(max |dv|), written with dv by the evaluation
    // of the level (|delta H| <= max |dv| since |S_kj| <= 1)
    const float s = dyn ? dyn->s_dh : scale_const;
    if (c >= N) return;
    // rows r, r + gridDim.y blockDim.y, ...: the scale prologue is paid once per block
    const float dvc = __ldg(dv + c);
    bool ok = true;
    const int stride = gy * blockDim.y;
    // eight rows per pass with their loads in flight together
    for (int row0 = r; row0 < N; row0 += 8 * stride) {
        float sv[8], dr[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int row = row0 + u * stride;
            sv[u] = row < N ? __ldg(S + static_cast<size_t>(row) * N + c) : 0.f;
            dr[u] = row < N ? __ldg(dv + row) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int row = row0 + u * stride;
            if (row >= N) break;
            uint16_t q[3];
            ok &= split_value<SCHEME>(0.5f * sv[u] * (dr[u] + dvc) * s, bf16, q);
            const size_t o = static_cast<size_t>(row) * ld_out + c;
#pragma unroll
            for (int t = 0; t < Cfg<SCHEME>::PIECES; ++t) out.p[t][o] = q[t];
        }
    }
    if (!ok && err) atomicCAS(err, 0, 4);
}

template <int SCHEME>
__global__ void k_split_dham(int N, const float* __restrict__ S, const float* __restrict__ dv,
                             float scale_const, int bf16, Pieces out, int ld_out,
                             DynScales* __restrict__ dyn, int* err) {
    split_dham_block<SCHEME>(N, S, dv, scale_const, bf16, out, ld_out, dyn, err, blockIdx.x,
                             blockIdx.y, gridDim.y);
}

template <int SCHEME>
__global__ void k_split_dham_grouped(const SplitDhArgs* __restrict__ args,
                                     const int2* __restrict__ work) {
    const int2 w = work[blockIdx.x];
    const SplitDhArgs& a = args[w.x];
    const int gx = (a.N + 31) / 32, gy = (a.N + 63) / 64;
    const Pieces out{{a.out[0], a.out[1], a.out[2]}};
    split_dham_block<SCHEME>(a.N, a.S, a.dv, a.scale, a.bf16, out, a.ld_out, a.dyn, a.err,
                             w.y % gx, w.y / gx, gy);
}

// Failure-detection probe: one thread waits on an mbarrier that nothing arrives on, polling
// at most `polls` times, then records a time-out (code 5).  No copy or MMA is in flight and
// no TMEM is held, so the expired wait leaves nothing behind.
__global__ void k_wait_probe(long long polls, int* err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    const uint32_t b = smem_u32(&bar);
    mbar_init(b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (long long i = 0; i < polls; ++i)
        if (mbar_try_wait(b, 0)) return;
    atomicCAS(err, 0, 5);
}

}  // namespace

void launch_wait_probe(long long polls, int* err, cudaStream_t st) {
    k_wait_probe<<<1, 32, 0, st>>>(polls, err);
}

size_t smem_bytes(int scheme) {
    return scheme == kHiLo ? smem_total<kHiLo, 128>() : smem_total<kHead3, 128>();
}

bool make_map(CUtensorMap* map, const void* ptr, int rows, int cols, int ld, int bf16,
              int box_rows) {
    using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static EncodeFn encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = reinterpret_cast<EncodeFn>(fn);
    }
    const cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
    const cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * 2};
    const cuuint32_t box[2] = {BK, static_cast<cuuint32_t>(box_rows)};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r =
        encode(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
               const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

uint32_t idesc_f16(int bf16, int bn) {
    // D = F32 (bits 4-5), A/B format (7-9, 10-12: 0 F16, 1 BF16), both K-major,
    // N >> 3 at bit 17, M >> 4 at bit 24
    return (1u << 4) | (static_cast<uint32_t>(bf16) << 7) | (static_cast<uint32_t>(bf16) << 10) |
           (static_cast<uint32_t>(bn >> 3) << 17) | (static_cast<uint32_t>(BM >> 4) << 24);
}

template <int S, int BN>
cudaError_t set_smem() {
    return cudaFuncSetAttribute(k_split_gemm<S, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smem_total<S, BN>());
}

template <int S, int BN>
cudaError_t set_smem_grouped() {
    return cudaFuncSetAttribute(k_split_gemm_grouped<S, BN>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem_total<S, BN>());
}

cudaError_t prepare() {
    cudaError_t e = set_smem<kHiLo, 64>();
    if (e == cudaSuccess) e = set_smem_grouped<kHiLo, 64>();
    if (e == cudaSuccess) e = set_smem_grouped<kHead3, 64>();
    if (e == cudaSuccess) e = set_smem_grouped<kHiLo, 128>();
    if (e == cudaSuccess) e = set_smem_grouped<kHead3, 128>();
    if (e == cudaSuccess) e = set_smem_grouped<kHiLo, 176>();
    if (e == cudaSuccess) e = set_smem_grouped<kHead3, 176>();
    if (e == cudaSuccess) e = set_smem_grouped<kHiLo, 256>();
    if (e == cudaSuccess) e = set_smem_grouped<kHead3, 256>();
    if (e == cudaSuccess) e = set_smem<kHead3, 64>();
    if (e == cudaSuccess) e = set_smem<kHiLo, 128>();
    if (e == cudaSuccess) e = set_smem<kHead3, 128>();
    if (e == cudaSuccess) e = set_smem<kHiLo, 256>();
    if (e == cudaSuccess) e = set_smem<kHead3, 256>();
    if (e == cudaSuccess) e = set_smem<kHiLo, 176>();
    if (e == cudaSuccess) e = set_smem<kHead3, 176>();
    return e;
}

bool launchable(int scheme, const GemmParams& p, int nparts, int bn) {
    if (nparts < 1 || nparts > kMaxParts || (bn != 64 && bn != 128 && bn != 176 && bn != 256))
        return false;
    for (int z = 0; z < nparts; ++z)
        if (p.part[z].K < 1 || tmem_cols(scheme, p.part[z].K, bn) > 512) return false;
    return true;
}

cudaError_t launch(int scheme, const Maps& m, const GemmParams& p, int nparts, cudaStream_t st,
                   int bn) {
    if (!launchable(scheme, p, nparts, bn)) return cudaErrorInvalidValue;
    dim3 grid((p.N + bn - 1) / bn, (p.M + BM - 1) / BM, nparts);
    cudaError_t e;
    if (bn == 64) {
        if (scheme == kHiLo)
            e = launch_pdl(k_split_gemm<kHiLo, 64>, grid, dim3(kThreads), smem_total<kHiLo, 64>(), st, m, p);
        else
            e = launch_pdl(k_split_gemm<kHead3, 64>, grid, dim3(kThreads), smem_total<kHead3, 64>(), st, m, p);
    } else if (bn == 256) {
        if (scheme == kHiLo)
            e = launch_pdl(k_split_gemm<kHiLo, 256>, grid, dim3(kThreads), smem_total<kHiLo, 256>(), st, m, p);
        else
            e = launch_pdl(k_split_gemm<kHead3, 256>, grid, dim3(kThreads), smem_total<kHead3, 256>(), st, m, p);
    } else if (bn == 176) {
        if (scheme == kHiLo)
            e = launch_pdl(k_split_gemm<kHiLo, 176>, grid, dim3(kThreads), smem_total<kHiLo, 176>(), st, m, p);
        else
            e = launch_pdl(k_split_gemm<kHead3, 176>, grid, dim3(kThreads), smem_total<kHead3, 176>(), st, m, p);
    } else {
        if (scheme == kHiLo)
            e = launch_pdl(k_split_gemm<kHiLo, 128>, grid, dim3(kThreads), smem_total<kHiLo, 128>(), st, m, p);
        else
            e = launch_pdl(k_split_gemm<kHead3, 128>, grid, dim3(kThreads), smem_total<kHead3, 128>(), st, m, p);
    }
    return e;
}

cudaError_t launch_grouped(int scheme, const GroupedGemm* g, const int2* work, int nwork,
                           cudaStream_t st, int bn) {
    if (nwork < 1 || (bn != 64 && bn != 128 && bn != 176 && bn != 256)) return cudaErrorInvalidValue;
    cudaError_t e;
#define TDB_GROUPED(S, W)                                                                     \
    e = launch_pdl(k_split_gemm_grouped<S, W>, dim3(nwork), dim3(kThreads), smem_total<S, W>(), st, g, work)
    if (scheme == kHiLo) {
        if (bn == 64) TDB_GROUPED(kHiLo, 64);
        else if (bn == 128) TDB_GROUPED(kHiLo, 128);
        else if (bn == 176) TDB_GROUPED(kHiLo, 176);
        else TDB_GROUPED(kHiLo, 256);
    } else {
        if (bn == 64) TDB_GROUPED(kHead3, 64);
        else if (bn == 128) TDB_GROUPED(kHead3, 128);
        else if (bn == 176) TDB_GROUPED(kHead3, 176);
        else TDB_GROUPED(kHead3, 256);
    }
#undef TDB_GROUPED
    return e;
}

void launch_split(int scheme, int rows, int cols, const double* in, int ld_in, float scale, int sign,
                  int bf16, uint16_t* const* pieces, int ld_out, cudaStream_t st, const double* sub,
                  const float* scale_dev, int* err) {
    dim3 b(32, 8);
    dim3 g((cols + 31) / 32, (rows + 7) / 8);
    Pieces o{{pieces[0], pieces[1], scheme == kHead3 ? pieces[2] : nullptr}};
    if (scheme == kHiLo)
        k_split<kHiLo><<<g, b, 0, st>>>(rows, cols, in, sub, ld_in, scale, scale_dev, sign, bf16, o,
                                        ld_out, err);
    else
        k_split<kHead3><<<g, b, 0, st>>>(rows, cols, in, sub, ld_in, scale, scale_dev, sign, bf16,
                                         o, ld_out, err);
}

SplitDhArgs split_dham_args(int scheme, int N, const float* S, const float* dv, float scale,
                            int bf16, uint16_t* const* pieces, int ld_out, DynScales* dyn, int* err) {
    SplitDhArgs a{};
    a.N = N;
    a.S = S;
    a.dv = dv;
    a.scale = scale;
    a.bf16 = bf16;
    for (int t = 0; t < 3; ++t) a.out[t] = (t < 2 || scheme == kHead3) ? pieces[t] : nullptr;
    a.ld_out = ld_out;
    a.dyn = scheme == kHead3 ? dyn : nullptr;
    a.err = err;
    return a;
}

int split_dham_blocks(int N) { return ((N + 31) / 32) * ((N + 63) / 64); }

void launch_split_dham_grouped(int scheme, const SplitDhArgs* args, const int2* work, int nwork,
                               cudaStream_t st) {
    if (scheme == kHiLo)
        k_split_dham_grouped<kHiLo><<<nwork, dim3(32, 8), 0, st>>>(args, work);
    else
        k_split_dham_grouped<kHead3><<<nwork, dim3(32, 8), 0, st>>>(args, work);
}

void launch_split_dham(int scheme, int N, const float* S, const float* dv, float scale, int bf16,
                       uint16_t* const* pieces, int ld_out, DynScales* dyn, cudaStream_t st,
                       int* err) {
    dim3 b(32, 8);
    // about 8 rows per thread
    dim3 g((N + 31) / 32, (N + 63) / 64);
    Pieces o{{pieces[0], pieces[1], scheme == kHead3 ? pieces[2] : nullptr}};
    if (scheme == kHiLo)
        k_split_dham<kHiLo><<<g, b, 0, st>>>(N, S, dv, scale, bf16, o, ld_out, nullptr, err);
    else
        k_split_dham<kHead3><<<g, b, 0, st>>>(N, S, dv, scale, bf16, o, ld_out, dyn, err);
}

}  // namespace tc
}  // namespace tdb
