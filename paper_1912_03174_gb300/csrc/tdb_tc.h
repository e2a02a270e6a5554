// Host interface of the tensor-core split-precision GEMM (kern_tc.cu).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "pdl.cuh"

namespace tdb {
namespace tc {

// Piece schemes of an operand x (already multiplied by its power-of-two scale s):
//  kHiLo  (2 pieces): hi = r16(x), lo = r16(x - hi); products hh + hl + lh, one accumulator.
//  kHead3 (3 pieces): head = clamp(rint(x), -127, 127) (an integer), r = x - head,
//          rh = fp16(r), rl = fp16(r - rh); the head*head products (integers) go to one
//          accumulator per 1024-deep slice of K, whose sums stay exact below 2^24, the five
//          products head*rh, rh*head, rh*rh, head*rl, rl*head to a further one.
enum Scheme { kHiLo = 3, kHead3 = 6 };
constexpr int kHeadK = 1024;    // K depth of one exact head accumulator (1040 * 127^2 < 2^24)
constexpr int kMaxParts = 6;    // output blocks of one launch (grid z)

// One output block of the GEMM: C[M x N] = sum_k A[:, k0_a + k] Bt[:, k0_b + k], k < K,
// times 1 / (scale_a scale_b); a scale is sa_dev[0] when sa_dev is set, else sa.
struct GemmPart {
    int k0_a, k0_b, K;
    int mode;        // 0: FP32 output C; 1: delta-M epilogue (re-split into A pieces)
    float* C;
    int ldc;
    float sa, sb;
    const float* sa_dev;
    const float* sb_dev;
    int b_set;       // which B map set (0..2) this part reads
};

struct GemmParams {
    int M, N;
    GemmPart part[kMaxParts];
    double* max_out;   // mode 0: atomicMax of |C| per part into max_out[part] (may be null)
    uint32_t idesc;
    int bf16;
    // mode 1 (delta M): writes the pieces of s_dm dM at column j and of s_m (Mgs + dM) at
    // column col_m + j of out[piece] (row stride ld_out)
    const float* Mgs;
    int ld_mgs;
    uint16_t* out[3];
    int ld_out, col_m;
    float s_m;
    const float* s_dm_dev;
    int* err;          // device error flag: 1-3 bounded-wait time-outs, 4 piece overflow
    // L2 prefetch of the next kernel's operands, issued by the epilogue warps while the
    // products run (parts = the CTAs of this product: tiles x parts)
    L2Prefetch pf;
};

// A: maps of the A pieces; b[set][piece]: maps of the Bt pieces.
struct Maps {
    CUtensorMap a[3];
    CUtensorMap b[3][3];
};

// Tensor map of a rows x cols row-major 16-bit matrix (row stride ld elements):
// box 32 (K) x box_rows rows, 64-byte swizzle, zero fill out of bounds.  A operands
// use 128-row boxes; B operands use boxes of the tile width bn of the launch.
bool make_map(CUtensorMap* map, const void* ptr, int rows, int cols, int ld, int bf16,
              int box_rows = 128);
uint32_t idesc_f16(int bf16, int bn = 128);
size_t smem_bytes(int scheme);
// Once per process and device before the first launch (and outside stream capture).
cudaError_t prepare();
// Output tiles of 128 x bn (bn = 64, 128, 176 or 256; the B maps must have bn-row boxes); nparts <=
// kMaxParts.  kHead3 needs (ceil(K / kHeadK) + 1) bn <= 512 TMEM columns for every part
// (cudaErrorInvalidValue otherwise).
// Whether launch() accepts these parts at tile width bn (sizes, accumulator columns).
bool launchable(int scheme, const GemmParams& p, int nparts, int bn);
cudaError_t launch(int scheme, const Maps& m, const GemmParams& p, int nparts, cudaStream_t st,
                   int bn = 128);

// One product of a grouped launch: its tensor maps and parameters (in device memory) and its
// tile grid (tiles_x column tiles x tiles_y row tiles x nparts parts).
struct GroupedGemm {
    Maps maps;
    GemmParams p;
    int tiles_x, tiles_y, nparts, pad;
};
// Many products in one launch of 128 x bn tiles: block b computes tile work[b].y (parts
// outermost, then rows, then columns) of product work[b].x.  Every product must satisfy the
// conditions of launch() for bn; g and work are device arrays.
cudaError_t launch_grouped(int scheme, const GroupedGemm* g, const int2* work, int nwork,
                           cudaStream_t st, int bn);

// Pieces of sign * scale * (in - sub) (sub may be null) for a rows x cols block.
// scale_dev (if set) overrides scale.
void launch_split(int scheme, int rows, int cols, const double* in, int ld_in, float scale,
                  int sign, int bf16, uint16_t* const* pieces, int ld_out, cudaStream_t st,
                  const double* sub = nullptr, const float* scale_dev = nullptr, int* err = nullptr);
// Pieces of delta H_kj = 1/2 S_kj (dv_k + dv_j) from FP32 S and dv = v - v_ref.  With dyn
// (kHead3) the scale is dyn->s_dh = pscale(max|dv|), which the evaluation of the level
// writes together with dv and s_dm = pscale(||S^-1||_inf max|dv|).
struct DynScales {
    double max_dv;        // max |v - v_ref| of this step
    double max_drho[3];   // max |rho - rho_ref| per density buffer; [2]: the one being written
    double sinv_norm;     // ||S^-1||_inf
    double max_x[kMaxParts];   // max |X| of each product output of this step
    float s_dh, s_dm, s_rho;
    int pad;
};
void launch_split_dham(int scheme, int N, const float* S, const float* dv, float scale, int bf16,
                       uint16_t* const* pieces, int ld_out, DynScales* dyn, cudaStream_t st,
                       int* err);
// The same for many contexts in one launch: block b runs block work[b].y (of
// split_dham_blocks(N) per problem) of args[work[b].x].
struct SplitDhArgs {
    int N, bf16, ld_out, pad;
    const float* S;
    const float* dv;
    float scale;
    uint16_t* out[3];
    DynScales* dyn;
    int* err;
};
SplitDhArgs split_dham_args(int scheme, int N, const float* S, const float* dv, float scale,
                            int bf16, uint16_t* const* pieces, int ld_out, DynScales* dyn, int* err);
int split_dham_blocks(int N);
void launch_split_dham_grouped(int scheme, const SplitDhArgs* args, const int2* work, int nwork,
                               cudaStream_t st);

// One kernel whose bounded mbarrier wait (at most polls polls) runs out and sets *err = 5.
void launch_wait_probe(long long polls, int* err, cudaStream_t st);

// Power-of-two scale mapping a magnitude bound m into (63.5, 127]: the integer heads then
// use their full 7-bit range and up to 1040 head products (<= 127^2 each) sum exactly in FP32.
// Every caller passes a rigorous bound (an exact maximum or a norm bound), so no value
// exceeds the head range.
__host__ __device__ inline float pscale(double m) {
    if (!(m > 0)) return 1099511627776.0f;   // 2^40
    int e;
    frexp(127.0 / m, &e);                    // 127/m = f 2^e, f in [0.5, 1)
    e -= 1;
    if (e > 40) e = 40;
    if (e < -40) e = -40;
    return (float)ldexp(1.0, e);
}

}  // namespace tc
}  // namespace tdb
