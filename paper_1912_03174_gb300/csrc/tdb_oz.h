// Host interface of the integer-slice GEMM (kern_oz.cu): FP64 products on the FP16
// tensor cores with exact accumulation.
//
// Each row of A is scaled by a power of two 2^-e so that its entries lie in (-1, 1),
// then cut into kSlices signed 7-bit integers (|a_s| <= 64):
//     A_ik = 2^(e_i - 6) sum_s a_s,ik 2^(-7 s) + r_ik,   |r_ik| <= 2^(e_i - 7 kSlices).
// Columns of B are treated alike (stored as rows of B^T).  Every slice product
// a_s b_t is an integer of magnitude <= 2^12, so the K-sums of all pairs of equal
// weight w = s + t over a kChunk-deep slice of K stay below 2^24 and are exact in the
// tensor core's FP32 accumulator; the sum over weights and chunks is exact in 64-bit
// integers.  Pairs with s + t < kSlices are kept, so the product carries an error of
// about (kSlices + 1) 2^(-7 kSlices) of K max_k|A_ik| max_k|B_kj| (~2e-12 relative to
// those maxima): an FP64 product for the purposes of the propagation, at tensor-core
// speed.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace tdb {
namespace oz {

constexpr int kSlices = 6;
constexpr int kChunk = 512;     // 6 pairs x 512 x 64^2 < 2^24
constexpr int kMaxK = 4096;     // keeps the 64-bit sums below 2^63

// Slices of the rows of a rows x K matrix: s[q] is rows x ld 16-bit (FP16 integers),
// ld a multiple of 64; e[i] the power-of-two exponent of row i.  The tensor maps cover
// rows x K (zero fill beyond K) with boxes of 32 (K) x box_rows.
struct Sliced {
    uint16_t* s[kSlices] = {};
    int* e = nullptr;
    int rows = 0, K = 0, ld = 0;
    CUtensorMap map[kSlices];
};

// Bytes of device memory a Sliced of rows x K needs (slices + exponents).
size_t sliced_bytes(int rows, int K);
// Lays a Sliced out in base (256-byte aligned) and encodes its tensor maps; box_rows
// is 128 for an A operand and 64 for a B operand.  False if a map cannot be encoded.
bool sliced_init(Sliced& s, void* base, int rows, int K, int box_rows);

// Slices of sign * A (rows x K, row-major FP64 with row stride lda), row scales.  For
// a B operand that is symmetric (sign 1) or antisymmetric (sign -1) this is also the
// slicing of B^T.
void slice_rows(const double* A, int lda, double sign, Sliced& out, cudaStream_t st);
// Slices of B^T for a general B (K x cols, row-major FP64, row stride ldb); colmax is
// a device scratch of cols doubles.
void slice_cols(const double* B, int ldb, Sliced& out, double* colmax, cudaStream_t st);

// One product sharing the A operand: C (M x N, row-major FP64, row stride ldc) = A B.
struct Part {
    const Sliced* b = nullptr;
    double* C = nullptr;
    int ldc = 0;
};
// Once per process and device before the first launch (outside stream capture).
cudaError_t prepare();
// C_z = A B_z for z < nparts (<= 2); M = a.rows, N = b.rows, K = a.K = b.K (<= kMaxK).
// err: device flag, set to 1-3 if a bounded wait expired.
cudaError_t gemm(const Sliced& a, const Part* parts, int nparts, int* err, cudaStream_t st);

}  // namespace oz
}  // namespace tdb
