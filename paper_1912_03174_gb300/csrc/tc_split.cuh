// Pieces of one scaled FP32 value for the tensor-core split-precision products (the
// two schemes of tdb_tc.h), shared by every kernel that writes operand pieces.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>

#include "tdb_tc.h"

namespace tdb {
namespace tc {

__device__ __forceinline__ uint16_t to16(float x, int bf16) {
    if (bf16) return __bfloat16_as_ushort(__float2bfloat16_rn(x));
    return __half_as_ushort(__float2half_rn(x));
}
__device__ __forceinline__ float from16(uint16_t x, int bf16) {
    if (bf16) return __bfloat162float(__ushort_as_bfloat16(x));
    return __half2float(__ushort_as_half(x));
}

// Pieces of one scaled FP32 value (see tdb_tc.h); FP32 arithmetic only (FP64 is slow
// on this part).  For the head scheme the pieces reproduce the FP32 value exactly:
// x - head is exact, and 11 + 11 tail bits cover the <= 17 bits left after the head.
// Returns false if a tail overflows FP16.
template <int SCHEME>
__device__ __forceinline__ bool split_value(float x, int bf16, uint16_t (&q)[3]) {
    if (SCHEME == kHiLo) {
        q[0] = to16(x, bf16);
        q[1] = to16(x - from16(q[0], bf16), bf16);
        q[2] = 0;
        return fabsf(x) < 65000.f;
    } else {
        const float h = fminf(fmaxf(rintf(x), -127.f), 127.f);
        const float r = x - h;
        const __half rh = __float2half_rn(r);
        q[0] = __half_as_ushort(__float2half_rn(h));
        q[1] = __half_as_ushort(rh);
        q[2] = __half_as_ushort(__float2half_rn(r - __half2float(rh)));
        return fabsf(r) < 65000.f;
    }
}

}  // namespace tc
}  // namespace tdb
