// Programmatic dependent launch between the kernels of a step.  A kernel launched with
// launch_pdl may be scheduled while its predecessor in the stream is still running: what it
// does before pdl_wait() (loads of constant operands, L2 prefetches, barrier and tensor
// memory set-up) overlaps the predecessor's tail, and pdl_wait() blocks until the
// predecessor grid has completed with its writes visible.  Without the launch attribute
// pdl_wait() returns at once.  pdl_launch_dependents() lets the next kernel be scheduled
// before this one ends; without it that happens when this grid completes.
#pragma once

#include <cuda_runtime.h>

namespace tdb {

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// L2 prefetch of another kernel's operands: regions ptr[r] of bytes[r] bytes (r < n), shared
// out in 128-byte lines over the `parts` CTAs of the launch that issues them.
struct L2Prefetch {
    const void* ptr[6];
    size_t bytes[6];
    int n, parts;
};

// The lines of share `part` (of pf.parts), issued by threads tid = 0 .. nthreads - 1.
__device__ __forceinline__ void l2_prefetch_share(const L2Prefetch& pf, long long part, int tid,
                                                  int nthreads) {
    long long total = 0;
    for (int r = 0; r < pf.n; ++r) total += (long long)(pf.bytes[r] >> 7);
    const long long l0 = total * part / pf.parts, l1 = total * (part + 1) / pf.parts;
    long long off = 0;
    for (int r = 0; r < pf.n; ++r) {
        const long long nl = (long long)(pf.bytes[r] >> 7);
        const long long a = l0 > off ? l0 : off, b = l1 < off + nl ? l1 : off + nl;
        const char* base = static_cast<const char*>(pf.ptr[r]);
        for (long long i = a + tid; i < b; i += nthreads)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(base + ((i - off) << 7)));
        off += nl;
    }
}

template <typename... P, typename... A>
inline cudaError_t launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, A&&... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<A&&>(args)...);
}

}  // namespace tdb
