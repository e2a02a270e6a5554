// tdb_split_gemm_noalloc: the tensor-core split-precision GEMM for callers that
// cannot allocate device memory.
//
// Some callers may not call cudaMalloc (or any allocator) at the point where
// they need a product: code running inside a fixed, pre-reserved memory budget
// (a serving process that has handed all free memory to its own pool), code
// that runs while another component owns the allocator, or code that must not
// synchronise the device, which cudaMalloc/cudaFree can do.  This entry point
// takes device inputs and a device output from the caller and keeps its
// intermediate operands in one file-scope device array instead.
//
// That array (kScratchBytes) is reserved on every GPU that loads the library
// and stays reserved until the process exits.  Every call shares it and it
// keeps the contents of the last call, so calls whose GPU work overlaps (two
// streams, or two host threads) race on it; serialise them.  The first call on
// a device looks up the array's device address (cudaGetSymbolAddress) and sets
// the kernel's shared-memory attribute; make that first call before any CUDA
// stream capture.
//
// The call returns before the GPU work runs, so a failure on the device (a bounded
// wait of the product that ran out, or an operand piece that overflows, e.g. from an
// Inf or NaN input) cannot be returned as a status: the last kernel then fills all of
// C with NaN instead of a wrong product.
#include <cmath>
#include <cstdint>
#include <mutex>

#include "tc_split.cuh"
#include "tdb_internal.h"
#include "tdb_tc.h"

namespace tdb {
void launch_absmax(size_t n, const double* x, double* out, cudaStream_t st, const double* sub);
void set_last_error(const char* msg);
}

namespace {

constexpr size_t kScratchBytes = 8u << 20;   // 8 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once per device).
tdb_status scratch_address(unsigned char** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TDB_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return TDB_ERR_CUDA;
        }
        if (tdb::tc::prepare() != cudaSuccess) {
            cudaGetLastError();
            return TDB_ERR_CUDA;
        }
        g_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_addr[dev];
    return TDB_OK;
}

size_t up256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// Scale from a maximum (the same rules as tdb_split_gemm).
__global__ void k_scales(int fmt, const double* mx, float* s) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = 0; i < 2; ++i) {
        const double m = mx[i];
        float v = 1.0f;
        if (fmt == 0 && m > 0)
            v = static_cast<float>(ldexp(1.0, static_cast<int>(floor(log2(2048.0 / m)))));
        else if (fmt == 2)
            v = tdb::tc::pscale(m);
        s[i] = v;
    }
}

// Pieces of the transpose of B (K x N row-major, device) into Bt rows (N x ldk), with the
// arithmetic of the A pieces (tc::split_value on the scaled FP32 value); an overflowing
// piece sets err = 4.
template <int SCHEME>
__global__ void k_split_bt(int K, int N, const double* __restrict__ B, const float* __restrict__ s,
                           int bf16, uint16_t* p0, uint16_t* p1, uint16_t* p2, int ldk, int* err) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y * blockDim.y + threadIdx.y;
    if (k >= K || n >= N) return;
    uint16_t q[3];
    const bool ok = tdb::tc::split_value<SCHEME>(
        static_cast<float>(B[static_cast<size_t>(k) * N + n]) * s[1], bf16, q);
    const size_t o = static_cast<size_t>(n) * ldk + k;
    p0[o] = q[0];
    p1[o] = q[1];
    if (SCHEME == tdb::tc::kHead3) p2[o] = q[2];
    if (!ok) atomicCAS(err, 0, 4);
}

// C = FP32 product, or NaN everywhere when the device error flag is set
__global__ void k_finish(size_t n, const float* __restrict__ in, const int* __restrict__ err,
                         double* __restrict__ out) {
    const bool bad = *err != 0;
    for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<size_t>(gridDim.x) * blockDim.x)
        out[i] = bad ? __longlong_as_double(0x7ff8000000000000ll) : static_cast<double>(in[i]);
}

tdb_status fail(tdb_status st, const char* msg) {
    tdb::set_last_error(msg);
    return st;
}

}  // namespace

extern "C" tdb_status tdb_split_gemm_noalloc(int M, int N, int K, const double* A, const double* B,
                                             int fmt, double* C, void* stream) {
    if (M < 1 || N < 1 || K < 1 || M > 32768 || N > 32768 || K > 65536 || !A || !B || !C ||
        fmt < 0 || fmt > 2 || (fmt == 2 && K > 3 * tdb::tc::kHeadK))
        return fail(TDB_ERR_ARG, "tdb_split_gemm_noalloc: invalid sizes, pointers or format");
    const size_t ldk = (static_cast<size_t>(K) + 63) / 64 * 64;
    const int npc = fmt == 2 ? 3 : 2;
    // scratch layout: flags | maxima, scales | A pieces | Bt pieces | C (FP32)
    const size_t a_bytes = up256(2 * static_cast<size_t>(M) * ldk);
    const size_t b_bytes = up256(2 * static_cast<size_t>(N) * ldk);
    const size_t need = 512 + npc * (a_bytes + b_bytes) + up256(4 * static_cast<size_t>(M) * N);
    if (need > kScratchBytes)
        return fail(TDB_ERR_NOMEM,
                    "tdb_split_gemm_noalloc: M, N, K need more than the fixed 8 MiB scratch "
                    "(pieces of A and B^T plus an FP32 C); use tdb_split_gemm for larger products");
    unsigned char* base = nullptr;
    if (scratch_address(&base) != TDB_OK)
        return fail(TDB_ERR_CUDA,
                    "tdb_split_gemm_noalloc: looking up the scratch array on this device failed");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int* err = reinterpret_cast<int*>(base);
    double* mx = reinterpret_cast<double*>(base + 256);
    float* sc = reinterpret_cast<float*>(base + 256 + 2 * sizeof(double));
    uint16_t* ap[3] = {};
    uint16_t* bp[3] = {};
    unsigned char* q = base + 512;
    for (int i = 0; i < npc; ++i, q += a_bytes) ap[i] = reinterpret_cast<uint16_t*>(q);
    for (int i = 0; i < npc; ++i, q += b_bytes) bp[i] = reinterpret_cast<uint16_t*>(q);
    float* c32 = reinterpret_cast<float*>(q);
    // what must start at zero: the error flag and the two maxima
    if (cudaMemsetAsync(base, 0, 512, st) != cudaSuccess) {
        cudaGetLastError();
        return fail(TDB_ERR_CUDA, "tdb_split_gemm_noalloc: clearing the scratch flags failed");
    }
    tdb::launch_absmax(static_cast<size_t>(M) * K, A, mx, st, nullptr);
    tdb::launch_absmax(static_cast<size_t>(K) * N, B, mx + 1, st, nullptr);
    k_scales<<<1, 32, 0, st>>>(fmt, mx, sc);
    const int bf16 = fmt == 1 ? 1 : 0;
    const int scheme = fmt == 2 ? tdb::tc::kHead3 : tdb::tc::kHiLo;
    const int ld = static_cast<int>(ldk);
    tdb::tc::launch_split(scheme, M, K, A, K, 1.0f, 1, bf16, ap, ld, st, nullptr, sc, err);
    dim3 b(32, 8), g((K + 31) / 32, (N + 7) / 8);
    if (scheme == tdb::tc::kHead3)
        k_split_bt<tdb::tc::kHead3><<<g, b, 0, st>>>(K, N, B, sc, bf16, bp[0], bp[1], bp[2], ld, err);
    else
        k_split_bt<tdb::tc::kHiLo><<<g, b, 0, st>>>(K, N, B, sc, bf16, bp[0], bp[1], nullptr, ld, err);
    const cudaError_t e1 = cudaGetLastError();
    if (e1 != cudaSuccess)
        return fail(TDB_ERR_CUDA, "tdb_split_gemm_noalloc: launching the split kernels failed");
    tdb::tc::Maps maps{};
    for (int i = 0; i < npc; ++i)
        if (!tdb::tc::make_map(&maps.a[i], ap[i], M, K, ld, bf16) ||
            !tdb::tc::make_map(&maps.b[0][i], bp[i], N, K, ld, bf16))
            return fail(TDB_ERR_CUDA, "tdb_split_gemm_noalloc: cuTensorMapEncodeTiled failed");
    tdb::tc::GemmParams p{};
    p.M = M;
    p.N = N;
    p.part[0] = {0, 0, K, 0, c32, N, 1.0f, 1.0f, sc, sc + 1, 0};
    p.idesc = tdb::tc::idesc_f16(bf16);
    p.bf16 = bf16;
    p.err = err;
    if (tdb::tc::launch(scheme, maps, p, 1, st) != cudaSuccess) {
        cudaGetLastError();
        return fail(TDB_ERR_CUDA, "tdb_split_gemm_noalloc: launching the tensor-core product failed");
    }
    k_finish<<<256, 256, 0, st>>>(static_cast<size_t>(M) * N, c32, err, C);
    if (cudaGetLastError() != cudaSuccess)
        return fail(TDB_ERR_CUDA, "tdb_split_gemm_noalloc: launching the final conversion failed");
    return TDB_OK;
}
