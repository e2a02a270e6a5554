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
#include <cmath>
#include <cstdint>
#include <mutex>

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
        if (tdb::tc::prepare() != cudaSuccess) return TDB_ERR_CUDA;
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

// Pieces of the transpose of B (K x N row-major, device) into Bt rows (N x ldk).
__global__ void k_split_bt(int K, int N, const double* __restrict__ B, const float* __restrict__ s,
                           int fmt, uint16_t* p0, uint16_t* p1, uint16_t* p2, int ldk) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y * blockDim.y + threadIdx.y;
    if (k >= K || n >= N) return;
    const double x = B[static_cast<size_t>(k) * N + n] * static_cast<double>(s[1]);
    const size_t o = static_cast<size_t>(n) * ldk + k;
    if (fmt == 2) {
        double h = rint(x);
        h = fmin(fmax(h, -127.0), 127.0);
        const double r = x - h;
        const __half rh = __double2half(r);
        p0[o] = __half_as_ushort(__double2half(h));
        p1[o] = __half_as_ushort(rh);
        p2[o] = __half_as_ushort(__double2half(r - static_cast<double>(__half2float(rh))));
    } else if (fmt == 1) {
        const float xf = static_cast<float>(x);
        const __nv_bfloat16 h = __float2bfloat16_rn(xf);
        p0[o] = __bfloat16_as_ushort(h);
        p1[o] = __bfloat16_as_ushort(__float2bfloat16_rn(xf - __bfloat162float(h)));
    } else {
        const float xf = static_cast<float>(x);
        const __half h = __float2half_rn(xf);
        p0[o] = __half_as_ushort(h);
        p1[o] = __half_as_ushort(__float2half_rn(xf - __half2float(h)));
    }
}

__global__ void k_f32_to_f64(size_t n, const float* __restrict__ in, double* __restrict__ out) {
    for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<size_t>(gridDim.x) * blockDim.x)
        out[i] = in[i];
}

}  // namespace

extern "C" tdb_status tdb_split_gemm_noalloc(int M, int N, int K, const double* A, const double* B,
                                             int fmt, double* C, void* stream) {
    if (M < 1 || N < 1 || K < 1 || !A || !B || !C || fmt < 0 || fmt > 2 ||
        (fmt == 2 && K > 3 * tdb::tc::kHeadK)) {
        tdb::set_last_error("tdb_split_gemm_noalloc: invalid sizes, pointers or format");
        return TDB_ERR_ARG;
    }
    const int ldk = (K + 63) / 64 * 64;
    const int npc = fmt == 2 ? 3 : 2;
    // scratch layout: flags | maxima, scales | A pieces | Bt pieces | C (FP32)
    const size_t a_bytes = up256(2ull * M * ldk), b_bytes = up256(2ull * N * ldk);
    const size_t need = 512 + npc * (a_bytes + b_bytes) + up256(4ull * M * N);
    if (need > kScratchBytes) {
        tdb::set_last_error(
            "tdb_split_gemm_noalloc: M, N, K need more than the fixed 8 MiB scratch "
            "(pieces of A and B^T plus an FP32 C); use tdb_split_gemm for larger products");
        return TDB_ERR_NOMEM;
    }
    unsigned char* base = nullptr;
    const tdb_status st0 = scratch_address(&base);
    if (st0 != TDB_OK) {
        tdb::set_last_error("tdb_split_gemm_noalloc: cudaGetSymbolAddress of the scratch failed");
        return st0;
    }
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
    if (cudaMemsetAsync(base, 0, 512, st) != cudaSuccess) return TDB_ERR_CUDA;
    tdb::launch_absmax(static_cast<size_t>(M) * K, A, mx, st, nullptr);
    tdb::launch_absmax(static_cast<size_t>(K) * N, B, mx + 1, st, nullptr);
    k_scales<<<1, 32, 0, st>>>(fmt, mx, sc);
    const int bf16 = fmt == 1 ? 1 : 0;
    const int scheme = fmt == 2 ? tdb::tc::kHead3 : tdb::tc::kHiLo;
    tdb::tc::launch_split(scheme, M, K, A, K, 1.0f, 1, bf16, ap, ldk, st, nullptr, sc, err);
    dim3 b(32, 8), g((K + 31) / 32, (N + 7) / 8);
    k_split_bt<<<g, b, 0, st>>>(K, N, B, sc, fmt, bp[0], bp[1], bp[2], ldk);
    if (cudaGetLastError() != cudaSuccess) return TDB_ERR_CUDA;
    tdb::tc::Maps maps{};
    for (int i = 0; i < npc; ++i)
        if (!tdb::tc::make_map(&maps.a[i], ap[i], M, K, ldk, bf16) ||
            !tdb::tc::make_map(&maps.b[0][i], bp[i], N, K, ldk, bf16))
            return TDB_ERR_CUDA;
    tdb::tc::GemmParams p{};
    p.M = M;
    p.N = N;
    p.part[0] = {0, 0, K, 0, c32, N, 1.0f, 1.0f, sc, sc + 1, 0};
    p.idesc = tdb::tc::idesc_f16(bf16);
    p.bf16 = bf16;
    p.err = err;
    if (tdb::tc::launch(scheme, maps, p, 1, st) != cudaSuccess) return TDB_ERR_CUDA;
    k_f32_to_f64<<<256, 256, 0, st>>>(static_cast<size_t>(M) * N, c32, C);
    if (cudaGetLastError() != cudaSuccess) return TDB_ERR_CUDA;
    return TDB_OK;
}
