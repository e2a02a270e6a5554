// C ABI of the tensor-core split GEMM on its own (validation and measurement).
#include <cmath>
#include <cstring>
#include <vector>

#include "tdb_internal.h"
#include "tdb_tc.h"

namespace {

float pow2_scale(const std::vector<double>& x, double target) {
    double m = 0;
    for (double v : x) m = std::fmax(m, std::fabs(v));
    if (!(m > 0)) return 1.0f;
    return static_cast<float>(std::ldexp(1.0, static_cast<int>(std::floor(std::log2(target / m)))));
}

}  // namespace

extern "C" tdb_status tdb_split_gemm(int M, int N, int K, const double* A, const double* B, int fmt,
                                     double* C, double* ms) {
    if (M < 1 || N < 1 || K < 1 || !A || !B || !C || fmt < 0 || fmt > 2 || M > 32768 ||
        N > 32768 || K > 65536 || (fmt == 2 && K > 3 * tdb::tc::kHeadK))
        return TDB_ERR_ARG;
    const int ldk = (K + 63) / 64 * 64;
    std::vector<double> a(A, A + static_cast<size_t>(M) * K), bt(static_cast<size_t>(N) * K);
    for (int k = 0; k < K; ++k)
        for (int n = 0; n < N; ++n) bt[static_cast<size_t>(n) * K + k] = B[static_cast<size_t>(k) * N + n];
    const int bf16 = fmt == 1 ? 1 : 0;
    const int scheme = fmt == 2 ? tdb::tc::kHead3 : tdb::tc::kHiLo;
    const int npc = fmt == 2 ? 3 : 2;
    float sa = 1.0f, sb = 1.0f;
    if (fmt == 0) {
        sa = pow2_scale(a, 2048.0);
        sb = pow2_scale(bt, 2048.0);
    } else if (fmt == 2) {
        double ma = 0, mb = 0;
        for (double v : a) ma = std::fmax(ma, std::fabs(v));
        for (double v : bt) mb = std::fmax(mb, std::fabs(v));
        sa = tdb::tc::pscale(ma);
        sb = tdb::tc::pscale(mb);
    }
    double *dA = nullptr, *dB = nullptr;
    uint16_t* ap[3] = {nullptr, nullptr, nullptr};
    uint16_t* bp[3] = {nullptr, nullptr, nullptr};
    float* dC = nullptr;
    int* err = nullptr;
    tdb_status rc = TDB_OK;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto ok = [&](cudaError_t e) {
        if (e != cudaSuccess && rc == TDB_OK) rc = TDB_ERR_CUDA;
        return e == cudaSuccess;
    };
    ok(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    ok(cudaMalloc(&dA, sizeof(double) * a.size()));
    ok(cudaMalloc(&dB, sizeof(double) * bt.size()));
    for (int q = 0; q < npc; ++q) {
        ok(cudaMalloc(&ap[q], 2ull * M * ldk));
        ok(cudaMalloc(&bp[q], 2ull * N * ldk));
    }
    ok(cudaMalloc(&dC, sizeof(float) * M * N));
    ok(cudaMalloc(&err, sizeof(int)));
    if (rc == TDB_OK) {
        for (int q = 0; q < npc; ++q) {
            ok(cudaMemsetAsync(ap[q], 0, 2ull * M * ldk, st));
            ok(cudaMemsetAsync(bp[q], 0, 2ull * N * ldk, st));
        }
        ok(cudaMemsetAsync(err, 0, sizeof(int), st));
        ok(cudaMemcpyAsync(dA, a.data(), sizeof(double) * a.size(), cudaMemcpyHostToDevice, st));
        ok(cudaMemcpyAsync(dB, bt.data(), sizeof(double) * bt.size(), cudaMemcpyHostToDevice, st));
        tdb::tc::launch_split(scheme, M, K, dA, K, sa, 1, bf16, ap, ldk, st, nullptr, nullptr, err);
        tdb::tc::launch_split(scheme, N, K, dB, K, sb, 1, bf16, bp, ldk, st, nullptr, nullptr, err);
        ok(cudaGetLastError());
    }
    tdb::tc::Maps maps{};
    for (int q = 0; q < npc && rc == TDB_OK; ++q)
        if (!(tdb::tc::make_map(&maps.a[q], ap[q], M, K, ldk, bf16) &&
              tdb::tc::make_map(&maps.b[0][q], bp[q], N, K, ldk, bf16)))
            rc = TDB_ERR_CUDA;
    if (rc == TDB_OK) {
        tdb::tc::GemmParams p{};
        p.M = M;
        p.N = N;
        p.part[0] = {0, 0, K, 0, dC, N, sa, sb, nullptr, nullptr, 0};
        p.idesc = tdb::tc::idesc_f16(bf16);
        p.bf16 = bf16;
        p.err = err;
        ok(tdb::tc::prepare());
        ok(cudaEventCreate(&e0));
        ok(cudaEventCreate(&e1));
        ok(cudaEventRecord(e0, st));
        ok(tdb::tc::launch(scheme, maps, p, 1, st));
        ok(cudaEventRecord(e1, st));
        ok(cudaStreamSynchronize(st));
        int h_err = 0;
        ok(cudaMemcpy(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost));
        if (rc == TDB_OK && h_err) rc = TDB_ERR_TIMEOUT;
        float t = 0;
        ok(cudaEventElapsedTime(&t, e0, e1));
        if (ms) *ms = t;
        std::vector<float> c(static_cast<size_t>(M) * N);
        ok(cudaMemcpy(c.data(), dC, sizeof(float) * c.size(), cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < c.size(); ++i) C[i] = c[i];
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(dA);
    cudaFree(dB);
    for (int q = 0; q < 3; ++q) {
        cudaFree(ap[q]);
        cudaFree(bp[q]);
    }
    cudaFree(dC);
    cudaFree(err);
    if (st) cudaStreamDestroy(st);
    return rc;
}
