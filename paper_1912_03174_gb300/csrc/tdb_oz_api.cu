// tdb_slice_gemm: the FP64-accurate integer-slice tensor-core product on its own
// (validation and measurement), with its own device buffers.
#include <cuda_runtime.h>

#include <cstdint>

#include "tdb.h"
#include "tdb_oz.h"

namespace tdb {
void set_last_error(const char* msg);
}

extern "C" tdb_status tdb_slice_gemm(int M, int N, int K, const double* A, const double* B,
                                     double* C, double* ms) {
    namespace oz = tdb::oz;
    if (M < 1 || N < 1 || K < 1 || !A || !B || !C || M > 32768 || N > 32768 || K > oz::kMaxK) {
        tdb::set_last_error("tdb_slice_gemm: invalid sizes or pointers (K <= 4096)");
        return TDB_ERR_ARG;
    }
    tdb_status rc = TDB_OK;
    auto ok = [&](cudaError_t e) {
        if (e != cudaSuccess && rc == TDB_OK) rc = TDB_ERR_CUDA;
        return e == cudaSuccess;
    };
    double *dA = nullptr, *dB = nullptr, *dC = nullptr, *colmax = nullptr;
    void *bufA = nullptr, *bufB = nullptr;
    int* err = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ok(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    ok(cudaMalloc(&dA, sizeof(double) * M * K));
    ok(cudaMalloc(&dB, sizeof(double) * K * N));
    ok(cudaMalloc(&dC, sizeof(double) * M * N));
    ok(cudaMalloc(&colmax, sizeof(double) * N));
    ok(cudaMalloc(&bufA, oz::sliced_bytes(M, K)));
    ok(cudaMalloc(&bufB, oz::sliced_bytes(N, K)));
    ok(cudaMalloc(&err, sizeof(int)));
    ok(cudaEventCreate(&e0));
    ok(cudaEventCreate(&e1));
    oz::Sliced sa, sb;
    if (rc == TDB_OK &&
        (!oz::sliced_init(sa, bufA, M, K, 128) || !oz::sliced_init(sb, bufB, N, K, 64)))
        rc = TDB_ERR_CUDA;
    if (rc == TDB_OK) {
        ok(oz::prepare());
        ok(cudaMemsetAsync(err, 0, sizeof(int), st));
        ok(cudaMemcpyAsync(dA, A, sizeof(double) * M * K, cudaMemcpyHostToDevice, st));
        ok(cudaMemcpyAsync(dB, B, sizeof(double) * K * N, cudaMemcpyHostToDevice, st));
        oz::slice_rows(dA, K, 1.0, sa, st);
        oz::slice_cols(dB, N, sb, colmax, st);
        ok(cudaGetLastError());
        oz::Part part;
        part.b = &sb;
        part.C = dC;
        part.ldc = N;
        ok(cudaEventRecord(e0, st));
        ok(oz::gemm(sa, &part, 1, err, st));
        ok(cudaEventRecord(e1, st));
        ok(cudaMemcpyAsync(C, dC, sizeof(double) * M * N, cudaMemcpyDeviceToHost, st));
        int h_err = 0;
        ok(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st));
        ok(cudaStreamSynchronize(st));
        if (rc == TDB_OK && h_err != 0) {
            tdb::set_last_error("tdb_slice_gemm: a bounded device wait timed out");
            rc = TDB_ERR_TIMEOUT;
        }
        float t = 0.f;
        if (rc == TDB_OK && ms && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess) *ms = t;
    }
    if (rc == TDB_ERR_CUDA) tdb::set_last_error("tdb_slice_gemm: CUDA error");
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dC);
    cudaFree(colmax);
    cudaFree(bufA);
    cudaFree(bufB);
    cudaFree(err);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    return rc;
}
