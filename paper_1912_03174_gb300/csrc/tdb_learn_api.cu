// C ABI of the per-atom shift network (the learned form): create, parameters, predict,
// gradient and Adam training, all on the GPU kernels of kern_learn.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "tdb.h"

namespace tdb {
void set_last_error(const char* msg);
namespace learn {
int n_params(int F, int H);
cudaError_t prepare(int F, int H);
void launch_forward(int F, int H, const float* params, const float* X, long n, float* Y,
                    cudaStream_t st);
void launch_grad(int F, int H, const float* params, const float* X, const float* Y, long n,
                 float scale, float* grad, double* sse, cudaStream_t st);
void launch_adam(int n, float* p, const float* g, float* m, float* v, float lr, float b1,
                 float b2, float c1, float c2, float eps, cudaStream_t st);
}  // namespace learn
}  // namespace tdb

struct tdb_shiftnet {
    int F = 0, H = 0, np = 0;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    double* sse = nullptr;
    float *X = nullptr, *Y = nullptr;
    long cap = 0;
    long t = 0;                  // Adam steps taken
    cudaStream_t st = nullptr;
};

namespace {

tdb_status fail(const char* msg, tdb_status s) {
    tdb::set_last_error(msg);
    return s;
}

// Device staging for n samples of X (n x F) and Y (n).
bool reserve(tdb_shiftnet* net, long n) {
    if (n <= net->cap) return true;
    cudaFree(net->X);
    cudaFree(net->Y);
    net->X = net->Y = nullptr;
    net->cap = 0;
    if (cudaMalloc(&net->X, sizeof(float) * n * net->F) != cudaSuccess ||
        cudaMalloc(&net->Y, sizeof(float) * n) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    net->cap = n;
    return true;
}

bool upload(tdb_shiftnet* net, const float* X, const float* Y, long n) {
    if (!reserve(net, n)) return false;
    if (cudaMemcpyAsync(net->X, X, sizeof(float) * n * net->F, cudaMemcpyHostToDevice, net->st) !=
        cudaSuccess)
        return false;
    if (Y && cudaMemcpyAsync(net->Y, Y, sizeof(float) * n, cudaMemcpyHostToDevice, net->st) !=
                 cudaSuccess)
        return false;
    return true;
}

}  // namespace

extern "C" {

tdb_status tdb_shiftnet_create(int n_features, int hidden, unsigned long long seed,
                               tdb_shiftnet** out) {
    if (!out || n_features < 1 || n_features > 32 || hidden < 1 || hidden > 64)
        return fail("tdb_shiftnet_create: need 1 <= n_features <= 32, 1 <= hidden <= 64",
                    TDB_ERR_ARG);
    *out = nullptr;
    tdb_shiftnet* net = new tdb_shiftnet();
    net->F = n_features;
    net->H = hidden;
    net->np = tdb::learn::n_params(n_features, hidden);
    const size_t b = sizeof(float) * net->np;
    bool ok = cudaStreamCreateWithFlags(&net->st, cudaStreamNonBlocking) == cudaSuccess &&
              cudaMalloc(&net->p, b) == cudaSuccess && cudaMalloc(&net->g, b) == cudaSuccess &&
              cudaMalloc(&net->m, b) == cudaSuccess && cudaMalloc(&net->v, b) == cudaSuccess &&
              cudaMalloc(&net->sse, sizeof(double)) == cudaSuccess &&
              tdb::learn::prepare(n_features, hidden) == cudaSuccess;
    if (ok) {
        // uniform weights in +-sqrt(3 / fan_in) (splitmix64 stream), zero biases
        std::vector<float> h(net->np, 0.f);
        uint64_t x = seed;
        auto u01 = [&]() {
            x += 0x9E3779B97F4A7C15ull;
            uint64_t z = x;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z ^= z >> 31;
            return static_cast<double>(z >> 11) * 0x1p-53;
        };
        const int F = n_features, H = hidden;
        auto fill = [&](int off, int count, int fan_in) {
            const double a = std::sqrt(3.0 / fan_in);
            for (int i = 0; i < count; ++i) h[off + i] = static_cast<float>((2.0 * u01() - 1.0) * a);
        };
        fill(0, F * H, F);                   // W1
        fill(F * H + H, H * H, H);           // W2
        fill(F * H + H + H * H + H, H, H);   // w3
        ok = cudaMemcpy(net->p, h.data(), b, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemset(net->m, 0, b) == cudaSuccess && cudaMemset(net->v, 0, b) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        tdb_shiftnet_destroy(net);
        return fail("tdb_shiftnet_create: CUDA setup failed", TDB_ERR_CUDA);
    }
    *out = net;
    return TDB_OK;
}

long tdb_shiftnet_param_count(const tdb_shiftnet* net) { return net ? net->np : 0; }

tdb_status tdb_shiftnet_get_params(tdb_shiftnet* net, float* params) {
    if (!net || !params) return fail("tdb_shiftnet_get_params: NULL argument", TDB_ERR_ARG);
    if (cudaMemcpy(params, net->p, sizeof(float) * net->np, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail("tdb_shiftnet_get_params: copy failed", TDB_ERR_CUDA);
    return TDB_OK;
}

tdb_status tdb_shiftnet_set_params(tdb_shiftnet* net, const float* params) {
    if (!net || !params) return fail("tdb_shiftnet_set_params: NULL argument", TDB_ERR_ARG);
    if (cudaMemcpy(net->p, params, sizeof(float) * net->np, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(net->m, 0, sizeof(float) * net->np) != cudaSuccess ||
        cudaMemset(net->v, 0, sizeof(float) * net->np) != cudaSuccess)
        return fail("tdb_shiftnet_set_params: copy failed", TDB_ERR_CUDA);
    net->t = 0;
    return TDB_OK;
}

tdb_status tdb_shiftnet_predict(tdb_shiftnet* net, const float* X, long n, float* Y) {
    if (!net || !X || !Y || n < 1) return fail("tdb_shiftnet_predict: bad arguments", TDB_ERR_ARG);
    if (!upload(net, X, nullptr, n)) return fail("tdb_shiftnet_predict: upload failed", TDB_ERR_CUDA);
    tdb::learn::launch_forward(net->F, net->H, net->p, net->X, n, net->Y, net->st);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(Y, net->Y, sizeof(float) * n, cudaMemcpyDeviceToHost, net->st) != cudaSuccess ||
        cudaStreamSynchronize(net->st) != cudaSuccess)
        return fail("tdb_shiftnet_predict: CUDA error", TDB_ERR_CUDA);
    return TDB_OK;
}

tdb_status tdb_shiftnet_gradient(tdb_shiftnet* net, const float* X, const float* Y, long n,
                                 float* grad, double* loss) {
    if (!net || !X || !Y || !grad || n < 1)
        return fail("tdb_shiftnet_gradient: bad arguments", TDB_ERR_ARG);
    if (!upload(net, X, Y, n)) return fail("tdb_shiftnet_gradient: upload failed", TDB_ERR_CUDA);
    double sse = 0.0;
    cudaMemsetAsync(net->g, 0, sizeof(float) * net->np, net->st);
    cudaMemsetAsync(net->sse, 0, sizeof(double), net->st);
    tdb::learn::launch_grad(net->F, net->H, net->p, net->X, net->Y, n, 1.0f / n, net->g, net->sse,
                            net->st);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(grad, net->g, sizeof(float) * net->np, cudaMemcpyDeviceToHost, net->st) !=
            cudaSuccess ||
        cudaMemcpyAsync(&sse, net->sse, sizeof(double), cudaMemcpyDeviceToHost, net->st) !=
            cudaSuccess ||
        cudaStreamSynchronize(net->st) != cudaSuccess)
        return fail("tdb_shiftnet_gradient: CUDA error", TDB_ERR_CUDA);
    if (loss) *loss = sse / n;
    return TDB_OK;
}

tdb_status tdb_shiftnet_train(tdb_shiftnet* net, const float* X, const float* Y, long n,
                              int epochs, long batch, float lr, double* loss_out) {
    if (!net || !X || !Y || n < 1 || epochs < 1 || batch < 1 || !(lr > 0))
        return fail("tdb_shiftnet_train: bad arguments", TDB_ERR_ARG);
    if (!upload(net, X, Y, n)) return fail("tdb_shiftnet_train: upload failed", TDB_ERR_CUDA);
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    double last = 0.0;
    for (int ep = 0; ep < epochs; ++ep) {
        cudaMemsetAsync(net->sse, 0, sizeof(double), net->st);
        for (long s = 0; s < n; s += batch) {
            const long nb = std::min(batch, n - s);
            cudaMemsetAsync(net->g, 0, sizeof(float) * net->np, net->st);
            tdb::learn::launch_grad(net->F, net->H, net->p, net->X + s * net->F, net->Y + s, nb,
                                    1.0f / nb, net->g, net->sse, net->st);
            ++net->t;
            const float c1 = 1.0f - std::pow(b1, static_cast<float>(net->t));
            const float c2 = 1.0f - std::pow(b2, static_cast<float>(net->t));
            tdb::learn::launch_adam(net->np, net->p, net->g, net->m, net->v, lr, b1, b2, c1, c2, eps,
                                    net->st);
        }
        if (ep == epochs - 1) {
            double sse = 0.0;
            if (cudaMemcpyAsync(&sse, net->sse, sizeof(double), cudaMemcpyDeviceToHost, net->st) !=
                    cudaSuccess ||
                cudaStreamSynchronize(net->st) != cudaSuccess)
                return fail("tdb_shiftnet_train: CUDA error", TDB_ERR_CUDA);
            last = sse / n;
        }
    }
    if (cudaGetLastError() != cudaSuccess) return fail("tdb_shiftnet_train: CUDA error", TDB_ERR_CUDA);
    if (loss_out) *loss_out = last;
    return TDB_OK;
}

void tdb_shiftnet_destroy(tdb_shiftnet* net) {
    if (!net) return;
    if (net->st) cudaStreamSynchronize(net->st);
    cudaFree(net->p);
    cudaFree(net->g);
    cudaFree(net->m);
    cudaFree(net->v);
    cudaFree(net->sse);
    cudaFree(net->X);
    cudaFree(net->Y);
    if (net->st) cudaStreamDestroy(net->st);
    delete net;
}

}  // extern "C"
