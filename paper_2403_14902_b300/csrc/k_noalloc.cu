// Allocation-free FP32 MLP scoring: the same SIMT layer kernels as the
// query path, with the inter-layer activations in a fixed device array that
// lives in this library's module instead of memory from cudaMalloc.
//
// Who needs this: callers that must not allocate device memory once they
// are running.  A framework that owns the device memory pool may forbid
// allocations from outside it during its steps; a latency-bound service may
// not take the device-wide synchronisation and unbounded time a cudaMalloc
// can cost; a process that reserved nearly all device memory up front has
// nothing left to allocate from.  They pass their own inputs, weights and
// outputs; the library allocates nothing.
#include <cstdio>
#include <mutex>

#include "../../include/hydro.h"
#include "common.cuh"
#include "internal.h"

namespace hydro {
namespace {

// Two ping-pong activation buffers plus the row count the kernels read.
constexpr long long kNoAllocFloats = 1LL << 20;   // per buffer: 1,048,576 floats (4 MiB)
static __device__ __align__(256) float g_noalloc_scratch[2 * kNoAllocFloats + 64];

std::mutex g_noalloc_mu;
float *g_noalloc_ptr[64] = {};   // per device ordinal, from cudaGetSymbolAddress

__global__ void k_set_count(int *count, int n) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *count = n;
}

// scores[i] = (double)(s[i] + bias[0]): the last layer's bias, read on the
// device (the query path adds the same fp32 bias inside the dot kernel).
__global__ void k_add_bias_to_f64(const float *s, const float *bias, double *scores, int n) {
    const float b = *bias;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        scores[i] = (double)(s[i] + b);
}

hydro_status noalloc_fail(hydro_status s, const char *msg) {
    set_last_error(msg);
    return s;
}

}  // namespace
}  // namespace hydro

using namespace hydro;

extern "C" HYDRO_API hydro_status hydro_mlp_scores_noalloc(const float *d_x, int64_t n, int32_t n_layers,
                                                           const int32_t *dims, const float *const *d_weights,
                                                           const float *const *d_biases, double *d_scores,
                                                           void *stream) {
    set_last_error("");
    if (n < 0 || n_layers < 1 || n_layers > HYDRO_MAX_LAYERS || !dims || !d_weights || !d_biases)
        return noalloc_fail(HYDRO_EINVAL, "bad MLP description");
    if (n > 0 && (!d_x || !d_scores)) return noalloc_fail(HYDRO_EINVAL, "NULL tuples or scores");
    if (dims[n_layers] != 1) return noalloc_fail(HYDRO_EINVAL, "the last layer must have one output");
    long long wmax = 1;
    for (int l = 0; l <= n_layers; ++l) {
        if (dims[l] < 1) return noalloc_fail(HYDRO_EINVAL, "layer width must be >= 1");
        if (l > 0 && l < n_layers && dims[l] > wmax) wmax = dims[l];
    }
    for (int l = 0; l < n_layers; ++l)
        if (!d_weights[l] || !d_biases[l]) return noalloc_fail(HYDRO_EINVAL, "NULL weights");
    // n is bounded before any product is formed, so nothing here can overflow
    if (n > kNoAllocFloats || n > kNoAllocFloats / wmax)
        return noalloc_fail(HYDRO_EINVAL,
                            "n * widest hidden layer exceeds the static scratch of 1,048,576 floats per buffer");
    if (n == 0) return HYDRO_OK;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return noalloc_fail(HYDRO_ECUDA, "no current CUDA device");
    }
    float *base = nullptr;
    {
        // once per device, with that device current: device address of the
        // array.  The address is kept for the life of the process; after a
        // cudaDeviceReset of that device it is stale (the module is unloaded),
        // so callers must not reset a device they keep using this entry point on.
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return noalloc_fail(HYDRO_ECUDA, "cudaGetSymbolAddress of the static scratch failed");
            }
            g_noalloc_ptr[dev] = static_cast<float *>(p);
        }
        base = g_noalloc_ptr[dev];
    }
    int sms = 148;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        sms = 148;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float *act[2] = {base, base + kNoAllocFloats};
    int *count = reinterpret_cast<int *>(base + 2 * kNoAllocFloats);
    float *score32 = nullptr;   // the buffer the last layer writes; every branch below sets it
    const int rows = (int)n;
    // the row count is rewritten on every call before any kernel reads it
    k_set_count<<<1, 32, 0, st>>>(count, rows);
    const int K0 = dims[0];
    int cur = 0;
    if (n_layers == 1) {
        launch_mlp_dot_f32(count, nullptr, d_x, K0, d_weights[0], 0.f, K0, act[0], rows, sms, st);
        score32 = act[0];
    } else {
        launch_mlp_layer_f32(count, nullptr, d_x, K0, d_weights[0], d_biases[0], act[0], K0, dims[1], 1, rows, sms,
                             st);
        for (int l = 1; l + 1 < n_layers; ++l) {
            launch_mlp_layer_f32(count, nullptr, act[cur], dims[l], d_weights[l], d_biases[l], act[1 - cur], dims[l],
                                 dims[l + 1], 1, rows, sms, st);
            cur = 1 - cur;
        }
        const int L = n_layers - 1;
        score32 = act[1 - cur];
        launch_mlp_dot_f32(count, nullptr, act[cur], dims[L], d_weights[L], 0.f, dims[L], score32, rows, sms, st);
    }
    k_add_bias_to_f64<<<(rows + 255) / 256, 256, 0, st>>>(score32, d_biases[n_layers - 1], d_scores, rows);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(HYDRO_ECUDA, cudaGetErrorString(e));
    return HYDRO_OK;
}
