// Shared device-side definitions of the CUDA path (not part of the C ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>

namespace hydro {

// Bits of the per-query device error word (latched, reported by poll).
enum : uint32_t {
    ERR_BAND_OVERFLOW = 1u << 0,   // an FP64 recheck band exceeded its capacity
    ERR_COUNT_RANGE = 1u << 1,     // a device count exceeded its buffer
    ERR_TC_TIMEOUT = 1u << 2,      // a tensor-core pipeline wait ran out
    ERR_TC_CONFIG = 1u << 3,       // a tensor-core kernel got an unsupported shape
    ERR_ID_RANGE = 1u << 4,        // a tuple id outside the reuse cache's capacity
};

constexpr int kMaxPred = 8;

// Per batch and predicate statistics row (device, int64).
struct StatRow {
    long long evaluated;
    long long passed;
    long long recheck_tf32;   // re-evaluated by the FP32-accurate 3xTF32 tensor-core path
    long long recheck32;      // re-evaluated in FP32 (CUDA cores)
    long long recheck64;      // re-evaluated in FP64
    long long hits;           // reuse-cache hits (shared upstream UDF outputs found cached)
    long long ns;             // measured cost: device time of the stage (0 unless measured)
};

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ double to_d(float v) { return (double)v; }
__device__ __forceinline__ double to_d(double v) { return v; }

template <typename T> __device__ __forceinline__ T from_f(float v);
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// v rounded to the nearest TF32 number (sign, 8 exponent bits, 10 explicit
// mantissa bits), ties to even, on the fp32 bit pattern (finite v).  The
// 3xTF32 split forms store hi = tf32_rne(x) and lo = tf32_rne(x - hi): both
// are exact TF32 values, so the tensor core drops no bits of them, and the
// rounding errors are unbiased (truncating instead biases every product of a
// long dot product the same way).
__host__ __device__ __forceinline__ float tf32_rne(float v) {
    uint32_t b;
    memcpy(&b, &v, sizeof b);
    b = (b + 0x0FFFu + ((b >> 13) & 1u)) & 0xFFFFE000u;
    float r;
    memcpy(&r, &b, sizeof r);
    return r;
}

// Exclusive prefix of one 0/1 flag per thread over a 1,024-thread block
// (nonzero counts as 1): a warp's flags are one __ballot_sync word, a lane's
// prefix is the popcount of the word's lower lanes, and warp 0 scans the 32
// warp totals.  Returns the thread's exclusive prefix and writes the block
// total to *total; every thread of the block must call it.
__device__ __forceinline__ int block_scan_flags_1024(int flag, int *total) {
    __shared__ int warp_sums[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned word = __ballot_sync(0xffffffffu, flag != 0);
    const int in_warp = __popc(word & ((1u << lane) - 1u));
    if (lane == 0) warp_sums[warp] = __popc(word);
    __syncthreads();
    if (warp == 0) {
        int w = warp_sums[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_sums[lane] = w;   // inclusive
    }
    __syncthreads();
    const int excl = in_warp + (warp ? warp_sums[warp - 1] : 0);
    *total = warp_sums[31];
    __syncthreads();
    return excl;
}

template <typename T> struct Acc { using type = float; };
template <> struct Acc<double> { using type = double; };

}  // namespace hydro
