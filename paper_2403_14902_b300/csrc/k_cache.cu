// Reuse cache of a shared upstream UDF's outputs, keyed by tuple id (the
// materialized UDF results a predicate reuses, Sec. 2.1; reuse-aware routing,
// Sec. 4.3): a dense device array values[id][D] plus tags[id]
// (0 absent, -1 prefilled before the query, b+1 computed by batch b).
#include "common.cuh"
#include "internal.h"

namespace hydro {

constexpr int kProbeThreads = 1024;

// Alive tuples whose id is not cached yet, in alive-list order.
__global__ void __launch_bounds__(kProbeThreads)
k_cache_probe_miss(const int *count_in, const int *list_in, const long long *ids, const int *tags, long long cap,
                   int *miss_list, int *miss_count, unsigned int *err) {
    const int n = *count_in;
    int base = 0;
    // four chunks of 1,024 entries: their dependent loads (list, id, tag) are
    // in flight together, then the four scans run back to back
    constexpr int K = 4;
    for (int m0 = 0; m0 < n; m0 += K * kProbeThreads) {
        int lv[K], miss[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int m = m0 + k * kProbeThreads + threadIdx.x;
            lv[k] = m < n ? list_in[m] : -1;
        }
        long long idv[K];
#pragma unroll
        for (int k = 0; k < K; ++k) idv[k] = lv[k] >= 0 ? ids[lv[k]] : 0;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            miss[k] = 0;
            if (lv[k] >= 0) {
                if (idv[k] < 0 || idv[k] >= cap) atomicOr(err, ERR_ID_RANGE);
                else miss[k] = tags[idv[k]] == 0;
            }
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            int total;
            const int pos = base + block_scan_flags_1024(miss[k], &total);
            if (miss[k]) miss_list[pos] = lv[k];
            base += total;
        }
    }
    if (threadIdx.x == 0) *miss_count = base;
}

// values[ids[miss_list[j]]][:] = src[j][:], tags[...] = tag_value.
__global__ void k_cache_store(const int *miss_count, const int *miss_list, const long long *ids, const float *src,
                              int D, float *values, int *tags, int tag_value) {
    const int n = *miss_count;
    const int per_row = D / 4;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)n * per_row;
         i += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(i / per_row), q = (int)(i % per_row);
        const long long id = ids[miss_list[j]];
        reinterpret_cast<float4 *>(values + (size_t)id * D)[q] = reinterpret_cast<const float4 *>(src + (size_t)j * D)[q];
        if (q == 0) tags[id] = tag_value;
    }
}

// Misses the router sees for a batch: ids neither prefilled nor computed by
// a batch <= last (the batches whose statistics the router may use).
__global__ void k_probe_visible(const long long *ids, int n, const int *tags, long long cap, long long last,
                                int *out_miss) {
    __shared__ int block_miss;
    if (threadIdx.x == 0) block_miss = 0;
    __syncthreads();
    int miss = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const long long id = ids[i];
        if (id < 0 || id >= cap) continue;
        const int t = tags[id];
        const bool visible = t == -1 || (t > 0 && (long long)(t - 1) <= last);
        miss += visible ? 0 : 1;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) miss += __shfl_xor_sync(0xffffffffu, miss, o);
    if ((threadIdx.x & 31) == 0 && miss) atomicAdd(&block_miss, miss);
    __syncthreads();
    if (threadIdx.x == 0 && block_miss) atomicAdd(out_miss, block_miss);
}

void launch_cache_probe_miss(const int *count_in, const int *list_in, const long long *ids, const int *tags,
                             long long cap, int *miss_list, int *miss_count, unsigned int *err, cudaStream_t st) {
    k_cache_probe_miss<<<1, kProbeThreads, 0, st>>>(count_in, list_in, ids, tags, cap, miss_list, miss_count, err);
}

void launch_cache_store(const int *miss_count, const int *miss_list, const long long *ids, const float *src, int D,
                        float *values, int *tags, int tag_value, int max_rows, int sms, cudaStream_t st) {
    long long work = (long long)max_rows * (D / 4);
    int grid = (int)((work + 255) / 256);
    if (grid > sms * 8) grid = sms * 8;
    if (grid < 1) grid = 1;
    k_cache_store<<<grid, 256, 0, st>>>(miss_count, miss_list, ids, src, D, values, tags, tag_value);
}

void launch_probe_visible(const long long *ids, int n, const int *tags, long long cap, long long last, int *out_miss,
                          cudaStream_t st) {
    int grid = (n + 255) / 256;
    if (grid > 64) grid = 64;
    if (grid < 1) grid = 1;
    k_probe_visible<<<grid, 256, 0, st>>>(ids, n, tags, cap, last, out_miss);
}

}  // namespace hydro
