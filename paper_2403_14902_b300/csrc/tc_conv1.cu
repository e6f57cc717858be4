// First conv layer of the CNN UDFs (uint8 CHW frames, up to 3 channels, 32
// output channels) on the tensor cores, for the BF16 path.
//
// out[m][p][co] = relu(b[co] + sum_{ci,ky,kx} W[co][ci][ky][kx] * f[ci][y+ky-1][x+kx-1] / 255)
//
// A 128-pixel tile (two image rows) is one MMA M; its im2col rows (27 taps,
// padded to K = 32) are built by the CTA's threads straight from the frame
// bytes into shared memory, as BF16 in the no-swizzle K-major core-matrix
// layout (8 rows x 16 bytes per core matrix).  The pixel values 0..255 are
// exact in BF16; 1/255 is folded into the BF16 weights.  Two kind::f16 MMAs
// (K = 16 each) accumulate 128 x 32 in TMEM; the epilogue adds the bias,
// applies ReLU and writes the BF16 NHWC row of each pixel (64 bytes).
#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace hydro {

namespace {

using namespace tcx;

constexpr int kC1Threads = 128;

// K-major, no swizzle: core matrices of 8 rows x 16 B, lbo bytes apart along
// K and sbo bytes apart along M/N.
__device__ __forceinline__ uint64_t desc_noswizzle(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Byte offset of element (row, k) of a [rows][32] BF16 tile: core matrix
// (row / 8, k / 8) at ((row / 8) * 4 + k / 8) * 128, row r at 16 r, element
// k % 8 at 2 (k % 8).  So lbo = 128 (next 8 k), sbo = 512 (next 8 rows).
__device__ __forceinline__ int core_off(int row, int k) {
    return ((row >> 3) * 4 + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__global__ void __launch_bounds__(kC1Threads) k_conv1_tc(const int *count, const int *list,
                                                         const unsigned char *frames, int C0, int H, int Wd,
                                                         const float *W, const float *bias, __nv_bfloat16 *out,
                                                         unsigned int *err) {
    __shared__ __align__(1024) unsigned char sA[128 * 64];
    __shared__ __align__(1024) unsigned char sB[32 * 64];
    __shared__ float sbias[32];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    const int t = threadIdx.x, warp = t >> 5;
    const int K = 9 * C0;
    for (int i = t; i < 32 * 32; i += kC1Threads) {
        const int co = i >> 5, k = i & 31;
        const float v = k < K ? W[co * K + k] * (1.0f / 255.0f) : 0.f;
        *reinterpret_cast<__nv_bfloat16 *>(sB + core_off(co, k)) = __float2bfloat16_rn(v);
    }
    if (t < 32) sbias[t] = bias[t];
    if (t == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(32u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const int M = *count, HW = H * Wd, tiles = HW / 128;
    constexpr uint32_t idesc = idesc_bf16(128, 32);
    uint32_t phase = 0;
    for (int w = blockIdx.x; w < M * tiles; w += gridDim.x) {
        const int m = w / tiles;
        const int p = (w % tiles) * 128 + t;
        const int y = p / Wd, x = p % Wd;
        const unsigned char *f = frames + (size_t)list[m] * C0 * HW;
        // this pixel's im2col row: k = ci*9 + ky*3 + kx, raw pixel values
        float v[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = 0.f;
#pragma unroll
        for (int ci = 0; ci < 3; ++ci) {
            if (ci >= C0) break;
#pragma unroll
            for (int ky = 0; ky < 3; ++ky) {
                const int yy = y + ky - 1;
                if (yy < 0 || yy >= H) continue;
                const unsigned char *row = f + (size_t)ci * HW + (size_t)yy * Wd;
#pragma unroll
                for (int kx = 0; kx < 3; ++kx) {
                    const int xx = x + kx - 1;
                    if (xx >= 0 && xx < Wd) v[ci * 9 + ky * 3 + kx] = (float)row[xx];
                }
            }
        }
#pragma unroll
        for (int kc = 0; kc < 4; ++kc) {
            uint4 q;
            q.x = pack_bf16x2(v[kc * 8 + 0], v[kc * 8 + 1]);
            q.y = pack_bf16x2(v[kc * 8 + 2], v[kc * 8 + 3]);
            q.z = pack_bf16x2(v[kc * 8 + 4], v[kc * 8 + 5]);
            q.w = pack_bf16x2(v[kc * 8 + 6], v[kc * 8 + 7]);
            *reinterpret_cast<uint4 *>(sA + core_off(t, kc * 8)) = q;
        }
        // the tile's rows are visible to the tensor core once every thread wrote them
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        if (t == 0) {
            tc_fence_after();
#pragma unroll
            for (int ks = 0; ks < 2; ++ks)
                mma_bf16(tmem, desc_noswizzle(smem_u32(sA) + ks * 256, 128, 512),
                         desc_noswizzle(smem_u32(sB) + ks * 256, 128, 512), idesc, ks > 0);
            mma_commit(&bar);
            volatile int *ab = &abort_flag;
            if (!mbar_wait(&bar, phase, ab)) {
                *ab = 1;
                atomicOr(err, ERR_TC_TIMEOUT);
            }
        }
        phase ^= 1u;
        __syncthreads();
        if (*(volatile int *)&abort_flag) break;
        tc_fence_after();
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), r);
        tmem_ld_wait();
        uint32_t pk[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            float a = __uint_as_float(r[2 * j]) + sbias[2 * j];
            float b = __uint_as_float(r[2 * j + 1]) + sbias[2 * j + 1];
            pk[j] = pack_bf16x2(a > 0.f ? a : 0.f, b > 0.f ? b : 0.f);
        }
        uint4 *dst = reinterpret_cast<uint4 *>(out + ((size_t)m * HW + p) * 32);
#pragma unroll
        for (int j = 0; j < 4; ++j) dst[j] = make_uint4(pk[4 * j], pk[4 * j + 1], pk[4 * j + 2], pk[4 * j + 3]);
        tc_fence_before();
        __syncthreads();   // TMEM and the A tile are reused by the next tile
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32u) : "memory");
    }
}

}  // namespace

bool tc_conv1_supported(int C0, int H, int W, int Cout) { return C0 >= 1 && C0 <= 3 && Cout == 32 && (H * W) % 128 == 0; }

void launch_conv1_tc(const int *count, const int *list, const unsigned char *frames, int C0, int H, int Wd,
                     const float *W, const float *bias, __nv_bfloat16 *out, int max_frames, int sms,
                     unsigned int *err, cudaStream_t st) {
    long long work = (long long)max_frames * (H * Wd / 128);
    int grid = (int)(work < (long long)sms * 8 ? work : (long long)sms * 8);
    if (grid < 1) grid = 1;
    k_conv1_tc<<<grid, kC1Threads, 0, st>>>(count, list, frames, C0, H, Wd, W, bias, out, err);
}

}  // namespace hydro
