// First conv layer of the CNN UDFs (uint8 CHW frames, up to 3 channels, 32
// output channels) on the tensor cores, for the BF16 path.
//
// out[m][p][co] = relu(b[co] + sum_{ci,ky,kx} W[co][ci][ky][kx] * f[ci][y+ky-1][x+kx-1] / 255)
//
// A 128-pixel tile is one MMA M, one pixel per thread and TMEM lane.
//  - Input window: the frame rows from one above the tile to one below it,
//    every channel, in shared memory with a zero column on each side and
//    zero rows outside the frame, so no tap needs a bounds check.  The
//    window of the CTA's next tile is copied with 16-byte cp.async while the
//    current tile computes.
//  - Operands: each pixel byte b enters as the FP16 number 1024 + b, whose
//    bit pattern is 0x6400 | b (the FP16 step between 1024 and 2048 is 1), so
//    the im2col row takes integer ops only.  The weights are FP16(W / 255).
//    The constant 1024 * sum_k W'[co][k] is taken out of the bias; the
//    remaining bias, split into three FP16 parts, rides in taps 29..31 whose
//    A value is 1.  Taps 27..28 (and 9 * C0 .. 28 for fewer channels) are
//    zero.  Products of FP16 values are exact and accumulate in FP32 (K = 32,
//    two kind::f16 MMAs), so the result carries the FP16 rounding of W / 255
//    and FP32 accumulation error of about 2^-24 times the 1024-offset sum.
//  - Epilogue: ReLU and rounding to BF16 in one conversion per channel pair;
//    the tile's 128 BF16 NHWC rows (8 KB, contiguous in the output) replace
//    the A tile in shared memory and one thread stores them with a bulk copy.
//    The A/output buffers alternate between tiles, so a tile's store drains
//    while the next one computes.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>

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

// Window of a tile: rows y_first - 1 .. y_last + 1 of every channel, at
// most 127 / Wd + 4 rows of RS = Wd + 32 bytes (rounded up to 16); column x
// of a row sits at byte 16 + x, so bytes 15 and 16 + Wd are the zero border.
struct C1Geom {
    int H, Wd, HW, tiles, RS, CS;
};

__host__ __device__ inline C1Geom c1_geom(int H, int Wd) {
    C1Geom g;
    g.H = H;
    g.Wd = Wd;
    g.HW = H * Wd;
    g.tiles = g.HW / 128;
    g.RS = (Wd + 32 + 15) & ~15;
    g.CS = (127 / Wd + 4) * g.RS;
    return g;
}

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void *g) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void bulk_store(void *g, uint32_t saddr, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(g), "r"(saddr), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// relu(lo), relu(hi) rounded to BF16 and packed (lo in the low half)
__device__ __forceinline__ uint32_t relu_bf16x2(uint32_t lo, uint32_t hi) {
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(__uint_as_float(hi)), "f"(__uint_as_float(lo)));
    return d;
}

// Copies tile w's window into sw.  With vec (16-byte aligned frames, Wd a
// multiple of 16) the rows move as 16-byte cp.async, otherwise byte by byte.
// A tile inside one row takes only columns x0 - 16 .. x0 + 143 of it.
template <int C0>
__device__ __forceinline__ void load_window(unsigned char *sw, const C1Geom &g, const unsigned char *frames,
                                            const int *list, int w, bool vec) {
    const int m = w / g.tiles, p0 = (w % g.tiles) * 128;
    const int y_first = p0 / g.Wd, y_last = (p0 + 127) / g.Wd, R = y_last - y_first + 3;
    const int x0 = p0 - y_first * g.Wd;
    const bool single = y_first == y_last;
    const int c_lo = single ? max(0, x0 - 16) : 0, c_hi = single ? min(g.Wd, x0 + 144) : g.Wd;
    const unsigned char *f = frames + (size_t)list[m] * C0 * g.HW;
    if (vec) {
        const int n16 = (c_hi - c_lo) >> 4, per_ch = R * n16;
        for (int i = threadIdx.x; i < C0 * per_ch; i += kC1Threads) {
            const int ci = i / per_ch, rem = i - ci * per_ch, r = rem / n16, c = c_lo + (rem - r * n16) * 16;
            const int yy = y_first - 1 + r;
            unsigned char *dst = sw + ci * g.CS + r * g.RS + 16 + c;
            if (yy >= 0 && yy < g.H)
                cp_async16(smem_u32(dst), f + (size_t)ci * g.HW + (size_t)yy * g.Wd + c);
            else
                *reinterpret_cast<uint4 *>(dst) = make_uint4(0, 0, 0, 0);
        }
    } else {
        const int n = c_hi - c_lo, per_ch = R * n;
        for (int i = threadIdx.x; i < C0 * per_ch; i += kC1Threads) {
            const int ci = i / per_ch, rem = i - ci * per_ch, r = rem / n, c = c_lo + (rem - r * n);
            const int yy = y_first - 1 + r;
            sw[ci * g.CS + r * g.RS + 16 + c] =
                (yy >= 0 && yy < g.H) ? f[(size_t)ci * g.HW + (size_t)yy * g.Wd + c] : (unsigned char)0;
        }
    }
}

template <int C0>
__global__ void __launch_bounds__(kC1Threads) k_conv1_tc(const int *count, const int *list,
                                                         const unsigned char *frames, int H, int Wd,
                                                         const float *W, const float *bias, __nv_bfloat16 *out,
                                                         unsigned int *err, int vec) {
    constexpr int K = 9 * C0;
    extern __shared__ __align__(1024) unsigned char dsm[];
    unsigned char *sX = dsm;                    // [2][128 x 64 B]: A tile, then the output tile
    unsigned char *sB = dsm + 2 * 8192;         // [32 x 64 B]
    unsigned char *sWin = dsm + 2 * 8192 + 2048;   // [2][C0 x CS]
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    const int t = threadIdx.x, warp = t >> 5;
    const C1Geom g = c1_geom(H, Wd);
    // weights: B[co][k] = FP16(W[co][k] / 255) for k < K, zero up to tap 28,
    // and the bias less 1024 * sum_k B[co][k] in three FP16 parts at 29..31
    if (t < 32) {
        const int co = t;
        double off = 0.0;
        for (int k = 0; k < 29; ++k) {
            const __half h = __float2half_rn(k < K ? W[co * K + k] * (1.0f / 255.0f) : 0.f);
            off += 1024.0 * (double)__half2float(h);
            *reinterpret_cast<__half *>(sB + core_off(co, k)) = h;
        }
        double rb = (double)bias[co] - off;
        for (int k = 29; k < 32; ++k) {
            const __half h = __float2half_rn((float)rb);
            rb -= (double)__half2float(h);
            *reinterpret_cast<__half *>(sB + core_off(co, k)) = h;
        }
    }
    // zero both windows once: the border columns are never written again
    for (int i = t * 16; i < 2 * C0 * g.CS; i += kC1Threads * 16)
        *reinterpret_cast<uint4 *>(sWin + i) = make_uint4(0, 0, 0, 0);
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
    __syncthreads();   // the zeroed windows before any row lands in them
    const int total = *count * g.tiles;
    if (blockIdx.x < total) load_window<C0>(sWin, g, frames, list, blockIdx.x, vec != 0);
    cp_async_commit();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    constexpr uint32_t idesc = idesc_f16(128, 32);
    // the 3 x C0 tap rows of a pixel, relative to its own window byte
    int roff[3 * C0];
#pragma unroll
    for (int ci = 0; ci < C0; ++ci)
#pragma unroll
        for (int ky = 0; ky < 3; ++ky) roff[ci * 3 + ky] = ci * g.CS + ky * g.RS;
    uint32_t phase = 0;
    int it = 0;
    for (int w = blockIdx.x; w < total; w += gridDim.x, ++it) {
        const int b = it & 1;
        const int wn = w + gridDim.x;
        unsigned char *win = sWin + b * C0 * g.CS;
        // the other window was last read while building the previous tile's
        // A, which every thread finished before that tile's MMA
        if (wn < total) load_window<C0>(sWin + (b ^ 1) * C0 * g.CS, g, frames, list, wn, vec != 0);
        cp_async_commit();
        cp_async_wait1();   // this tile's window (committed one group earlier) has landed
        if (t == 0) bulk_wait_read1();   // sX[b]'s store from two tiles back has been read out
        __syncthreads();
        const int m = w / g.tiles, p0 = (w % g.tiles) * 128;
        const int p = p0 + t;
        const int y = p / Wd, x = p - y * Wd;
        // window byte of the pixel's top-left tap: row y - 1 is window row y - y_first
        const unsigned char *px = win + (y - p0 / Wd) * g.RS + 15 + x;
        uint32_t u[K];
#pragma unroll
        for (int r = 0; r < 3 * C0; ++r)
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) u[r * 3 + kx] = px[roff[r] + kx];
        uint32_t a[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int k0 = 2 * j, k1 = 2 * j + 1;
            uint32_t v = 0;
            if (k0 < K) v |= 0x6400u | u[k0 < K ? k0 : 0];
            if (k1 < K) v |= (0x6400u | u[k1 < K ? k1 : 0]) << 16;
            if (k0 >= 29) v |= 0x3C00u;
            if (k1 >= 29) v |= 0x3C00u << 16;
            a[j] = v;
        }
        unsigned char *sA = sX + b * 8192;
#pragma unroll
        for (int kc = 0; kc < 4; ++kc)
            *reinterpret_cast<uint4 *>(sA + core_off(t, kc * 8)) =
                make_uint4(a[kc * 4 + 0], a[kc * 4 + 1], a[kc * 4 + 2], a[kc * 4 + 3]);
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
        // the MMA has read sA, so the tile's output rows (pixel-major, 64 B
        // each) take its place
        uint4 *dst = reinterpret_cast<uint4 *>(sA + t * 64);
#pragma unroll
        for (int j = 0; j < 4; ++j)
            dst[j] = make_uint4(relu_bf16x2(r[8 * j + 0], r[8 * j + 1]), relu_bf16x2(r[8 * j + 2], r[8 * j + 3]),
                                relu_bf16x2(r[8 * j + 4], r[8 * j + 5]), relu_bf16x2(r[8 * j + 6], r[8 * j + 7]));
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();   // TMEM is free for the next tile and the output rows are in place
        if (t == 0) bulk_store(out + ((size_t)m * g.HW + p0) * 32, smem_u32(sA), 128 * 64);
    }
    cp_async_wait0();
    if (t == 0) bulk_wait_all();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32u) : "memory");
    }
}

size_t c1_smem_bytes(int C0, int H, int Wd) { return 2 * 8192 + 2048 + 2 * (size_t)C0 * c1_geom(H, Wd).CS; }

}  // namespace

// Frames 8 to 512 columns wide (a window then fits well inside 48 KB), and
// weights whose FP16 forms and 1024-offset bias stay far inside FP16 range.
bool tc_conv1_supported(int C0, int H, int W, int Cout, const float *w, const float *b) {
    if (!(C0 >= 1 && C0 <= 3 && Cout == 32 && W >= 8 && W <= 512 && (H * W) % 128 == 0)) return false;
    for (int co = 0; co < 32; ++co) {
        double off = std::fabs((double)b[co]);
        for (int k = 0; k < 9 * C0; ++k) off += 1024.0 * std::fabs((double)w[co * 9 * C0 + k] / 255.0);
        if (!(off < 30000.0)) return false;
    }
    return true;
}

void launch_conv1_tc(const int *count, const int *list, const unsigned char *frames, int C0, int H, int Wd,
                     const float *W, const float *bias, __nv_bfloat16 *out, int max_frames, int sms,
                     unsigned int *err, cudaStream_t st) {
    long long work = (long long)max_frames * (H * Wd / 128);
    int grid = (int)(work < (long long)sms * 8 ? work : (long long)sms * 8);
    if (grid < 1) grid = 1;
    const int vec = ((uintptr_t)frames & 15) == 0 && Wd % 16 == 0;
    const size_t smem = c1_smem_bytes(C0, H, Wd);
    if (C0 == 1)
        k_conv1_tc<1><<<grid, kC1Threads, smem, st>>>(count, list, frames, H, Wd, W, bias, out, err, vec);
    else if (C0 == 2)
        k_conv1_tc<2><<<grid, kC1Threads, smem, st>>>(count, list, frames, H, Wd, W, bias, out, err, vec);
    else
        k_conv1_tc<3><<<grid, kC1Threads, smem, st>>>(count, list, frames, H, Wd, W, bias, out, err, vec);
}

}  // namespace hydro
