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
//    the tile's 128 BF16 NHWC rows (64 B each) replace the A tile in shared
//    memory in the 64-byte swizzled layout (16-byte chunk j of row r at chunk
//    j ^ ((r >> 1) & 3)), so a warp's 16-byte stores hit distinct banks, and
//    one thread stores the tile with a TMA tensor store that writes it back
//    linear.  The A/output buffers alternate between tiles, so a tile's store
//    drains while the next one computes.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"
#include "tc_common.cuh"
#include "tc_conv.h"

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

// 128 output rows of 32 BF16 from shared memory to rows y .. y + 127
__device__ __forceinline__ void tma_store_rows(const CUtensorMap *map, uint32_t saddr, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(map),
                 "r"(saddr), "r"(0), "r"(y)
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

// n / d for 0 <= n < 2^22 through the FP32 reciprocal, corrected to the
// exact quotient (the FP32 estimate is off by at most one).
struct FDiv {
    int d;
    float inv;
    __device__ explicit FDiv(int d_) : d(d_), inv(1.0f / (float)d_) {}
    __device__ __forceinline__ int q(int n) const {
        int v = __float2int_rz((float)n * inv);
        const int r = n - v * d;
        v += (r >= d) - (r < 0);
        return v;
    }
};

// Copies the window of the tile at pixel p0 of frame `frame` into sw.  With
// vec (16-byte aligned frames, Wd a multiple of 16) the rows move as 16-byte
// cp.async, otherwise byte by byte.  A tile inside one row takes only
// columns x0 - 16 .. x0 + 143 of it.
template <int C0>
__device__ __forceinline__ void load_window(unsigned char *sw, const C1Geom &g, const FDiv &fw,
                                            const unsigned char *frames, int frame, int p0, bool vec) {
    const int y_first = fw.q(p0), y_last = fw.q(p0 + 127), R = y_last - y_first + 3;
    const int x0 = p0 - y_first * g.Wd;
    const bool single = y_first == y_last;
    const int c_lo = single ? max(0, x0 - 16) : 0, c_hi = single ? min(g.Wd, x0 + 144) : g.Wd;
    const unsigned char *f = frames + (size_t)frame * C0 * g.HW;
    const int per_row = vec ? (c_hi - c_lo) >> 4 : c_hi - c_lo, n = C0 * R * per_row;
    if ((int)threadIdx.x >= n) return;
    const FDiv fr(per_row);
    for (int i = threadIdx.x; i < n; i += kC1Threads) {
        const int rr = fr.q(i), c = c_lo + (i - rr * per_row) * (vec ? 16 : 1);
        const int ci = rr >= 2 * R ? 2 : rr >= R ? 1 : 0;
        const int r = rr - ci * R, yy = y_first - 1 + r;
        const bool in = yy >= 0 && yy < g.H;
        unsigned char *dst = sw + ci * g.CS + r * g.RS + 16 + c;
        const unsigned char *src = f + (size_t)ci * g.HW + (size_t)(in ? yy : 0) * g.Wd + c;
        if (vec) {
            if (in)
                cp_async16(smem_u32(dst), src);
            else
                *reinterpret_cast<uint4 *>(dst) = make_uint4(0, 0, 0, 0);
        } else {
            *dst = in ? *src : (unsigned char)0;
        }
    }
}

// Epilogue of one tile: accumulator columns tcol -> ReLU -> BF16 rows in the
// swizzled layout at sO.
__device__ __forceinline__ void store_rows(uint32_t tmem, int warp, int t, unsigned char *sO) {
    uint32_t r[32];
    tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), r);
    tmem_ld_wait();
    unsigned char *row = sO + t * 64;
    const int sw = (t >> 1) & 3;
#pragma unroll
    for (int j = 0; j < 4; ++j)
        *reinterpret_cast<uint4 *>(row + ((j ^ sw) << 4)) =
            make_uint4(relu_bf16x2(r[8 * j + 0], r[8 * j + 1]), relu_bf16x2(r[8 * j + 2], r[8 * j + 3]),
                       relu_bf16x2(r[8 * j + 4], r[8 * j + 5]), relu_bf16x2(r[8 * j + 6], r[8 * j + 7]));
}

// Tiles w = blockIdx.x + k * gridDim.x.  Iteration i builds tile i's A in
// buffer i % 3 and issues its MMA into accumulator i % 2, then runs tile
// i - 1's epilogue (its MMA has had a whole build to finish) into that
// tile's own buffer and stores it.  Buffer i % 3 was last stored from in
// iteration i - 2, so one outstanding store may still be reading.
template <int C0>
__global__ void __launch_bounds__(kC1Threads) k_conv1_tc(const __grid_constant__ CUtensorMap tmOut,
                                                         const int *count, const int *list,
                                                         const unsigned char *frames, int H, int Wd,
                                                         const uint4 *__restrict__ Bt, unsigned int *err, int vec) {
    constexpr int K = 9 * C0;
    extern __shared__ __align__(16) unsigned char dsm_raw[];
    // the swizzle pattern repeats every 512 bytes of shared address
    // aligned to 1 KB by pointer arithmetic on the shared array itself, so that the compiler
    // keeps every access through it in the shared state space (no generic loads or stores)
    unsigned char *dsm = dsm_raw + ((1024u - (smem_u32(dsm_raw) & 1023u)) & 1023u);
    unsigned char *sX = dsm;                        // [3][128 x 64 B]: A tile, then the output tile
    unsigned char *sB = dsm + 3 * 8192;             // [32 x 64 B]
    unsigned char *sWin = dsm + 3 * 8192 + 2048;    // [2][C0 x CS]
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    const int t = threadIdx.x, warp = t >> 5;
    const C1Geom g = c1_geom(H, Wd);
    const FDiv fw(Wd);
    // the packed FP16 weight tile, bias taps included (2 KB)
    for (int i = t; i < 2048 / 16; i += kC1Threads) reinterpret_cast<uint4 *>(sB)[i] = Bt[i];
    // zero both windows once: the border columns are never written again
    for (int i = t * 16; i < 2 * C0 * g.CS; i += kC1Threads * 16)
        *reinterpret_cast<uint4 *>(sWin + i) = make_uint4(0, 0, 0, 0);
    if (t == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(64u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();   // the zeroed windows before any row lands in them
    const int total = *count * g.tiles;
    const int G = gridDim.x, Gq = G / g.tiles, Gr = G - Gq * g.tiles;
    int m = blockIdx.x / g.tiles, j = blockIdx.x - m * g.tiles;   // frame slot and tile of w
    if (blockIdx.x < total) load_window<C0>(sWin, g, fw, frames, list[m], j * 128, vec != 0);
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
    uint32_t phase = 0;   // bit b: parity of accumulator b's next completion
    int it = 0, b3 = 0, prev_row = 0;
    bool aborted = false;
    for (int w = blockIdx.x; w < total; w += G, ++it) {
        const int b = it & 1;
        int mn = m + Gq, jn = j + Gr;
        if (jn >= g.tiles) {
            jn -= g.tiles;
            ++mn;
        }
        unsigned char *win = sWin + b * C0 * g.CS;
        // the other window was last read while building the previous tile's
        // A, which every thread finished before that tile's MMA
        if (w + G < total) load_window<C0>(sWin + (b ^ 1) * C0 * g.CS, g, fw, frames, list[mn], jn * 128, vec != 0);
        cp_async_commit();
        cp_async_wait1();   // this tile's window (committed one group earlier) has landed
        if (t == 0) bulk_wait_read1();   // buffer b3's store from two iterations back has been read out
        __syncthreads();
        const int p0 = j * 128, p = p0 + t;
        const int y = fw.q(p), x = p - y * Wd;
        // window byte of the pixel's top-left tap: row y - 1 is window row y - y_first
        const unsigned char *px = win + (y - fw.q(p0)) * g.RS + 15 + x;
        uint32_t u[K];
#pragma unroll
        for (int r = 0; r < 3 * C0; ++r)
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) u[r * 3 + kx] = px[roff[r] + kx];
        uint32_t a[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int k0 = 2 * q, k1 = 2 * q + 1;
            uint32_t v = 0;
            if (k0 < K) v |= 0x6400u | u[k0 < K ? k0 : 0];
            if (k1 < K) v |= (0x6400u | u[k1 < K ? k1 : 0]) << 16;
            if (k0 >= 29) v |= 0x3C00u;
            if (k1 >= 29) v |= 0x3C00u << 16;
            a[q] = v;
        }
        unsigned char *sA = sX + b3 * 8192;
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
                mma_bf16(tmem + b * 32, desc_noswizzle(smem_u32(sA) + ks * 256, 128, 512),
                         desc_noswizzle(smem_u32(sB) + ks * 256, 128, 512), idesc, ks > 0);
            mma_commit(&bar[b]);
        }
        if (it > 0) {
            // the previous tile: its accumulator, then its rows into its own buffer
            const int pb = b ^ 1, pb3 = b3 == 0 ? 2 : b3 - 1;
            if (!mbar_wait(&bar[pb], (phase >> pb) & 1u, &abort_flag)) {
                abort_flag = 1;
                atomicOr(err, ERR_TC_TIMEOUT);
            }
            phase ^= 1u << pb;
            tc_fence_after();
            store_rows(tmem + pb * 32, warp, t, sX + pb3 * 8192);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc_fence_before();
            __syncthreads();   // its rows are in place and its accumulator is free
            if (*(volatile int *)&abort_flag) {
                aborted = true;
                break;
            }
            if (t == 0) tma_store_rows(&tmOut, smem_u32(sX + pb3 * 8192), prev_row);
        }
        prev_row = m * g.HW + p0;
        m = mn;
        j = jn;
        b3 = b3 == 2 ? 0 : b3 + 1;
    }
    if (it > 0 && !aborted) {
        // the last tile's epilogue
        const int pb = (it - 1) & 1, pb3 = b3 == 0 ? 2 : b3 - 1;
        if (!mbar_wait(&bar[pb], (phase >> pb) & 1u, &abort_flag)) {
            abort_flag = 1;
            atomicOr(err, ERR_TC_TIMEOUT);
        }
        tc_fence_after();
        store_rows(tmem + pb * 32, warp, t, sX + pb3 * 8192);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        if (t == 0 && !*(volatile int *)&abort_flag) tma_store_rows(&tmOut, smem_u32(sX + pb3 * 8192), prev_row);
    }
    cp_async_wait0();
    if (t == 0) bulk_wait_all();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(64u) : "memory");
    }
}

size_t c1_smem_bytes(int C0, int H, int Wd) { return 1024 + 3 * 8192 + 2048 + 2 * (size_t)C0 * c1_geom(H, Wd).CS; }

}  // namespace

// B[co][k] = FP16(w[co][k] / 255) for k < 9 * C0, zero up to tap 28, and
// b[co] - 1024 * sum_k B[co][k] in three FP16 parts at taps 29..31, in the
// kernel's core-matrix order (2 KB).
void tc_conv1_pack_weights(const float *w, const float *b, int C0, std::vector<__half> &out) {
    const int K = 9 * C0;
    out.assign(32 * 32, __float2half_rn(0.f));
    auto at = [](int row, int k) { return (((row >> 3) * 4 + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2) / 2; };
    for (int co = 0; co < 32; ++co) {
        double off = 0.0;
        for (int k = 0; k < K; ++k) {
            const __half h = __float2half_rn(w[co * K + k] * (1.0f / 255.0f));
            off += 1024.0 * (double)__half2float(h);
            out[at(co, k)] = h;
        }
        double rb = (double)b[co] - off;
        for (int k = 29; k < 32; ++k) {
            const __half h = __float2half_rn((float)rb);
            rb -= (double)__half2float(h);
            out[at(co, k)] = h;
        }
    }
}

// Frames 8 to 512 columns wide (a window then fits well inside 48 KB) of
// fewer than 2^22 pixels (exact FP32-reciprocal division), batches of fewer
// than 2^31 pixels (32-bit tensor coordinates), and weights whose FP16 forms
// and 1024-offset bias stay far inside FP16 range.
bool tc_conv1_supported(int C0, int H, int W, int Cout, int max_frames, const float *w, const float *b) {
    if (!(C0 >= 1 && C0 <= 3 && Cout == 32 && W >= 8 && W <= 512 && (H * W) % 128 == 0 && H * W < (1 << 22) &&
          (long long)max_frames * H * W < (1LL << 31)))
        return false;
    for (int co = 0; co < 32; ++co) {
        double off = std::fabs((double)b[co]);
        for (int k = 0; k < 9 * C0; ++k) off += 1024.0 * std::fabs((double)w[co * 9 * C0 + k] / 255.0);
        if (!(off < 30000.0)) return false;
    }
    return true;
}

hydro_status launch_conv1_tc(TcConvPlan *plan, const int *count, const int *list, const unsigned char *frames,
                             int C0, int H, int Wd, const void *Bt, __nv_bfloat16 *out, int max_frames, int sms,
                             unsigned int *err, cudaStream_t st) {
    if (!plan->ready || (long long)max_frames * H * Wd >= (1LL << 31)) return HYDRO_EUNSUPPORTED;
    // the output as rows of 32 BF16 channels, one row per pixel, 128-row boxes
    CUtensorMap tmOut;
    {
        using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                      const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                      CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                      CUtensorMapFloatOOBfill);
        const cuuint64_t dims[2] = {32, (cuuint64_t)max_frames * H * Wd};
        const cuuint64_t strides[1] = {64};
        const cuuint32_t box[2] = {32, 128};
        const cuuint32_t es[2] = {1, 1};
        CUresult r = reinterpret_cast<EncodeFn>(plan->encode)(
            &tmOut, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, out, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return HYDRO_ECUDA;
    }
    const long long work = (long long)max_frames * (H * Wd / 128);
    const int vec = ((uintptr_t)frames & 15) == 0 && Wd % 16 == 0;
    const size_t smem = c1_smem_bytes(C0, H, Wd);
    // persistent: as many CTAs as fit on an SM (1 KB of shared memory is
    // reserved per CTA; 64 TMEM columns each allow 8), all resident
    const int per_sm = std::max(1, std::min(8, plan->smem_per_sm / (int)(smem + 1024)));
    const int grid = (int)std::max(1LL, std::min(work, (long long)sms * per_sm));
    auto run = [&](auto kern) {
        kern<<<grid, kC1Threads, smem, st>>>(tmOut, count, list, frames, H, Wd, (const uint4 *)Bt, err, vec);
    };
    if (C0 == 1)
        run(k_conv1_tc<1>);
    else if (C0 == 2)
        run(k_conv1_tc<2>);
    else
        run(k_conv1_tc<3>);
    return cudaPeekAtLastError() == cudaSuccess ? HYDRO_OK : HYDRO_ECUDA;
}

}  // namespace hydro
