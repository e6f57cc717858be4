// BF16 conv3x3 (stride 1, zero pad 1) + bias + ReLU on the 5th-generation
// tensor cores: tcgen05.mma with the accumulator in TMEM, operands staged in
// shared memory by TMA, warp-specialised and persistent.
//
// Implicit GEMM per CTA tile: M = 128 output pixels (two 64-pixel image rows
// of one frame), N = Cout (64 or 128), K = 9 taps x Cin.  For one chunk of
// CC input channels and one horizontal tap kx, a single 4-D TMA box
// {CC channels, 64 px, 4 rows, 1 frame} at (c0, kx-1, y0-1, frame) holds the
// input rows y0-1 .. y0+2 shifted by kx-1; the three vertical taps ky are the
// 128-row windows starting at rows 64*ky of that box, so one load serves
// three taps.  Out-of-range coordinates are zero-filled by TMA, which is the
// conv's zero padding.  The matching weights are one 3-D TMA box
// {CC, Cout, 3 taps}.
//
// Roles (192 threads): warp 0 issues TMA, warp 1 owns TMEM and issues the
// MMAs, warps 2-5 drain the accumulator (bias, ReLU, BF16, NHWC store).  Two
// TMEM accumulators let the epilogue of one tile overlap the MMAs of the
// next.  Every mbarrier wait is bounded by the global timer; on expiry the
// CTA raises ERR_TC_TIMEOUT, drains its issued copies and frees TMEM.
#include <cuda.h>

#include <cstdio>
#include <cstring>
#include <string>

#include "common.cuh"
#include "tc_common.cuh"
#include "tc_conv.h"

namespace hydro {

namespace {

using namespace tcx;
thread_local std::string g_tc_err;
// MT: 128-pixel subtiles per CTA tile (2 or 4).  One A box of 2 + 2 MT image
// rows feeds all subtiles and every B box is used MT times, which cuts the
// L2->SM operand traffic per output pixel (the 64-output layers, whose double-
// buffered accumulators fit TMEM at MT = 4, are the most operand-bound).
// MODE: 0 BF16; 1 3xTF32 (fp32 [hi | lo] TF32 planes, kind::tf32); 2 split
// BF16 ([hi | lo] BF16 planes, kind::f16).  Modes 1 and 2 run three passes
// (A hi, B hi), (A hi, B lo), (A lo, B hi) into one accumulator.
template <int CC, int N, int S, int MODE, int MT>
struct TcCfg {
    static constexpr bool SPLIT = MODE != 0;
    static constexpr int ESZ = MODE == 1 ? 4 : 2;         // operand bytes
    static constexpr int ROWB = CC * ESZ;                 // bytes of one pixel's K chunk
    static constexpr int A_ROWS = 2 + 2 * MT;             // image rows per A box (halo included)
    static constexpr int A_BYTES = A_ROWS * 64 * ROWB;
    static constexpr int B_TAP = N * ROWB;                // one tap's weights
    static constexpr int B_BYTES = 3 * B_TAP;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr uint32_t SWZ = ROWB == 128 ? 2u : 4u;  // 128B or 64B swizzle
    static constexpr uint32_t SBO = 8 * ROWB;              // 8-row group stride
    static constexpr int TMEM_COLS = 2 * MT * N;          // double-buffered accumulators
    static constexpr int PASSES = SPLIT ? 3 : 1;
    // staging of the stores: BF16 32 pixel rows a warp; split BF16 32 pixels x 128 B (one channel group)
    static constexpr int EPI_STG = MODE == 0 ? 4 * 32 * N * 2 : MODE == 2 ? 4 * 32 * 128 : 0;
    static constexpr int SMEM = S * STAGE + 1024 /*align*/ + 256 /*barriers*/ + EPI_STG;
    static_assert(SMEM <= 227 * 1024, "shared memory per CTA");
};

template <int CC, int N, int S, int MODE, int MT>
__global__ void __launch_bounds__(192, 1)
k_conv3x3_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const int *count,
             int nchunks, int cin, int tiles_per_frame, int HW, const float *__restrict__ bias, void *out,
             const float *__restrict__ head_w, float *partials, unsigned int *err) {
    using C = TcCfg<CC, N, S, MODE, MT>;
    extern __shared__ unsigned char smem_raw[];
    // aligned to 1 KB by pointer arithmetic on the shared array itself, so that the compiler
    // keeps every access through it in the shared state space (no generic loads or stores)
    unsigned char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + S * C::STAGE);
    uint64_t *empty = full + S;
    uint64_t *tfull = empty + S;
    uint64_t *tempty = tfull + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tempty + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    uint4 *stg_all = reinterpret_cast<uint4 *>(smem + S * C::STAGE + 256);   // C::EPI_STG bytes

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int total = (*count) * tiles_per_frame;
    const int ksteps = C::PASSES * nchunks * 3;
    // a CTA without tiles takes neither barriers nor TMEM (small recheck
    // bands leave most of the grid idle)
    if ((int)blockIdx.x >= total) return;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 4);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)C::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer
            int s = 0;
            uint32_t ph = 0;
            uint32_t issued = 0, last_par = 0;   // per stage bit: load in flight, its parity
            bool ok = true;
            for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
                const int m = t / tiles_per_frame;
                const int y0 = (t % tiles_per_frame) * 2 * MT;
                for (int ps = 0; ps < C::PASSES && ok; ++ps)
                for (int c = 0; c < nchunks && ok; ++c)
                    for (int kx = 0; kx < 3 && ok; ++kx) {
                        if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag)) {
                            ok = false;
                            break;
                        }
                        // passes of the split form: (A hi, B hi), (A hi, B lo), (A lo, B hi)
                        const int pa = ps == 2 ? 1 : 0, pb = ps == 1 ? 1 : 0;
                        unsigned char *sa = smem + s * C::STAGE;
                        mbar_expect_tx(&full[s], (uint32_t)C::STAGE);
                        tma_load_4d(sa, &tmA, &full[s], pa * cin + c * CC, kx - 1, y0 - 1, m);
                        tma_load_3d(sa + C::A_BYTES, &tmB, &full[s], 0, 0, ((pb * nchunks + c) * 3 + kx) * 3);
                        issued |= 1u << s;
                        last_par = (last_par & ~(1u << s)) | (ph << s);
                        if (++s == S) {
                            s = 0;
                            ph ^= 1u;
                        }
                    }
            }
            if (!ok) {
                *abort_flag = 1;
                // drain the copies this CTA issued before leaving (bounded)
                volatile int never = 0;
                for (int k = 0; k < S; ++k)
                    if (issued & (1u << k)) mbar_wait(&full[k], (last_par >> k) & 1u, &never, 100000000ull);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer
            constexpr uint32_t idesc = MODE == 1 ? idesc_tf32(128, N) : idesc_bf16(128, N);
            int s = 0;
            uint32_t ph = 0;
            int tl = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < total && ok; t += gridDim.x, ++tl) {
                const int buf = tl & 1;
                const uint32_t tph = (uint32_t)(tl >> 1) & 1u;
                if (!mbar_wait(&tempty[buf], tph ^ 1u, abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                for (int k = 0; k < ksteps; ++k) {
                    if (!mbar_wait(&full[s], ph, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(smem + s * C::STAGE);
                    const uint32_t sb = sa + C::A_BYTES;
                    const uint64_t a0 = smem_desc(sa, C::SBO, C::SWZ), b0 = smem_desc(sb, C::SBO, C::SWZ);
#pragma unroll
                    for (int sub = 0; sub < MT; ++sub) {
                        // subtile sub covers output rows y0 + 2*sub, +1: A rows start at 64*(2*sub + ky)
                        const uint32_t dt = tmem_base + (uint32_t)((buf * MT + sub) * N);
#pragma unroll
                        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
                            for (int kk = 0; kk < C::ROWB / 32; ++kk) {
                                const uint64_t ad = desc_add(a0, (2 * sub + ky) * 64 * C::ROWB + kk * 32);
                                const uint64_t bd = desc_add(b0, ky * C::B_TAP + kk * 32);
                                if constexpr (MODE == 1)
                                    mma_tf32(dt, ad, bd, idesc, (k | ky | kk) != 0);
                                else
                                    mma_bf16(dt, ad, bd, idesc, (k | ky | kk) != 0);
                            }
                    }
                    mma_commit(&empty[s]);
                    if (++s == S) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
                if (ok) mma_commit(&tfull[buf]);
            }
            if (!ok) *abort_flag = 1;
        }
    } else {
        // ---- epilogue: warps 2..5, TMEM lane quarter = warp % 4
        const int qtr = warp & 3;
        const int row = qtr * 32 + lane;
        int tl = 0;
        for (int t = blockIdx.x; t < total; t += gridDim.x, ++tl) {
            const int buf = tl & 1;
            const uint32_t tph = (uint32_t)(tl >> 1) & 1u;
            if (!mbar_wait(&tfull[buf], tph, abort_flag)) {
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            const int m = t / tiles_per_frame;
#pragma unroll
            for (int sub = 0; sub < MT; ++sub) {
                const int p0 = (t % tiles_per_frame) * 128 * MT + 128 * sub;
                const uint32_t col0 = (uint32_t)((buf * MT + sub) * N);
                if (head_w) {
                    // last layer of the UDF: fold global average pooling and the
                    // linear head into the epilogue; each warp leaves one partial
                    // sum of hw . relu(conv) over its 32 pixels
                    float hsum = 0.f;
#pragma unroll
                    for (int c0 = 0; c0 < N; c0 += 32) {
                        uint32_t r[32];
                        tmem_ld32(tmem_base + ((uint32_t)(qtr * 32) << 16) + col0 + (uint32_t)c0, r);
                        tmem_ld_wait();
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            float v = __uint_as_float(r[j]) + __ldg(bias + c0 + j);
                            v = v > 0.f ? v : 0.f;
                            hsum = fmaf(__ldg(head_w + c0 + j), v, hsum);
                        }
                    }
#pragma unroll
                    for (int d = 16; d > 0; d >>= 1) hsum += __shfl_xor_sync(0xffffffffu, hsum, d);
                    if (lane == 0) partials[((size_t)t * MT + sub) * 4 + qtr] = hsum;
                } else if constexpr (MODE == 2) {
                    // split-BF16 output as two planes per pixel: [hi(N) | lo(N)].  Each 32-channel group's
                    // hi and lo halves go through the warp's staging rows (128 B a pixel, 16-byte chunk j
                    // at slot j ^ (p % 8)) so that a store instruction writes both 64-byte halves of 4
                    // pixels whole
                    __nv_bfloat16 *o = static_cast<__nv_bfloat16 *>(out) + ((size_t)m * HW + p0 + qtr * 32) * (2 * N);
                    uint4 *stg = stg_all + (warp - 2) * (32 * 8);
#pragma unroll
                    for (int c0 = 0; c0 < N; c0 += 32) {
                        uint32_t r[32];
                        tmem_ld32(tmem_base + ((uint32_t)(qtr * 32) << 16) + col0 + (uint32_t)c0, r);
                        tmem_ld_wait();
                        uint32_t hi[16], lo[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            float v0 = __uint_as_float(r[2 * j]) + __ldg(bias + c0 + 2 * j);
                            float v1 = __uint_as_float(r[2 * j + 1]) + __ldg(bias + c0 + 2 * j + 1);
                            v0 = v0 > 0.f ? v0 : 0.f;
                            v1 = v1 > 0.f ? v1 : 0.f;
                            hi[j] = pack_bf16x2(v0, v1);
                            lo[j] = pack_bf16x2(v0 - __uint_as_float(hi[j] << 16), v1 - __uint_as_float(hi[j] & 0xFFFF0000u));
                        }
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            stg[lane * 8 + (j ^ (lane & 7))] = make_uint4(hi[4 * j], hi[4 * j + 1], hi[4 * j + 2], hi[4 * j + 3]);
                            stg[lane * 8 + ((4 + j) ^ (lane & 7))] =
                                make_uint4(lo[4 * j], lo[4 * j + 1], lo[4 * j + 2], lo[4 * j + 3]);
                        }
                        __syncwarp();
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            // lanes 8k .. 8k+7: the hi (chunks 0..3) and lo (4..7) halves of pixel 4 i + k
                            const int pp = i * 4 + (lane >> 3), cq = lane & 7;
                            const int dst = cq < 4 ? c0 + cq * 8 : N + c0 + (cq - 4) * 8;
                            *reinterpret_cast<uint4 *>(o + (size_t)pp * (2 * N) + dst) = stg[pp * 8 + (cq ^ (pp & 7))];
                        }
                        __syncwarp();
                    }
                } else if constexpr (MODE == 1) {
                    // fp32 output as two planes per pixel: [hi(N) | lo(N)]
                    float *o = static_cast<float *>(out) + ((size_t)m * HW + p0 + row) * (2 * N);
#pragma unroll
                    for (int c0 = 0; c0 < N; c0 += 32) {
                        uint32_t r[32];
                        tmem_ld32(tmem_base + ((uint32_t)(qtr * 32) << 16) + col0 + (uint32_t)c0, r);
                        tmem_ld_wait();
#pragma unroll
                        for (int j = 0; j < 32; j += 4) {
                            float v[4], hi[4], lo[4];
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                v[e] = __uint_as_float(r[j + e]) + __ldg(bias + c0 + j + e);
                                v[e] = v[e] > 0.f ? v[e] : 0.f;
                                hi[e] = tf32_rne(v[e]);
                                lo[e] = tf32_rne(v[e] - hi[e]);
                            }
                            *reinterpret_cast<float4 *>(o + c0 + j) = make_float4(hi[0], hi[1], hi[2], hi[3]);
                            *reinterpret_cast<float4 *>(o + N + c0 + j) = make_float4(lo[0], lo[1], lo[2], lo[3]);
                        }
                    }
                } else {
                    // through the warp's staging rows, one per pixel (16-byte chunk j of pixel p at slot
                    // j ^ (p % Q), conflict-free both ways).  Layers with several input chunks (long MMA
                    // phases) store whole pixel rows once all channel groups are staged: 32 / Q complete
                    // rows per instruction, full 128-byte lines.  One-chunk layers, whose epilogue is
                    // closer to the MMA time, store each 64-byte channel group as soon as it is staged.
                    constexpr int Q = N / 8;   // 16-byte chunks per pixel row
                    __nv_bfloat16 *o = static_cast<__nv_bfloat16 *>(out) + ((size_t)m * HW + p0 + qtr * 32) * N;
                    uint4 *stg = stg_all + (warp - 2) * (32 * Q);
                    const bool rows = nchunks > 1;
#pragma unroll
                    for (int c0 = 0; c0 < N; c0 += 32) {
                        uint32_t r[32];
                        tmem_ld32(tmem_base + ((uint32_t)(qtr * 32) << 16) + col0 + (uint32_t)c0, r);
                        tmem_ld_wait();
                        uint32_t pk[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            float v0 = __uint_as_float(r[2 * j]) + __ldg(bias + c0 + 2 * j);
                            float v1 = __uint_as_float(r[2 * j + 1]) + __ldg(bias + c0 + 2 * j + 1);
                            v0 = v0 > 0.f ? v0 : 0.f;
                            v1 = v1 > 0.f ? v1 : 0.f;
                            pk[j] = pack_bf16x2(v0, v1);
                        }
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            stg[lane * Q + ((c0 / 8 + j) ^ (lane % Q))] =
                                make_uint4(pk[4 * j], pk[4 * j + 1], pk[4 * j + 2], pk[4 * j + 3]);
                        if (!rows) {
                            __syncwarp();
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                // lanes 4k .. 4k+3 write the four chunks of this group of pixel 8 i + k
                                const int pp = i * 8 + (lane >> 2), cq = c0 / 8 + (lane & 3);
                                reinterpret_cast<uint4 *>(o + (size_t)pp * N)[cq] = stg[pp * Q + (cq ^ (pp % Q))];
                            }
                            __syncwarp();
                        }
                    }
                    if (rows) {
                        __syncwarp();
#pragma unroll
                        for (int i = 0; i < Q; ++i) {
                            const int pp = i * (32 / Q) + lane / Q, cq = lane % Q;
                            reinterpret_cast<uint4 *>(o + (size_t)pp * N)[cq] = stg[pp * Q + (cq ^ (pp % Q))];
                        }
                        __syncwarp();
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[buf]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                     "r"((uint32_t)C::TMEM_COLS)
                     : "memory");
    }
    if (threadIdx.x == 0 && *abort_flag) atomicOr(err, ERR_TC_TIMEOUT);
}

// ---------------------------------------------------------------------------
// Window variant for the 64-output BF16 layers (Cin 32 or 64).  The
// narrow layers are bound by operand traffic from L2 when every horizontal
// tap loads its own shifted box.  Here the output pixels are numbered in a
// padded frame of WP = 66 columns (q = y * 66 + x; x = 64, 65 are padding
// and never stored), so every tap (ky, kx) reads the input at the uniform
// shift (ky - 1) * 66 + kx of one window box {32 channels, 66 columns
// x = -1 .. 64, 9 rows} that TMA zero-fills outside the frame.  One box per
// 32-channel chunk feeds all nine taps of three 128-pixel subtiles: the
// MMA's A descriptor starts at the shifted pixel row, which need not be
// aligned to the 64-byte swizzle atom: the tensor core applies the swizzle
// to absolute shared-memory address bits, as TMA does when it writes the box,
// so a start at any pixel row reads that row (base-offset field 0; measured
// on this GPU for every row shift of 64- and 128-byte swizzled operands).  The weights stay in
// shared memory for the whole launch.  The padded pixels cost 3 % more MMA
// work; the operand bytes per output pixel drop 2.3x.
constexpr int kWP = 66;                        // padded frame width
constexpr int kWMT = 3;                        // 128-pixel subtiles per CTA tile (384 padded pixels)
constexpr int kWRows = 9;                      // window rows: up to 7 output rows + 2 halo rows
constexpr int kWBox = kWRows * kWP * 64;       // one 32-channel window box (bytes)
constexpr int kWStage = (kWBox + 1023) / 1024 * 1024;
// Warp roles: 0 TMA, 1 MMA, 2-9 epilogue.  With 64 output channels an MMA
// takes half as long per output value as with 128, so the epilogue is split
// over eight warps: warp w drains TMEM lanes 32 (w % 4) .. + 31 and the
// column half (w - 2) / 4, with its 32 biases (and head weights) in registers.
constexpr int kWThreads = 320;
constexpr int kWEpi = 8;
constexpr int kWStg = 32 * 64;                 // an epilogue warp's store staging: 32 pixels x 64 B

template <int CIN, int S>
struct TcWCfg {
    static constexpr int CCB = CIN == 32 ? 32 : 64;        // weight packing chunk (channels)
    static constexpr int ROWB_B = CCB * 2;
    static constexpr int B_TAP = 64 * ROWB_B;               // one tap's weights [64 co][CCB]
    static constexpr int B_BYTES = 3 * B_TAP;               // one (chunk, kx) box
    static constexpr int RES_BYTES = (CIN / CCB) * 3 * B_BYTES;
    static constexpr uint32_t SWZ_B = ROWB_B == 128 ? 2u : 4u;
    static constexpr int NCH = CIN / 32;                    // window boxes (stages) per tile
    static constexpr int TMEM_COLS = 512;                   // 2 x 3 x 64 used
    static constexpr int SMEM = RES_BYTES + S * kWStage + 1024 + 256 + kWEpi * kWStg;
    static_assert(SMEM <= 227 * 1024, "shared memory per CTA");
};

// K-major SW64 descriptor of an A operand starting at any pixel row (64 B).
__device__ __forceinline__ uint64_t wdesc_a(uint32_t saddr) { return smem_desc(saddr, 512, 4u); }

template <int CIN, int S>
__global__ void __launch_bounds__(kWThreads, 1)
k_conv3x3_tcw(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const int *count,
              int H, int tiles_per_frame, const float *__restrict__ bias, __nv_bfloat16 *out,
              const float *__restrict__ head_w, float *partials, unsigned int *err) {
    using C = TcWCfg<CIN, S>;
    extern __shared__ unsigned char smem_raw[];
    // aligned to 1 KB by pointer arithmetic on the shared array itself, so that the compiler
    // keeps every access through it in the shared state space (no generic loads or stores)
    unsigned char *wres = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char *smem = wres + C::RES_BYTES;   // window stages
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + S * kWStage);
    uint64_t *empty = full + S;
    uint64_t *tfull = empty + S;
    uint64_t *tempty = tfull + 2;
    uint64_t *wbar = tempty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(wbar + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    uint4 *stg_all = reinterpret_cast<uint4 *>(smem + S * kWStage + 256);   // kWEpi x kWStg bytes

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int total = (*count) * tiles_per_frame;
    if ((int)blockIdx.x >= total) return;
    const int Q = H * kWP;   // padded pixels per frame

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], kWEpi);
        }
        mbar_init(wbar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)C::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer: the weights once, then one window box per 32-channel chunk
            int s = 0;
            uint32_t ph = 0, issued = 0, last_par = 0;
            bool ok = true;
            mbar_expect_tx(wbar, (uint32_t)C::RES_BYTES);
            for (int cb = 0; cb < CIN / C::CCB; ++cb)
                for (int kx = 0; kx < 3; ++kx)
                    tma_load_3d(wres + (cb * 3 + kx) * C::B_BYTES, &tmB, wbar, 0, 0, (cb * 3 + kx) * 3);
            for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
                const int m = t / tiles_per_frame;
                const int q0 = (t % tiles_per_frame) * 128 * kWMT;
                const int y_lo = q0 / kWP - 1;
                for (int c = 0; c < C::NCH; ++c) {
                    if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&full[s], (uint32_t)kWBox);
                    tma_load_4d(smem + s * kWStage, &tmA, &full[s], c * 32, -1, y_lo, m);
                    issued |= 1u << s;
                    last_par = (last_par & ~(1u << s)) | (ph << s);
                    if (++s == S) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
            }
            if (!ok) {
                *abort_flag = 1;
                volatile int never = 0;
                for (int k = 0; k < S; ++k)
                    if (issued & (1u << k)) mbar_wait(&full[k], (last_par >> k) & 1u, &never, 100000000ull);
                mbar_wait(wbar, 0u, &never, 100000000ull);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer: 3 subtiles x 9 taps x 2 K-steps per window box
            constexpr uint32_t idesc = idesc_bf16(128, 64);
            int s = 0;
            uint32_t ph = 0;
            int tl = 0;
            bool ok = mbar_wait(wbar, 0u, abort_flag);
            for (int t = blockIdx.x; t < total && ok; t += gridDim.x, ++tl) {
                const int buf = tl & 1;
                const uint32_t tph = (uint32_t)(tl >> 1) & 1u;
                if (!mbar_wait(&tempty[buf], tph ^ 1u, abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const int q0 = (t % tiles_per_frame) * 128 * kWMT;
                const int pix0 = q0 % kWP + kWP;   // padded pixel q0 in the window (row y_lo + 1)
                for (int c = 0; c < C::NCH; ++c) {
                    if (!mbar_wait(&full[s], ph, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(smem + s * kWStage);
                    // weights of this 32-channel chunk: packing chunk cb, K offset kb inside its rows
                    const int cb = (c * 32) / C::CCB, kb = (c * 32) % C::CCB;
                    // descriptors of the chunk's first A row (padded pixel pix0) and first weight row
                    const uint64_t a0 = wdesc_a(sa + (uint32_t)(pix0 * 64));
                    const uint64_t b0 = smem_desc(smem_u32(wres) + (uint32_t)(cb * 3 * C::B_BYTES + kb * 2),
                                                  8 * C::ROWB_B, C::SWZ_B);
#pragma unroll
                    for (int sub = 0; sub < kWMT; ++sub) {
                        const uint32_t dt = tmem_base + (uint32_t)((buf * kWMT + sub) * 64);
#pragma unroll
                        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
                            for (int kx = 0; kx < 3; ++kx) {
                                const int dpix = 128 * sub + (ky - 1) * kWP + kx;
#pragma unroll
                                for (int kk = 0; kk < 2; ++kk) {
                                    const uint64_t ad = desc_add(a0, dpix * 64 + kk * 32);
                                    const uint64_t bd = desc_add(b0, kx * C::B_BYTES + ky * C::B_TAP + kk * 32);
                                    mma_bf16(dt, ad, bd, idesc, (c | ky | kx | kk) != 0);
                                }
                            }
                    }
                    mma_commit(&empty[s]);
                    if (++s == S) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
                if (ok) mma_commit(&tfull[buf]);
            }
            if (!ok) *abort_flag = 1;
        }
    } else {
        // ---- epilogue: warps 2..9, TMEM lane quarter = warp % 4, column half (warp - 2) / 4;
        // padded pixels are dropped.  Stores go through the warp's staging rows (16-byte chunk j
        // of pixel p at slot j ^ ((p >> 1) & 3), conflict-free both ways) so that each store
        // instruction writes whole 64-byte pixel halves of 8 pixels: full 32-byte sectors.
        const int qtr = warp & 3, ch = (warp - 2) >> 2;
        const int row = qtr * 32 + lane;
        uint4 *stg = stg_all + (warp - 2) * (kWStg / 16);
        float bv[32], hv[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            bv[j] = __ldg(bias + ch * 32 + j);
            hv[j] = head_w ? __ldg(head_w + ch * 32 + j) : 0.f;
        }
        int tl = 0;
        for (int t = blockIdx.x; t < total; t += gridDim.x, ++tl) {
            const int buf = tl & 1;
            const uint32_t tph = (uint32_t)(tl >> 1) & 1u;
            if (!mbar_wait(&tfull[buf], tph, abort_flag)) {
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            const int m = t / tiles_per_frame;
            const int q0 = (t % tiles_per_frame) * 128 * kWMT;
#pragma unroll
            for (int sub = 0; sub < kWMT; ++sub) {
                const int q = q0 + 128 * sub + row;
                const int x = q - (q / kWP) * kWP;
                const bool valid = q < Q && x < 64;
                uint32_t r[32];
                tmem_ld32(tmem_base + ((uint32_t)(qtr * 32) << 16) + (uint32_t)((buf * kWMT + sub) * 64 + ch * 32), r);
                tmem_ld_wait();
                if (head_w) {
                    float hsum = 0.f;
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        float v = __uint_as_float(r[j]) + bv[j];
                        v = v > 0.f ? v : 0.f;
                        hsum = fmaf(hv[j], v, hsum);
                    }
                    hsum = valid ? hsum : 0.f;
#pragma unroll
                    for (int d = 16; d > 0; d >>= 1) hsum += __shfl_xor_sync(0xffffffffu, hsum, d);
                    if (lane == 0) partials[(((size_t)t * kWMT + sub) * 4 + qtr) * 2 + ch] = hsum;
                } else {
                    uint32_t pk[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        float v0 = __uint_as_float(r[2 * j]) + bv[2 * j];
                        float v1 = __uint_as_float(r[2 * j + 1]) + bv[2 * j + 1];
                        v0 = v0 > 0.f ? v0 : 0.f;
                        v1 = v1 > 0.f ? v1 : 0.f;
                        pk[j] = pack_bf16x2(v0, v1);
                    }
                    const int sw = (lane >> 1) & 3;
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        stg[lane * 4 + (j ^ sw)] = make_uint4(pk[4 * j], pk[4 * j + 1], pk[4 * j + 2], pk[4 * j + 3]);
                    __syncwarp();
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        // lanes 4k .. 4k+3 write the four chunks of pixel 8 i + k of the warp's 32
                        const int pp = i * 8 + (lane >> 2), cq = lane & 3;
                        const uint4 v = stg[pp * 4 + (cq ^ ((pp >> 1) & 3))];
                        const int qp = q0 + 128 * sub + qtr * 32 + pp;
                        const int yp = qp / kWP, xp = qp - (qp / kWP) * kWP;
                        if (qp < Q && xp < 64)
                            reinterpret_cast<uint4 *>(out + ((size_t)m * H * 64 + (size_t)yp * 64 + xp) * 64 +
                                                      ch * 32)[cq] = v;
                    }
                    __syncwarp();
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[buf]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                     "r"((uint32_t)C::TMEM_COLS)
                     : "memory");
    }
    if (threadIdx.x == 0 && *abort_flag) atomicOr(err, ERR_TC_TIMEOUT);
}

constexpr int kSW32 = 4, kSW64 = 3;   // window stages for Cin 32 / 64

// score[m] = hb + (sum of the frame's epilogue partials) / HW, one warp per
// frame, fixed lane order and butterfly reduction (deterministic).
__global__ void k_head_finalize(const int *count, const float *partials, int parts_per_frame, double hb, int HW,
                                float *score) {
    const int M = *count;
    const int lane = threadIdx.x & 31;
    for (int m = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; m < M; m += (gridDim.x * blockDim.x) >> 5) {
        const float *pp = partials + (size_t)m * parts_per_frame;
        float s = 0.f;
        for (int j = lane; j < parts_per_frame; j += 32) s += pp[j];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
        if (lane == 0) score[m] = (float)(hb + (double)s / (double)HW);
    }
}

// Self-test of the bounded wait: one thread waits on an mbarrier nothing
// arrives on, with a limit of limit_ns; *status = 1 if the wait ran out (the
// designed outcome), 0 if it completed.  The kernel always returns.
__global__ void k_wait_selftest(unsigned long long limit_ns, int *status) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        const bool ok = mbar_wait(&bar, 0u, &abort_flag, limit_ns);
        *status = ok ? 0 : 1;
    }
}

using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                              const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

template <int CC, int N, int S, int MODE, int MT>
cudaError_t set_smem() {
    return cudaFuncSetAttribute(k_conv3x3_tc<CC, N, S, MODE, MT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                TcCfg<CC, N, S, MODE, MT>::SMEM);
}

// 128-output layers: two 128-pixel subtiles per CTA tile (2 x 2 x 128 TMEM
// columns); 64-output layers: four (2 x 4 x 64).  Stage counts per shape sized
// to 180-216 KB of shared memory.
constexpr int kMT = 2, kMT64 = 4;
constexpr int kS_64_128 = 2, kS_64_64 = 2, kS_32_128 = 4, kS_32_64 = 4;
constexpr int kS_t32_128 = 2, kS_t32_64 = 2;   // split TF32, CC = 32 fp32 channels

}  // namespace

bool tc_conv_supported(int cin, int cout, int H, int W) {
    if (W != 64 || H < 8 || (H % 8) != 0) return false;
    if (cout != 64 && cout != 128) return false;
    return cin == 32 || (cin % 64 == 0 && cin <= 512);
}

void tc_conv_pack_weights(const float *w, int cin, int cout, std::vector<__nv_bfloat16> &out) {
    const int CC = cin == 32 ? 32 : 64;
    const int nch = cin / CC;
    out.assign((size_t)nch * 9 * cout * CC, __float2bfloat16_rn(0.f));
    // layout [(c*3 + kx)*3 + ky][co][k], ci = c*CC + k; source W[co][ci][ky][kx]
    for (int c = 0; c < nch; ++c)
        for (int kx = 0; kx < 3; ++kx)
            for (int ky = 0; ky < 3; ++ky)
                for (int co = 0; co < cout; ++co)
                    for (int k = 0; k < CC; ++k) {
                        const int ci = c * CC + k;
                        const float v = w[(((size_t)co * cin + ci) * 3 + ky) * 3 + kx];
                        out[((((size_t)(c * 3 + kx) * 3 + ky) * cout + co) * CC) + k] = __float2bfloat16_rn(v);
                    }
}

void tc_conv_pack_weights_split_bf16(const float *w, int cin, int cout, std::vector<__nv_bfloat16> &out) {
    const int CC = cin == 32 ? 32 : 64;
    const int nch = cin / CC;
    out.assign((size_t)2 * nch * 9 * cout * CC, __float2bfloat16_rn(0.f));
    // layout [((plane*nch + c)*3 + kx)*3 + ky][co][k]; plane 0 = bf16(w), 1 = bf16(w - plane 0)
    for (int plane = 0; plane < 2; ++plane)
        for (int c = 0; c < nch; ++c)
            for (int kx = 0; kx < 3; ++kx)
                for (int ky = 0; ky < 3; ++ky)
                    for (int co = 0; co < cout; ++co)
                        for (int k = 0; k < CC; ++k) {
                            const int ci = c * CC + k;
                            const float v = w[(((size_t)co * cin + ci) * 3 + ky) * 3 + kx];
                            const __nv_bfloat16 hi = __float2bfloat16_rn(v);
                            const size_t o = ((((size_t)(plane * nch + c) * 3 + kx) * 3 + ky) * cout + co) * CC + k;
                            out[o] = plane == 0 ? hi : __float2bfloat16_rn(v - __bfloat162float(hi));
                        }
}

void tc_conv_pack_weights_split(const float *w, int cin, int cout, std::vector<float> &out) {
    const int CC = 32;
    const int nch = cin / CC;
    out.assign((size_t)2 * nch * 9 * cout * CC, 0.f);
    // layout [((plane*nch + c)*3 + kx)*3 + ky][co][k]; plane 0 = TF32 high part, 1 = remainder
    for (int plane = 0; plane < 2; ++plane)
        for (int c = 0; c < nch; ++c)
            for (int kx = 0; kx < 3; ++kx)
                for (int ky = 0; ky < 3; ++ky)
                    for (int co = 0; co < cout; ++co)
                        for (int k = 0; k < CC; ++k) {
                            const int ci = c * CC + k;
                            const float v = w[(((size_t)co * cin + ci) * 3 + ky) * 3 + kx];
                            const float hi = tf32_rne(v);
                            const size_t o = ((((size_t)(plane * nch + c) * 3 + kx) * 3 + ky) * cout + co) * CC + k;
                            out[o] = plane == 0 ? hi : tf32_rne(v - hi);
                        }
}

hydro_status tc_conv_init(TcConvPlan *plan, int device) {
    plan->device = device;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult qr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr);
    if (e != cudaSuccess || qr != cudaDriverEntryPointSuccess || !fn) {
        g_tc_err = "cuTensorMapEncodeTiled entry point not available";
        return HYDRO_ECUDA;
    }
    plan->encode = fn;
    if (cudaDeviceGetAttribute(&plan->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device) != cudaSuccess) {
        g_tc_err = "cudaDeviceGetAttribute(shared memory per SM) failed";
        return HYDRO_ECUDA;
    }
    cudaError_t r = cudaSuccess;
    if (r == cudaSuccess) r = set_smem<64, 128, kS_64_128, 0, kMT>();
    if (r == cudaSuccess) r = set_smem<64, 64, kS_64_64, 0, kMT64>();
    if (r == cudaSuccess) r = set_smem<32, 128, kS_32_128, 0, kMT>();
    if (r == cudaSuccess) r = set_smem<32, 128, kS_t32_128, 1, kMT>();
    if (r == cudaSuccess) r = set_smem<32, 64, kS_t32_64, 1, kMT64>();
    if (r == cudaSuccess) r = set_smem<64, 128, kS_64_128, 2, kMT>();
    if (r == cudaSuccess) r = set_smem<64, 64, kS_64_64, 2, kMT64>();
    if (r == cudaSuccess) r = set_smem<32, 128, kS_32_128, 2, kMT>();
    if (r == cudaSuccess) r = set_smem<32, 64, kS_32_64, 2, kMT64>();
    if (r == cudaSuccess)
        r = cudaFuncSetAttribute(k_conv3x3_tcw<32, kSW32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 TcWCfg<32, kSW32>::SMEM);
    if (r == cudaSuccess)
        r = cudaFuncSetAttribute(k_conv3x3_tcw<64, kSW64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 TcWCfg<64, kSW64>::SMEM);
    if (r != cudaSuccess) {
        g_tc_err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(r);
        return HYDRO_ECUDA;
    }
    plan->ready = true;
    return HYDRO_OK;
}

void tc_head_finalize(const int *count, const float *partials, int parts_per_frame, double hb, int HW,
                      float *score, int max_frames, int sms, cudaStream_t st) {
    int grid = (max_frames + 7) / 8;
    if (grid > sms * 8) grid = sms * 8;
    if (grid < 1) grid = 1;
    k_head_finalize<<<grid, 256, 0, st>>>(count, partials, parts_per_frame, hb, HW, score);
}

// The window kernel serves the BF16 64-output layers of 32 or 64 input channels.
bool use_window(int cin, int cout, int mode) { return mode == 0 && cout == 64 && (cin == 32 || cin == 64); }

int window_tiles_per_frame(int H) { return (H * kWP + 128 * kWMT - 1) / (128 * kWMT); }

hydro_status tc_conv_run_window(TcConvPlan *plan, const int *count, const void *in, int cin, int H,
                                const void *wpacked, const float *bias, void *out, int max_frames, int sms,
                                cudaStream_t st, unsigned int *err, const float *head_w, float *partials) {
    EncodeFn enc = reinterpret_cast<EncodeFn>(plan->encode);
    CUtensorMap tmA, tmB;
    {
        // activations [frame][y][x][cin] bf16; window box {32 channels, 66 columns, 9 rows, 1 frame}
        const cuuint64_t dims[4] = {(cuuint64_t)cin, 64, (cuuint64_t)H, (cuuint64_t)max_frames};
        const cuuint64_t strides[3] = {(cuuint64_t)cin * 2, (cuuint64_t)64 * cin * 2, (cuuint64_t)H * 64 * cin * 2};
        const cuuint32_t box[4] = {32, (cuuint32_t)kWP, (cuuint32_t)kWRows, 1};
        const cuuint32_t es[4] = {1, 1, 1, 1};
        CUresult r = enc(&tmA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(in), dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            g_tc_err = "cuTensorMapEncodeTiled(window activations) failed: " + std::to_string((int)r);
            return HYDRO_ECUDA;
        }
    }
    {
        const int CC = cin == 32 ? 32 : 64;
        const cuuint64_t dims[3] = {(cuuint64_t)CC, 64, (cuuint64_t)(cin / CC) * 9};
        const cuuint64_t strides[2] = {(cuuint64_t)CC * 2, (cuuint64_t)64 * CC * 2};
        const cuuint32_t box[3] = {(cuuint32_t)CC, 64, 3};
        const cuuint32_t es[3] = {1, 1, 1};
        CUresult r = enc(&tmB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(wpacked), dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CC == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            g_tc_err = "cuTensorMapEncodeTiled(window weights) failed: " + std::to_string((int)r);
            return HYDRO_ECUDA;
        }
    }
    const int tpf = window_tiles_per_frame(H);
    const long long tiles = (long long)max_frames * tpf;
    const int grid = (int)(tiles < sms ? tiles : sms);
    __nv_bfloat16 *o = static_cast<__nv_bfloat16 *>(out);
    if (cin == 32)
        k_conv3x3_tcw<32, kSW32><<<grid, kWThreads, TcWCfg<32, kSW32>::SMEM, st>>>(tmA, tmB, count, H, tpf, bias, o, head_w,
                                                                            partials, err);
    else
        k_conv3x3_tcw<64, kSW64><<<grid, kWThreads, TcWCfg<64, kSW64>::SMEM, st>>>(tmA, tmB, count, H, tpf, bias, o, head_w,
                                                                            partials, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_tc_err = std::string("launch: ") + cudaGetErrorString(e);
        return HYDRO_ECUDA;
    }
    return HYDRO_OK;
}

int tc_conv_head_parts(int cin, int cout, int H, int W, int mode) {
    return use_window(cin, cout, mode) ? window_tiles_per_frame(H) * kWMT * 8 : H * W / 128 * 4;
}

int tc_conv_max_head_parts(int H, int W) {
    const int a = H * W / 128 * 4, b = window_tiles_per_frame(H) * kWMT * 8;
    return a > b ? a : b;
}

hydro_status tc_conv_run(TcConvPlan *plan, const int *count, const void *in, int cin, int H, int W,
                         const void *wpacked, const float *bias, int cout, void *out, int max_frames, int sms,
                         cudaStream_t st, unsigned int *err, const float *head_w, float *partials, int mode) {
    if (!plan->ready || !tc_conv_supported(cin, cout, H, W)) {
        g_tc_err = "tensor-core conv not ready or shape unsupported";
        return HYDRO_EUNSUPPORTED;
    }
    if (use_window(cin, cout, mode))
        return tc_conv_run_window(plan, count, in, cin, H, wpacked, bias, out, max_frames, sms, st, err, head_w,
                                  partials);
    EncodeFn enc = reinterpret_cast<EncodeFn>(plan->encode);
    // operand chunk: 64 bf16 / 32 bf16 (128 B or 64 B rows); 3xTF32 fp32: 32 (128 B rows)
    const bool tf32 = mode == 1;
    const int CC = tf32 ? 32 : (cin == 32 ? 32 : 64);
    const int esz = tf32 ? 4 : 2;
    const int planes = mode ? 2 : 1;
    const int nch = cin / CC;
    const int mt = cout == 64 ? kMT64 : kMT;   // 128-pixel subtiles per CTA tile
    const CUtensorMapDataType dt = tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const CUtensorMapSwizzle swz = CC * esz == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
    const cuuint64_t ctot = (cuuint64_t)cin * planes;   // channels stored per pixel
    CUtensorMap tmA, tmB;
    {
        const cuuint64_t dims[4] = {ctot, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)max_frames};
        const cuuint64_t strides[3] = {ctot * esz, (cuuint64_t)W * ctot * esz, (cuuint64_t)H * W * ctot * esz};
        const cuuint32_t box[4] = {(cuuint32_t)CC, 64, (cuuint32_t)(2 + 2 * mt), 1};
        const cuuint32_t es[4] = {1, 1, 1, 1};
        CUresult r = enc(&tmA, dt, 4, const_cast<void *>(in), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            g_tc_err = "cuTensorMapEncodeTiled(activations) failed: " + std::to_string((int)r);
            return HYDRO_ECUDA;
        }
    }
    {
        const cuuint64_t dims[3] = {(cuuint64_t)CC, (cuuint64_t)cout, (cuuint64_t)planes * nch * 9};
        const cuuint64_t strides[2] = {(cuuint64_t)CC * esz, (cuuint64_t)cout * CC * esz};
        const cuuint32_t box[3] = {(cuuint32_t)CC, (cuuint32_t)cout, 3};
        const cuuint32_t es[3] = {1, 1, 1};
        CUresult r = enc(&tmB, dt, 3, const_cast<void *>(wpacked), dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            g_tc_err = "cuTensorMapEncodeTiled(weights) failed: " + std::to_string((int)r);
            return HYDRO_ECUDA;
        }
    }
    const int tpf = H / (2 * mt);   // CTA tiles per frame (W == 64)
    long long tiles = (long long)max_frames * tpf;
    const int grid = (int)(tiles < sms ? tiles : sms);
    const int HW = H * W;
#define HYDRO_TC_LAUNCH(CC_, N_, S_, MODE_, MT_)                                                            \
    k_conv3x3_tc<CC_, N_, S_, MODE_, MT_><<<grid, 192, TcCfg<CC_, N_, S_, MODE_, MT_>::SMEM, st>>>(      \
        tmA, tmB, count, nch, cin, tpf, HW, bias, out, head_w, partials, err)
    if (tf32) {
        if (cout == 128) HYDRO_TC_LAUNCH(32, 128, kS_t32_128, 1, kMT);
        else HYDRO_TC_LAUNCH(32, 64, kS_t32_64, 1, kMT64);
    } else if (mode == 2) {
        if (CC == 64 && cout == 128) HYDRO_TC_LAUNCH(64, 128, kS_64_128, 2, kMT);
        else if (CC == 64) HYDRO_TC_LAUNCH(64, 64, kS_64_64, 2, kMT64);
        else if (cout == 128) HYDRO_TC_LAUNCH(32, 128, kS_32_128, 2, kMT);
        else HYDRO_TC_LAUNCH(32, 64, kS_32_64, 2, kMT64);
    } else if (CC == 64) {
        if (cout == 128) HYDRO_TC_LAUNCH(64, 128, kS_64_128, 0, kMT);
        else HYDRO_TC_LAUNCH(64, 64, kS_64_64, 0, kMT64);
    } else {
        // Cin 32: the 64-output BF16 layer runs the window kernel (use_window)
        HYDRO_TC_LAUNCH(32, 128, kS_32_128, 0, kMT);
    }
#undef HYDRO_TC_LAUNCH
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_tc_err = std::string("launch: ") + cudaGetErrorString(e);
        return HYDRO_ECUDA;
    }
    return HYDRO_OK;
}

cudaError_t wait_selftest(unsigned long long limit_ns, int *d_status, cudaStream_t st) {
    k_wait_selftest<<<1, 32, 0, st>>>(limit_ns, d_status);
    return cudaGetLastError();
}

void tc_conv_destroy(TcConvPlan *plan) { plan->ready = false; }

const char *tc_conv_last_error() { return g_tc_err.c_str(); }

}  // namespace hydro
