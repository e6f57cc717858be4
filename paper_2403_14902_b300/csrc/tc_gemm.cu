// BF16 MLP layers on the tensor cores (tcgen05.mma, accumulator in TMEM,
// operands staged by 2-D TMA), and the 128-bit gather that turns the
// surviving fp32 tuple rows into the dense BF16 operand of the first layer.
//
// Y[m][n] = relu(sum_k X[m][k] W[n][k] + b[n]) for m < *count: CTA tiles of
// 128 rows x NT columns, K in 64-element (128-byte, 128B-swizzled) slices,
// persistent over tiles, warp-specialised like the conv kernel (TMA warp,
// MMA warp, four epilogue warps), two TMEM accumulators.  The UDF's last
// layer (one output) is folded into the epilogue of the last hidden layer:
// each row leaves one partial head . relu(...) per column tile, summed in a
// fixed order by a finalize kernel.
#include <cuda_fp8.h>

#include <cstring>
#include <string>
#include <utility>

#include "common.cuh"
#include "tc_common.cuh"
#include "tc_gemm.h"

namespace hydro {

namespace {

using namespace tcx;
thread_local std::string g_gemm_err;

// One launch serves up to kMaxGroups MLP layers ("groups"): group g owns the
// rows [off_g, off_g + count_g) of the stacked operand (off_g = sum of the
// earlier groups' counts, read on the device), its own weights, K, N and
// column-tile width NT_g (64, 128 or 256), all carried in the launch's
// parameters; tiles are numbered group by group and walked persistently.
constexpr int kA_BYTES = 128 * 128;   // 128 rows x 64 bf16 (one 128-byte swizzled K slice)
constexpr int kMaxStages = 8;

struct TcGroup {   // aligned as its tensor maps
    CUtensorMap tmA, tmB;
    const int *count;         // rows of the group (device)
    const float *bias;        // [N]
    const float *head_w;      // [N]: fold the one-output head into the epilogue; nullptr: store Y
    const float *ascale;      // FP8 groups: [stacked rows] activation scale per row
    const float *wscale;      // FP8 groups: [N] weight scale per output channel
    int K, N, NT;
    int fp8;                  // 1: E4M3 operands (kind::f8f6f4), 128-element K slices
};

struct TcLaunch {
    TcGroup g[kMaxGroups];
    __nv_bfloat16 *Y;         // stacked outputs, row stride ldy (elements)
    float *partials;          // stacked head partials, row stride pstride
    unsigned int *err;
    int n, ldy, pstride, S, stage_bytes, tmem_cols;
    int split3;               // store Y as [hi | hi | lo] BF16 splits (3N columns) for a split-BF16 next layer
    int min_rows;             // fewer stacked rows than this in all groups: no tiles
    int order[kMaxGroups];    // tiles are numbered group order[0] first, then order[1], ...
    int *sched;               // data-aware scheduling: {next tile to claim, CTAs done}, zero between launches
    unsigned long long *rec;  // nullable: per CTA {first, last} global-timer ns of its work
};

// Rows of group g start at off[g] (groups stacked in index order); its tiles
// are numbered from tstart[k] on, k its position in L.order.
__device__ __forceinline__ void group_layout(const TcLaunch &L, int *off, int *cnt, int *tstart) {
    int o = 0;
    for (int g = 0; g < L.n; ++g) {
        const int c = *L.g[g].count;
        off[g] = o;
        cnt[g] = c;
        o += c;
    }
    int t = 0;
    for (int k = 0; k < L.n; ++k) {
        const int g = L.order[k];
        tstart[k] = t;
        if (L.g[g].NT) t += ((cnt[g] + 127) / 128) * (L.g[g].N / L.g[g].NT);
    }
    tstart[L.n] = t;
    if (o < L.min_rows)
        for (int k = 0; k <= L.n; ++k) tstart[k] = 0;
}

// Tile t: its group and its index within the group.
__device__ __forceinline__ int tile_group(const TcLaunch &L, const int *tstart, int t, int *local) {
    int k = 0;
    while (k + 1 < L.n && t >= tstart[k + 1]) ++k;   // groups without tiles have tstart[k] == tstart[k + 1]
    *local = t - tstart[k];
    return L.order[k];
}

// Data-aware scheduling (the paper's load balancing by estimated work,
// Sec. 5.3, on one GPU): tiles are numbered heaviest first and every CTA
// claims its next tile only when its producer is ready for one, so the CTA
// with the least work in hand takes the next tile.  The producer publishes
// each claimed tile (or -1 at the end) in a small ring that the MMA warp and
// the epilogue warps read.
constexpr int kTileRing = 4;

// Warp roles: 0 TMA, 1 MMA (owns TMEM), 2-9 epilogue.  Epilogue warp w reads
// TMEM lanes 32 (w % 4) .. + 31 (its rows) and one half of the tile's
// columns, (w - 2) / 4; a head partial is left per row, tile and half.
constexpr int kGemmThreads = 320;
constexpr int kEpiWarps = 8;

// HAS_FP8: some group of the launch has E4M3 operands (its branches compile out otherwise).
// DYN: data-aware scheduling (claimed tiles, L.sched), else static round robin.
template <bool HAS_FP8, bool DYN>
__global__ void __launch_bounds__(kGemmThreads, 1) k_gemm_grouped_bf16_tc(const __grid_constant__ TcLaunch L) {
    extern __shared__ unsigned char smem_raw[];
    // aligned to 1 KB by pointer arithmetic on the shared array itself, so that the compiler
    // keeps every access through it in the shared state space (no generic loads or stores)
    unsigned char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const int S = L.S;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + S * L.stage_bytes);
    uint64_t *empty = full + kMaxStages;
    uint64_t *tfull = empty + kMaxStages;
    uint64_t *tempty = tfull + 2;
    uint64_t *rfull = tempty + 2;          // tile ring: claimed tile published
    uint64_t *rempty = rfull + kTileRing;  // tile ring: read by the MMA warp and every epilogue warp
    int *ring = reinterpret_cast<int *>(rempty + kTileRing);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(ring + kTileRing);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int off[kMaxGroups], cnt[kMaxGroups], start[kMaxGroups + 1];
    group_layout(L, off, cnt, start);
    const int total = start[L.n];
    // a CTA without tiles takes neither barriers nor TMEM (late rounds and
    // recheck levels leave most of the grid idle)
    if ((int)blockIdx.x >= total) return;
    if (L.rec && threadIdx.x == 0) L.rec[2 * blockIdx.x] = gtimer();

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], kEpiWarps);
        }
        for (int r = 0; r < kTileRing; ++r) {
            mbar_init(&rfull[r], 1);
            mbar_init(&rempty[r], 1 + kEpiWarps);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)L.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const int half = L.tmem_cols / 2;   // columns per accumulator buffer

    if (warp == 0) {
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0, issued = 0, last_par = 0;
            bool ok = true;
            for (int j = 0, t = blockIdx.x; ok; ++j, t += gridDim.x) {
                if constexpr (DYN) {
                    // claim the next tile and publish it (or the end) to the other roles
                    const int r = j % kTileRing;
                    if (!mbar_wait(&rempty[r], (uint32_t)((j / kTileRing) & 1) ^ 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                    t = atomicAdd(L.sched, 1);
                    if (t >= total) t = -1;
                    ring[r] = t;
                    mbar_arrive(&rfull[r]);
                    if (t < 0) break;
                } else if (t >= total) {
                    break;
                }
                int local;
                const int g = tile_group(L, start, t, &local);
                const TcGroup &G = L.g[g];
                const int tiles_n = G.N / G.NT;
                const int m0 = off[g] + (local / tiles_n) * 128, n0 = (local % tiles_n) * G.NT;
                const uint32_t bytes = (uint32_t)(kA_BYTES + G.NT * 128);
                const int kslice = HAS_FP8 && G.fp8 ? 128 : 64;   // elements per 128-byte K slice
                for (int kb = 0; kb < G.K / kslice; ++kb) {
                    if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                    unsigned char *sa = smem + s * L.stage_bytes;
                    mbar_expect_tx(&full[s], bytes);
                    tma_load_2d(sa, &G.tmA, &full[s], kb * kslice, m0);
                    tma_load_2d(sa + kA_BYTES, &G.tmB, &full[s], kb * kslice, n0);
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
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            int tl = 0;
            bool ok = true;
            for (int t = blockIdx.x; ok; t += gridDim.x, ++tl) {
                if constexpr (DYN) {
                    const int r = tl % kTileRing;
                    if (!mbar_wait(&rfull[r], (uint32_t)((tl / kTileRing) & 1), abort_flag)) {
                        ok = false;
                        break;
                    }
                    t = ring[r];
                    mbar_arrive(&rempty[r]);
                    if (t < 0) break;
                } else if (t >= total) {
                    break;
                }
                int local;
                const int g = tile_group(L, start, t, &local);
                (void)local;
                const int NT = L.g[g].NT, fp8 = HAS_FP8 && L.g[g].fp8, kblocks = L.g[g].K / (fp8 ? 128 : 64);
                const uint32_t idesc = fp8 ? idesc_e4m3(128, NT) : idesc_bf16(128, NT);
                const int buf = tl & 1;
                const uint32_t tph = (uint32_t)(tl >> 1) & 1u;
                if (!mbar_wait(&tempty[buf], tph ^ 1u, abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t dt = tmem_base + (uint32_t)(buf * half);
                for (int kb = 0; kb < kblocks; ++kb) {
                    if (!mbar_wait(&full[s], ph, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(smem + s * L.stage_bytes);
                    const uint32_t sb = sa + kA_BYTES;
                    if (fp8) {
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            mma_e4m3(dt, smem_desc(sa + kk * 32, 1024, 2u), smem_desc(sb + kk * 32, 1024, 2u), idesc,
                                     (kb | kk) != 0);
                    } else {
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            mma_bf16(dt, smem_desc(sa + kk * 32, 1024, 2u), smem_desc(sb + kk * 32, 1024, 2u), idesc,
                                     (kb | kk) != 0);
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
        const int qtr = warp & 3;
        const int chalf = (warp - 2) >> 2;
        int tl = 0;
        for (int t = blockIdx.x;; t += gridDim.x, ++tl) {
            if constexpr (DYN) {
                const int r = tl % kTileRing;
                int v = -1;
                if (lane == 0) {
                    if (mbar_wait(&rfull[r], (uint32_t)((tl / kTileRing) & 1), abort_flag)) {
                        v = ring[r];
                        mbar_arrive(&rempty[r]);
                    } else {
                        *abort_flag = 1;
                    }
                }
                t = __shfl_sync(0xffffffffu, v, 0);
                if (t < 0) break;
            } else if (t >= total) {
                break;
            }
            const int buf = tl & 1;
            const uint32_t tph = (uint32_t)(tl >> 1) & 1u;
            if (!mbar_wait(&tfull[buf], tph, abort_flag)) {
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            int local;
            const int g = tile_group(L, start, t, &local);
            const TcGroup &G = L.g[g];
            const int NT = G.NT, tiles_n = G.N / NT;
            const int tn = local % tiles_n;
            const int m = (local / tiles_n) * 128 + qtr * 32 + lane, n0 = tn * NT;
            const bool live = m < cnt[g];
            const size_t row = (size_t)off[g] + m;
            const float *bias = G.bias + n0;
            const float *hw = G.head_w ? G.head_w + n0 : nullptr;
            // FP8 groups: accumulator x ascale[row] x wscale[col]; BF16: x 1
            const float asc = HAS_FP8 && G.fp8 && live ? __ldg(G.ascale + row) : 1.f;
            const float *wsc = HAS_FP8 && G.fp8 ? G.wscale + n0 : nullptr;
            float hsum = 0.f;
#pragma unroll 1
            for (int c0 = chalf * (NT >> 1); c0 < (chalf + 1) * (NT >> 1); c0 += 32) {
                uint32_t r[32];
                tmem_ld32(tmem_base + ((uint32_t)(qtr * 32) << 16) + (uint32_t)(buf * half + c0), r);
                tmem_ld_wait();
                if (wsc) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) r[j] = __float_as_uint(__uint_as_float(r[j]) * (asc * __ldg(wsc + c0 + j)));
                }
                if (hw) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        float v = __uint_as_float(r[j]) + __ldg(bias + c0 + j);
                        v = v > 0.f ? v : 0.f;
                        hsum = fmaf(__ldg(hw + c0 + j), v, hsum);
                    }
                } else if (live) {
                    uint32_t pk[16], lo[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        float v0 = __uint_as_float(r[2 * j]) + __ldg(bias + c0 + 2 * j);
                        float v1 = __uint_as_float(r[2 * j + 1]) + __ldg(bias + c0 + 2 * j + 1);
                        v0 = v0 > 0.f ? v0 : 0.f;
                        v1 = v1 > 0.f ? v1 : 0.f;
                        pk[j] = pack_bf16x2(v0, v1);
                        if (L.split3) {
                            const float h0 = __uint_as_float(pk[j] << 16), h1 = __uint_as_float(pk[j] & 0xFFFF0000u);
                            lo[j] = pack_bf16x2(v0 - h0, v1 - h1);
                        }
                    }
                    uint4 *dst = reinterpret_cast<uint4 *>(L.Y + row * L.ldy + n0 + c0);
#pragma unroll
                    for (int j = 0; j < 4; ++j) dst[j] = make_uint4(pk[4 * j], pk[4 * j + 1], pk[4 * j + 2], pk[4 * j + 3]);
                    if (L.split3) {
                        uint4 *d1 = reinterpret_cast<uint4 *>(L.Y + row * L.ldy + G.N + n0 + c0);
                        uint4 *d2 = reinterpret_cast<uint4 *>(L.Y + row * L.ldy + 2 * G.N + n0 + c0);
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            d1[j] = make_uint4(pk[4 * j], pk[4 * j + 1], pk[4 * j + 2], pk[4 * j + 3]);
                            d2[j] = make_uint4(lo[4 * j], lo[4 * j + 1], lo[4 * j + 2], lo[4 * j + 3]);
                        }
                    }
                }
            }
            if (hw && live) L.partials[row * L.pstride + 2 * tn + chalf] = hsum;
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
                     "r"((uint32_t)L.tmem_cols)
                     : "memory");
    }
    if (threadIdx.x == 0) {
        if (*abort_flag) atomicOr(L.err, ERR_TC_TIMEOUT);
        if (L.rec) L.rec[2 * blockIdx.x + 1] = gtimer();
        if constexpr (DYN) {
            // the last CTA with tiles to finish clears the counters for the next launch
            // (every CTA's producer has stopped claiming before it counts itself done)
            const int participants = total < (int)gridDim.x ? total : (int)gridDim.x;
            __threadfence();
            if (atomicAdd(L.sched + 1, 1) == participants - 1) {
                L.sched[0] = 0;
                L.sched[1] = 0;
                __threadfence();
            }
        }
    }
}

// Gather the listed fp32 rows into a dense BF16 matrix, 8 values per thread:
// two 128-bit loads, one 128-bit store.
__global__ void k_gather_bf16(const int *count, const int *rows, const float *X, int ldx, int K,
                              __nv_bfloat16 *out) {
    const int M = *count;
    const int per_row = K / 8;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)M * per_row;
         i += (long long)gridDim.x * blockDim.x) {
        const int m = (int)(i / per_row), q = (int)(i % per_row);
        const float4 *src = reinterpret_cast<const float4 *>(X + (size_t)(rows ? rows[m] : m) * ldx) + 2 * q;
        const float4 a = src[0], b = src[1];
        const uint4 v = make_uint4(pack_bf16x2(a.x, a.y), pack_bf16x2(a.z, a.w), pack_bf16x2(b.x, b.y),
                                   pack_bf16x2(b.z, b.w));
        reinterpret_cast<uint4 *>(out + (size_t)m * K)[q] = v;
    }
}

using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                              const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

constexpr int kGemmSmem = 197888;   // S * stage + 1024 (alignment) + 256 (barriers), every NT

// 2-D map over [outer][inner] elements of 2 bytes (BF16) or 1 byte (E4M3
// codes, as UINT8), row stride ld elements.
bool encode2d(EncodeFn enc, CUtensorMap *m, const void *base, int inner, long long outer, int ld, int box_inner,
              int box_outer, int elem_bytes = 2) {
    const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * elem_bytes};
    const cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
    const cuuint32_t es[2] = {1, 1};
    return enc(m, elem_bytes == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
               const_cast<void *>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int col_tile(int N) { return N % 256 == 0 ? 256 : N % 128 == 0 ? 128 : 64; }

// Stacked rows: group g's rows follow the earlier groups' rows.
__global__ void k_gather_grouped_bf16(int n, const int *counts, const int *queues, int qstride,
                                      const float *const *Xp, int ldx, int K, __nv_bfloat16 *out) {
    const float *X = *Xp;
    int off[kMaxGroups + 1];
    off[0] = 0;
    for (int g = 0; g < n; ++g) off[g + 1] = off[g] + counts[g];
    const int per_row = K / 8;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)off[n] * per_row;
         i += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(i / per_row), q = (int)(i % per_row);
        int g = 0;
        while (e >= off[g + 1]) ++g;
        const int src = queues[(size_t)g * qstride + (e - off[g])];
        const float4 *p = reinterpret_cast<const float4 *>(X + (size_t)src * ldx) + 2 * q;
        const float4 a = p[0], b = p[1];
        reinterpret_cast<uint4 *>(out + (size_t)e * K)[q] =
            make_uint4(pack_bf16x2(a.x, a.y), pack_bf16x2(a.z, a.w), pack_bf16x2(b.x, b.y), pack_bf16x2(b.z, b.w));
    }
}

// Split-BF16 operand rows [hi | hi | lo] (3K columns): hi = bf16(x),
// lo = bf16(x - hi), so that with weights [W_hi | W_lo | W_hi] one BF16 GEMM
// over 3K sums hi*W_hi + hi*W_lo + lo*W_hi.
__global__ void k_gather_grouped_bf16x3(int n, const int *counts, const int *queues, int qstride,
                                        const float *const *Xp, int ldx, int K, __nv_bfloat16 *out, int min_rows) {
    const float *X = *Xp;
    int off[kMaxGroups + 1];
    off[0] = 0;
    for (int g = 0; g < n; ++g) off[g + 1] = off[g] + counts[g];
    if (off[n] < min_rows) return;
    const int per_row = K / 8;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)off[n] * per_row;
         i += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(i / per_row), q = (int)(i % per_row);
        int g = 0;
        while (e >= off[g + 1]) ++g;
        const int src = queues[(size_t)g * qstride + (e - off[g])];
        const float4 *p = reinterpret_cast<const float4 *>(X + (size_t)src * ldx) + 2 * q;
        const float4 a = p[0], b = p[1];
        const float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            hi[j] = pack_bf16x2(v[2 * j], v[2 * j + 1]);
            lo[j] = pack_bf16x2(v[2 * j] - __uint_as_float(hi[j] << 16), v[2 * j + 1] - __uint_as_float(hi[j] & 0xFFFF0000u));
        }
        uint4 *row = reinterpret_cast<uint4 *>(out + (size_t)e * 3 * K);
        row[q] = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        row[per_row + q] = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        row[2 * per_row + q] = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
}

// E4M3 codes of four values already divided by the row scale (saturating
// to +-448), packed little-endian.
__device__ __forceinline__ uint32_t pack_e4m3x4(float a, float b, float c, float d) {
    const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
    const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
    return lo | (hi << 16);
}

// One warp per row: max |x| by a shuffle reduction, then 4 codes per lane
// and 16-byte load (the row is read twice; the second pass hits L1/L2).
__device__ __forceinline__ void quant_row_e4m3(const float *x, int K, unsigned char *out, float *scale, int lane) {
    float amax = 0.f;
    for (int i = lane; i < K / 4; i += 32) {
        const float4 v = reinterpret_cast<const float4 *>(x)[i];
        amax = fmaxf(amax, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    const float inv = amax > 0.f ? 448.f / amax : 0.f;
    for (int i = lane; i < K / 4; i += 32) {
        const float4 v = reinterpret_cast<const float4 *>(x)[i];
        reinterpret_cast<uint32_t *>(out)[i] = pack_e4m3x4(v.x * inv, v.y * inv, v.z * inv, v.w * inv);
    }
    if (lane == 0) *scale = amax / 448.f;
}

__global__ void k_gather_grouped_mixed(int n, const int *counts, const int *queues, int qstride,
                                       const float *const *Xp, int ldx, int K, unsigned q8_mask,
                                       __nv_bfloat16 *out16, unsigned char *out8, float *ascale) {
    const float *X = *Xp;
    int off[kMaxGroups + 1];
    off[0] = 0;
    for (int g = 0; g < n; ++g) off[g + 1] = off[g] + counts[g];
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    for (int e = blockIdx.x * wpb + (threadIdx.x >> 5); e < off[n]; e += gridDim.x * wpb) {
        int g = 0;
        while (e >= off[g + 1]) ++g;
        const float *x = X + (size_t)queues[(size_t)g * qstride + (e - off[g])] * ldx;
        if (q8_mask & (1u << g)) {
            quant_row_e4m3(x, K, out8 + (size_t)e * K, ascale + e, lane);
        } else {
            for (int i = lane; i < K / 4; i += 32) {
                const float4 v = reinterpret_cast<const float4 *>(x)[i];
                reinterpret_cast<uint2 *>(out16 + (size_t)e * K)[i] = make_uint2(pack_bf16x2(v.x, v.y), pack_bf16x2(v.z, v.w));
            }
        }
    }
}

__global__ void k_quant_rows_e4m3(const float *X, int rows, int K, unsigned char *out, float *scale) {
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int r = blockIdx.x * wpb + (threadIdx.x >> 5); r < rows; r += gridDim.x * wpb)
        quant_row_e4m3(X + (size_t)r * K, K, out + (size_t)r * K, scale + r, lane);
}

__global__ void k_head_finalize_grouped(int n, const int *counts, TcHeads heads, const float *partials, int pstride,
                                        float *score, int sstride, int min_rows) {
    int off[kMaxGroups + 1];
    off[0] = 0;
    for (int g = 0; g < n; ++g) off[g + 1] = off[g] + counts[g];
    if (off[n] < min_rows) return;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < off[n]; e += gridDim.x * blockDim.x) {
        int g = 0;
        while (e >= off[g + 1]) ++g;
        const float *pp = partials + (size_t)e * pstride;
        float s = 0.f;
        for (int j = 0; j < heads.tiles[g]; ++j) s += pp[j];
        score[(size_t)g * sstride + (e - off[g])] = (float)((double)heads.b[g] + (double)s);
    }
}

}  // namespace

bool tc_gemm_supported(int K, int N) { return K >= 64 && K % 64 == 0 && N >= 64 && N % 64 == 0 && K <= 65536; }

bool tc_gemm_fp8_supported(int K, int N) { return tc_gemm_supported(K, N) && K % 128 == 0; }

hydro_status tc_gemm_init(void **encode) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult qr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr);
    if (e != cudaSuccess || qr != cudaDriverEntryPointSuccess || !fn) {
        g_gemm_err = "cuTensorMapEncodeTiled entry point not available";
        return HYDRO_ECUDA;
    }
    *encode = fn;
    cudaError_t r = cudaFuncSetAttribute(k_gemm_grouped_bf16_tc<false, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem);
    if (r == cudaSuccess)
        r = cudaFuncSetAttribute(k_gemm_grouped_bf16_tc<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kGemmSmem);
    if (r == cudaSuccess)
        r = cudaFuncSetAttribute(k_gemm_grouped_bf16_tc<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kGemmSmem);
    if (r == cudaSuccess)
        r = cudaFuncSetAttribute(k_gemm_grouped_bf16_tc<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kGemmSmem);
    if (r != cudaSuccess) {
        g_gemm_err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(r);
        return HYDRO_ECUDA;
    }
    return HYDRO_OK;
}

hydro_status tc_gemm_grouped_run(void *encode, const TcGemmGroup *groups, int n, __nv_bfloat16 *Y, int ldy,
                                 float *partials, int pstride, int sms, cudaStream_t st, unsigned int *err,
                                 bool split3, int min_rows, const TcSched *sched) {
    if (!encode || n < 1 || n > kMaxGroups || (ldy % 8) != 0) {
        g_gemm_err = "tensor-core GEMM not ready or bad group list";
        return HYDRO_EUNSUPPORTED;
    }
    EncodeFn enc = reinterpret_cast<EncodeFn>(encode);
    TcLaunch L;
    memset(&L, 0, sizeof L);
    int nt_max = 64;
    long long tiles = 0;
    for (int g = 0; g < n; ++g) {
        const TcGemmGroup &h = groups[g];
        const bool fp8 = h.W8 != nullptr;
        if (!h.W && !fp8) {   // rows only: the group takes its place in the stacking, no tiles
            L.g[g].count = h.count;
            continue;
        }
        if (fp8 && (!tc_gemm_fp8_supported(h.K, h.N) || !h.X8 || !h.ascale || !h.wscale || (h.ldx % 16) != 0)) {
            g_gemm_err = "tensor-core GEMM: unsupported FP8 group";
            return HYDRO_EUNSUPPORTED;
        }
        if (!tc_gemm_supported(h.K, h.N) || (h.nt && (h.nt % 64 || h.nt > 256 || h.N % h.nt)) || h.x_rows < 1 || (h.ldx % 8) != 0 || h.ldx < h.K ||
            (!h.head_w && (split3 ? 3 * h.N : h.N) > ldy) ||
            (h.head_w && 2 * (h.N / (h.nt ? h.nt : col_tile(h.N))) > pstride)) {
            g_gemm_err = "tensor-core GEMM: unsupported group shape";
            return HYDRO_EUNSUPPORTED;
        }
        TcGroup &G = L.g[g];
        G.K = h.K;
        G.N = h.N;
        G.NT = h.nt ? h.nt : col_tile(h.N);
        G.count = h.count;
        G.bias = h.bias;
        G.head_w = h.head_w;
        G.fp8 = fp8 ? 1 : 0;
        G.ascale = h.ascale;
        G.wscale = h.wscale;
        nt_max = G.NT > nt_max ? G.NT : nt_max;
        const bool mapped = fp8 ? encode2d(enc, &G.tmA, h.X8, h.K, h.x_rows, h.ldx, 128, 128, 1) &&
                                      encode2d(enc, &G.tmB, h.W8, h.K, h.N, h.K, 128, G.NT, 1)
                                : encode2d(enc, &G.tmA, h.X, h.K, h.x_rows, h.ldx, 64, 128) &&
                                      encode2d(enc, &G.tmB, h.W, h.K, h.N, h.K, 64, G.NT);
        if (!mapped) {
            g_gemm_err = "cuTensorMapEncodeTiled failed";
            return HYDRO_ECUDA;
        }
        tiles += ((h.x_rows + 127) / 128) * (h.N / G.NT);
    }
    L.n = n;
    L.Y = Y;
    L.ldy = ldy;
    L.partials = partials;
    L.pstride = pstride;
    L.err = err;
    L.stage_bytes = kA_BYTES + nt_max * 128;
    L.S = (kGemmSmem - 1280) / L.stage_bytes;
    if (L.S > kMaxStages) L.S = kMaxStages;
    L.tmem_cols = 2 * nt_max;
    L.split3 = split3 ? 1 : 0;
    L.min_rows = min_rows;
    for (int g = 0; g < n; ++g) L.order[g] = g;
    const bool dyn = sched && sched->data_aware && sched->counters;
    if (dyn) {
        // heaviest tiles first: a tile's work is 128 rows x NT columns x K (half for E4M3 operands)
        auto work = [&](int g) -> long long {
            const TcGroup &G = L.g[g];
            return G.NT ? (long long)G.K * G.NT / (G.fp8 ? 2 : 1) : 0;
        };
        for (int a = 1; a < n; ++a)
            for (int b = a; b > 0 && work(L.order[b]) > work(L.order[b - 1]); --b) std::swap(L.order[b], L.order[b - 1]);
        L.sched = sched->counters;
    }
    L.rec = sched ? sched->rec : nullptr;
    if (tiles == 0) return HYDRO_OK;   // only rows-only groups
    const int grid = (int)(tiles < sms ? tiles : sms);
    bool any_fp8 = false;
    for (int g = 0; g < n; ++g) any_fp8 = any_fp8 || L.g[g].fp8;
    if (any_fp8 && dyn)
        k_gemm_grouped_bf16_tc<true, true><<<grid, kGemmThreads, kGemmSmem, st>>>(L);
    else if (any_fp8)
        k_gemm_grouped_bf16_tc<true, false><<<grid, kGemmThreads, kGemmSmem, st>>>(L);
    else if (dyn)
        k_gemm_grouped_bf16_tc<false, true><<<grid, kGemmThreads, kGemmSmem, st>>>(L);
    else
        k_gemm_grouped_bf16_tc<false, false><<<grid, kGemmThreads, kGemmSmem, st>>>(L);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_gemm_err = std::string("launch: ") + cudaGetErrorString(e);
        return HYDRO_ECUDA;
    }
    return HYDRO_OK;
}

hydro_status tc_gemm_run(void *encode, const int *count, const __nv_bfloat16 *X, int K, const __nv_bfloat16 *W,
                         const float *bias, int N, __nv_bfloat16 *Y, int max_rows, int sms, cudaStream_t st,
                         unsigned int *err, const float *head_w, float *partials) {
    TcGemmGroup g{count, X, K, max_rows, W, bias, head_w, K, N, 0};
    return tc_gemm_grouped_run(encode, &g, 1, Y, N, partials, tc_gemm_col_tiles(N), sms, st, err);
}

int tc_gemm_col_tiles(int N) { return 2 * (N / col_tile(N)); }

int tc_gemm_head_parts(int N, int nt) { return 2 * (N / (nt ? nt : col_tile(N))); }

void launch_gather_bf16(const int *count, const int *rows, const float *X, int ldx, int K, __nv_bfloat16 *out,
                        int max_rows, int sms, cudaStream_t st) {
    long long work = (long long)max_rows * (K / 8);
    int grid = (int)((work + 255) / 256);
    if (grid > sms * 8) grid = sms * 8;
    if (grid < 1) grid = 1;
    k_gather_bf16<<<grid, 256, 0, st>>>(count, rows, X, ldx, K, out);
}

void launch_gather_grouped_bf16(int n, const int *counts, const int *queues, int qstride, const float *const *Xp,
                                int ldx, int K, __nv_bfloat16 *out, int max_rows, int sms, cudaStream_t st) {
    long long work = (long long)max_rows * (K / 8);
    int grid = (int)((work + 255) / 256);
    if (grid > sms * 8) grid = sms * 8;
    if (grid < 1) grid = 1;
    k_gather_grouped_bf16<<<grid, 256, 0, st>>>(n, counts, queues, qstride, Xp, ldx, K, out);
}

void launch_gather_grouped_bf16x3(int n, const int *counts, const int *queues, int qstride, const float *const *Xp,
                                  int ldx, int K, __nv_bfloat16 *out, int max_rows, int sms, cudaStream_t st,
                                  int min_rows) {
    long long work = (long long)max_rows * (K / 8);
    int grid = (int)((work + 255) / 256);
    if (grid > sms * 8) grid = sms * 8;
    if (grid < 1) grid = 1;
    k_gather_grouped_bf16x3<<<grid, 256, 0, st>>>(n, counts, queues, qstride, Xp, ldx, K, out, min_rows);
}

void launch_gather_grouped_mixed(int n, const int *counts, const int *queues, int qstride, const float *const *Xp,
                                 int ldx, int K, unsigned q8_mask, __nv_bfloat16 *out16, unsigned char *out8,
                                 float *ascale, int max_rows, int sms, cudaStream_t st) {
    int grid = (max_rows + 7) / 8;   // 8 warps, one row each
    if (grid > sms * 8) grid = sms * 8;
    if (grid < 1) grid = 1;
    k_gather_grouped_mixed<<<grid, 256, 0, st>>>(n, counts, queues, qstride, Xp, ldx, K, q8_mask, out16, out8,
                                                 ascale);
}

void launch_quant_rows_e4m3(const float *X, int rows, int K, unsigned char *out, float *scale, int sms,
                            cudaStream_t st) {
    int grid = (rows + 7) / 8;
    if (grid > sms * 8) grid = sms * 8;
    if (grid < 1) grid = 1;
    k_quant_rows_e4m3<<<grid, 256, 0, st>>>(X, rows, K, out, scale);
}

void launch_head_finalize_grouped(int n, const int *counts, const TcHeads &heads, const float *partials, int pstride,
                                  float *score, int sstride, int max_rows, int sms, cudaStream_t st, int min_rows) {
    int grid = (max_rows + 255) / 256;
    if (grid > sms * 4) grid = sms * 4;
    if (grid < 1) grid = 1;
    k_head_finalize_grouped<<<grid, 256, 0, st>>>(n, counts, heads, partials, pstride, score, sstride, min_rows);
}

const char *tc_gemm_last_error() { return g_gemm_err.c_str(); }

}  // namespace hydro
