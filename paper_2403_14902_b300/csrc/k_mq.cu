// Kernels of multi-query session steps (rounds of grouped launches).
//
// A step stacks every query's chunk; round r sends each surviving tuple to
// the pool UDF of the r-th slot of its query's order (Sec. 4.1 rank order per
// query, Sec. 3.3 eager dropping), evaluates all groups per layer depth in one
// persistent launch (Sec. 5.1 "Batch-agnostic Parallelization": many workers'
// work on one GPU at once), tests the scores against each tuple's own query
// threshold, rechecks the band around it at higher precision, and keeps the
// survivors.  Queue and list order is by atomics: every verdict and count is
// per tuple, so the results do not depend on it.
#include <math.h>

#include "mq.h"
#include "simt_tile.cuh"

namespace hydro {

namespace {

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// Append `want` lanes' items to a list whose length is *counter: one atomic
// per distinct counter among the warp's active lanes.  Returns each wanting
// lane's position.
__device__ __forceinline__ int warp_append(int *counter, bool want) {
    const unsigned active = __activemask();
    const unsigned mask = __ballot_sync(active, want);
    if (!want) return -1;
    const unsigned peers = __match_any_sync(mask, reinterpret_cast<uintptr_t>(counter));
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (lane_id() == leader) base = atomicAdd(counter, __popc(peers));
    base = __shfl_sync(peers, base, leader);
    return base + __popc(peers & ((1u << lane_id()) - 1u));
}

// Add 1 to *p for every active lane that passes want: one atomic per
// distinct address.
__device__ __forceinline__ void warp_count(unsigned long long *p, bool want) {
    const unsigned active = __activemask();
    const unsigned mask = __ballot_sync(active, want);
    if (!want) return;
    const unsigned peers = __match_any_sync(mask, reinterpret_cast<uintptr_t>(p));
    if (lane_id() == __ffs(peers) - 1) atomicAdd(p, (unsigned long long)__popc(peers));
}

// True in the last block of the grid to finish (the others' writes are
// visible to it).  The ticket is reset for the next launch.
__device__ __forceinline__ bool last_block(int *ticket) {
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1) == (int)gridDim.x - 1;
        if (last) *ticket = 0;
    }
    __syncthreads();
    return last;
}

__device__ __forceinline__ void set_cond(const Cond &c, bool v) {
    if (c.h) cudaGraphSetConditional((cudaGraphConditionalHandle)c.h, v ? 1u : 0u);
    if (c.flag) *c.flag = v ? 1 : 0;
}

// Query (tables, history) of virtual query v.
__device__ __forceinline__ int rq(const MqDev &d, int v) { return v / d.K; }

// Slot of tuple e (batch v) in round r: its own order (learned sessions) or
// its batch's.
__device__ __forceinline__ int slot_of(const MqDev &d, int e, int q, int r) {
    return d.order_t ? d.order_t[(size_t)e * kMqSlots + r] : d.order[q * kMqSlots + r];
}

__device__ __forceinline__ unsigned long long *ctr(StatRow *r, int field) {
    return reinterpret_cast<unsigned long long *>(r) + field;
}
enum { F_EVAL = 0, F_PASS = 1, F_RX3 = 2, F_R32 = 3, F_R64 = 4 };

int grid_for(long long work, int per_block, int sms, int per_sm) {
    long long g = (work + per_block - 1) / per_block;
    const long long cap = (long long)sms * per_sm;
    if (g > cap) g = cap;
    return g < 1 ? 1 : (int)g;
}

// ------------------------------------------------------------ step setup

// Offsets of the step, query of every tuple, first alive list (every tuple),
// cleared per-tuple flags, statistics and round counters.
__global__ void __launch_bounds__(256) k_mq_init(MqDev d, Cond round0) {
    __shared__ int s_off[kMqMaxQ + 1];
    if (threadIdx.x == 0) {
        int o = 0;
        for (int q = 0; q < d.Q; ++q) {
            s_off[q] = o;
            o += d.hdr->counts[q];
        }
        s_off[d.Q] = o;
    }
    __syncthreads();
    const int n = min(s_off[d.Q], d.cap);
    if (blockIdx.x == 0) {
        for (int i = threadIdx.x; i <= d.Q; i += blockDim.x) d.off[i] = s_off[i];
        for (int i = threadIdx.x; i < d.Q * kMqSlots; i += blockDim.x) d.rows[i] = StatRow{};
        for (int i = threadIdx.x; i < d.Q; i += blockDim.x) d.npass[i] = 0;
        for (int i = threadIdx.x; i < kMqGates; i += blockDim.x) d.gates[i] = 0;
        __syncthreads();
        if (threadIdx.x == 0) {
            if (s_off[d.Q] > d.cap) atomicOr(d.err, ERR_COUNT_RANGE);
            RoundCounters z{};
            z.alive[0] = n;
            *d.rc = z;
            set_cond(round0, n > 0);
        }
    }
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        int lo = 0, hi = d.Q - 1;   // last q with s_off[q] <= e
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_off[mid] <= e) lo = mid;
            else hi = mid - 1;
        }
        d.qid[e] = (unsigned short)lo;
        d.alive[0][e] = e;
        d.visited[e] = 0;
        d.label[e] = 0;
        d.ok[e] = 0;
    }
}

// Per query (one warp each): its batch number, warmup flag and slot order
// for the step from its own statistics of the batches before (lag 0): the
// window [b - W, b - 1], falling back to the warmup batches for a slot not
// evaluated in the window; rank c (e + 2) / (e - p + 1) compared exactly in
// 128-bit integers, ties to the lower slot.
__global__ void k_mq_router(MqDev d, MqHist h) {
    const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int i = lane_id();
    if (q >= d.Q) return;
    const int count = d.hdr->counts[q];
    const int qq = rq(d, q);
    const int P = d.np[qq];
    if (count <= 0) {
        if (i == 0) {
            d.bidx[q] = -1;
            d.evall[q] = 0;
        }
        if (i < kMqSlots) d.order[q * kMqSlots + i] = (unsigned char)i;
        return;
    }
    // sub-batches are filled in order, so this is the query's batch bdone + k
    const long long b = h.bdone[qq] + (q - qq * d.K);
    if (i == 0) d.bidx[q] = b;
    if (h.static_order) {
        if (i == 0) d.evall[q] = 0;
        if (i < kMqSlots) d.order[q * kMqSlots + i] = (unsigned char)i;
        return;
    }
    const long long last = b - 1 - h.lag;
    if (b < h.warmup || last < 0) {
        if (i == 0) d.evall[q] = b < h.warmup ? 1 : 0;
        if (i < kMqSlots) d.order[q * kMqSlots + i] = (unsigned char)i;
        return;
    }
    if (i == 0) d.evall[q] = 0;
    const long long lo = last - h.window + 1 > 0 ? last - h.window + 1 : 0;
    long long E = 0, Pp = 0;
    unsigned long long c = 0;
    if (i < P) {
        c = (unsigned long long)d.cost[qq * kMqSlots + i];
        for (long long bb = lo; bb <= last; ++bb) {
            const StatRow &r = h.ring[((size_t)qq * h.R + (size_t)(bb % h.R)) * kMqSlots + i];
            E += r.evaluated;
            Pp += r.passed;
        }
        if (E == 0) {
            const int nw = (int)(h.warmup < last + 1 ? h.warmup : last + 1);
            for (int w = 0; w < nw; ++w) {
                const StatRow &r = h.warm[((size_t)qq * h.warmup + w) * kMqSlots + i];
                E += r.evaluated;
                Pp += r.passed;
            }
        }
    }
    int pos = 0;
    for (int j = 0; j < P; ++j) {
        const long long Ej = __shfl_sync(0xffffffffu, E, j);
        const long long Pj = __shfl_sync(0xffffffffu, Pp, j);
        const unsigned long long cj = __shfl_sync(0xffffffffu, c, j);
        if (i >= P || j == i) continue;
        const unsigned __int128 lhs = (unsigned __int128)cj * (unsigned long long)(Ej + 2) * (unsigned long long)(E - Pp + 1);
        const unsigned __int128 rhs = (unsigned __int128)c * (unsigned long long)(E + 2) * (unsigned long long)(Ej - Pj + 1);
        pos += (lhs < rhs || (lhs == rhs && j < i)) ? 1 : 0;
    }
    if (i < P) d.order[q * kMqSlots + pos] = (unsigned char)i;
}

// ------------------------------------------------------------ rounds

// Round r: every alive tuple joins the queue of the pool UDF of its query's
// r-th slot.  Also clears the next alive list's length.
__global__ void __launch_bounds__(256) k_mq_partition(MqDev d, int r) {
    const int cur = r & 1;
    const int n = d.rc->alive[cur];
    if (blockIdx.x == 0 && threadIdx.x == 0) d.rc->alive[cur ^ 1] = 0;
    for (int m0 = blockIdx.x * blockDim.x; m0 < n; m0 += gridDim.x * blockDim.x) {
        const int m = m0 + threadIdx.x;
        int e = 0, g = 0;
        const bool live = m < n;
        if (live) {
            e = d.alive[cur][m];
            const int q = d.qid[e];
            const int slot = slot_of(d, e, q, r);
            g = d.udf[rq(d, q) * kMqSlots + slot];
        }
        const int pos = warp_append(live ? &d.rc->n[LV_MAIN][g] : nullptr, live);
        if (live) d.list[LV_MAIN][(size_t)g * d.cap + pos] = e;
    }
}

// Stacked grouped FP32 layer: tiles group by group, rows of group g at
// off_g; depth 0 reads X rows through the queue lists.
__global__ void __launch_bounds__(256) k_mq_layer_f32(MqLayers L) {
    __shared__ __align__(16) float As[2][16][68];
    __shared__ __align__(16) float Ws[2][16][68];
    int off[kMqPool + 1], start[kMqPool + 1];
    off[0] = 0;
    start[0] = 0;
    for (int g = 0; g < L.n; ++g) {
        const int c = L.counts[g];
        off[g + 1] = off[g] + c;
        start[g + 1] = start[g] + (L.l[g].W ? ((c + 63) / 64) * ((L.l[g].N + 63) / 64) : 0);
    }
    const float *X = L.hdr->X;
    for (int tile = blockIdx.x; tile < start[L.n]; tile += gridDim.x) {
        int g = 0;
        while (tile >= start[g + 1]) ++g;
        const MqLayer &l = L.l[g];
        const int local = tile - start[g], tn = (l.N + 63) / 64;
        const int *rows = L.rows ? L.rows + (size_t)g * L.cap : nullptr;
        const float *in = rows ? X : l.in + (size_t)off[g] * l.ldin;
        mlp_tile_f32(L.counts[g], (local / tn) * 64, (local % tn) * 64, rows, in, rows ? L.ldx : l.ldin, l.W, l.b,
                     L.Y + (size_t)off[g] * L.ldy, L.ldy, l.K, l.N, l.norelu ? 0 : 1, As, Ws);
    }
}

// Stacked grouped one-output last layer: a warp per row; score[g*sstride + m].
__global__ void __launch_bounds__(256) k_mq_dot_f32(MqLayers L, float *score, int sstride) {
    int off[kMqPool + 1];
    off[0] = 0;
    for (int g = 0; g < L.n; ++g) off[g + 1] = off[g] + L.counts[g];
    const float *X = L.hdr->X;
    for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < off[L.n]; w += (gridDim.x * blockDim.x) >> 5) {
        int g = 0;
        while (w >= off[g + 1]) ++g;
        const MqLayer &l = L.l[g];
        if (!l.W) continue;
        const int m = w - off[g];
        const float *x = L.rows ? X + (size_t)L.rows[(size_t)g * L.cap + m] * L.ldx : l.in + (size_t)w * l.ldin;
        float s = 0.f;
        for (int k = lane_id(); k < l.K; k += 32) s = fmaf(x[k], l.W[k], s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane_id() == 0) score[(size_t)g * sstride + m] = s + l.bconst;
    }
}

// Decide the entries of level `in`: the score of each list entry against
// its tuple's own threshold; within the level's margin the entry goes on to
// level `out`'s list of the same group.  Level 0 counts the evaluations and
// marks the slot visited; levels 1 and 2 count their rechecks (the FP64
// level counts its own).  The split-BF16 level runs only on a band of at
// least kMinSplitRows rows: below that its launches return at once and every
// entry passes on to the FP32 level unscored.
// heads.tiles[g] > 0 (tensor-core levels): the entry's score is summed here
// from the GEMM's head partials (row i of the stacked operand, fixed order)
// plus the head bias, instead of read from the level's score list.
__global__ void __launch_bounds__(256) k_mq_classify(MqDev d, int r, int in, int out, Cond next, int next_min,
                                                     TcHeads heads, const float *partials, int pstride) {
    const int *cnts = d.rc->n[in];
    const int *lists = d.list[in];
    const float *sc = d.score[in];
    const float *margin = d.margin[in];
    int *next_cnt = d.rc->n[out];
    int *next_list = d.list[out];
    const int rfield = in == LV_X3 ? F_RX3 : in == LV_F32 ? F_R32 : -1;
    int off[kMqPool + 1];
    off[0] = 0;
    for (int g = 0; g < d.G; ++g) off[g + 1] = off[g] + cnts[g];
    const bool skipped = in == LV_X3 && off[d.G] < kMinSplitRows;
    for (int i0 = blockIdx.x * blockDim.x; i0 < off[d.G]; i0 += gridDim.x * blockDim.x) {
        const int i = i0 + threadIdx.x;
        const bool live = i < off[d.G];
        int g = 0, m = 0, e = 0, q = 0, slot = 0;
        bool inband = false, pass = false;
        if (live) {
            while (i >= off[g + 1]) ++g;
            m = i - off[g];
            e = lists[(size_t)g * d.cap + m];
            q = d.qid[e];
            slot = slot_of(d, e, q, r);
            if (skipped) {
                inband = true;
            } else {
                const double t = d.thr[rq(d, q) * kMqSlots + slot];
                double s;
                if (partials) {
                    const float *pp = partials + (size_t)i * pstride;
                    float a = 0.f;
                    for (int j = 0; j < heads.tiles[g]; ++j) a += pp[j];
                    s = (double)heads.b[g] + (double)a;
                } else {
                    s = (double)sc[(size_t)g * d.cap + m];
                }
                inband = fabs(s - t) <= (double)margin[g];
                pass = !inband && s > t;
                d.ok[e] = (unsigned char)pass;
                if (pass) d.label[e] |= (unsigned char)(1u << slot);
            }
            if (in == LV_MAIN) d.visited[e] |= (unsigned char)(1u << slot);
        }
        StatRow *row = d.rows + q * kMqSlots + slot;
        if (in == LV_MAIN) warp_count(ctr(row, F_EVAL), live);
        warp_count(ctr(row, F_PASS), live && pass);
        // level-0 entries of groups that skip level 1 go to the FP32 level
        const bool direct = in == LV_MAIN && ((d.lv1_skip >> g) & 1u);
        const int pos = warp_append(live && inband ? (direct ? &d.rc->n[LV_F32][g] : &next_cnt[g]) : nullptr,
                                    live && inband);
        if (live && inband) (direct ? d.list[LV_F32] : next_list)[(size_t)g * d.cap + pos] = e;
        if (rfield >= 0) warp_count(ctr(row, rfield), live && !skipped);
    }
    if (next.flag && last_block(&d.rc->ticket[in]) && threadIdx.x == 0) {
        __threadfence();
        int tot = 0;
        for (int g = 0; g < d.G; ++g) tot += *((volatile int *)&next_cnt[g]);
        set_cond(next, tot >= next_min);
    }
}

// Lane `lane`'s share of the dot product w . x over K (fp32 weights, x in
// float or T): 16-byte loads and four independent accumulators when K is a
// multiple of 128 (every row 16-byte aligned), else one element at a time.
__device__ __forceinline__ void load4(const float *p, float (&v)[4]) {
    const float4 a = *reinterpret_cast<const float4 *>(p);
    v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w;
}
__device__ __forceinline__ void load4(const float *p, double (&v)[4]) {
    const float4 a = *reinterpret_cast<const float4 *>(p);
    v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w;
}
__device__ __forceinline__ void load4(const double *p, double (&v)[4]) {
    const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
}
template <typename T, typename X>
__device__ __forceinline__ T lane_dot(const float *w, const X *x, int K) {
    const int lane = lane_id();
    if ((K & 127) == 0) {
        T a[4] = {0, 0, 0, 0};
        for (int k = 4 * lane; k < K; k += 128) {
            float wv[4];
            T xv[4];
            load4(w + k, wv);
            load4(x + k, xv);
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] += (T)wv[i] * xv[i];
        }
        return (a[0] + a[1]) + (a[2] + a[3]);
    }
    T s = 0;
    for (int k = lane; k < K; k += 32) s += (T)w[k] * (T)x[k];
    return s;
}

// Band levels run layer-parallel as skinny GEMMs: a CTA computes 32 output
// neurons (lane = neuron, coalesced loads of the transposed weights
// WT[k][n]) for up to kBandE entries (accumulators in registers), its 8
// warps splitting K and summing through shared memory.  Entries are stacked
// group by group (the first `cap_lv` of the level); activations in T
// (float: the FP32 level, double: FP64).
constexpr int kBandE = 16;
constexpr int kBandWarps = 8;

__device__ __forceinline__ void band_offsets(const MqDev &d, const GroupedMlps &mlps, int level, int cap_lv,
                                             int depth, int *off, int *wstart) {
    const int *cnts = d.rc->n[level];
    off[0] = 0;
    wstart[0] = 0;
    for (int g = 0; g < d.G; ++g) {
        const int lim = max(0, min(cnts[g], cap_lv - off[g]));
        off[g + 1] = off[g] + lim;
        const MlpDev &m = mlps.m[g];
        const int blocks = (lim + kBandE - 1) / kBandE;
        wstart[g + 1] = wstart[g] + (depth >= 0 && depth + 1 < m.n_layers ? blocks * ((m.dims[depth + 1] + 31) / 32) : 0);
    }
}

template <typename T>
__global__ void __launch_bounds__(32 * kBandWarps) k_mq_band_layer(MqDev d, GroupedMlps mlps, int level, int depth,
                                                                   T *act0, T *act1, int ld, int cap_lv) {
    __shared__ T part[kBandWarps][kBandE][32];
    int off[kMqPool + 1], wstart[kMqPool + 1];
    band_offsets(d, mlps, level, cap_lv, depth, off, wstart);
    const T *in_act = (depth & 1) ? act0 : act1;   // depth - 1 wrote act[(depth - 1) & 1]
    T *out_act = (depth & 1) ? act1 : act0;
    const float *X = d.hdr->X;
    const int *list = d.list[level];
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    for (int item = blockIdx.x; item < wstart[d.G]; item += gridDim.x) {
        int g = 0;
        while (item >= wstart[g + 1]) ++g;
        const MlpDev &m = mlps.m[g];
        const int N = m.dims[depth + 1], K = m.dims[depth];
        const int nt = (N + 31) / 32, local = item - wstart[g];
        const int o = (local % nt) * 32 + lane, e0 = (local / nt) * kBandE;
        const int ne = min(kBandE, (off[g + 1] - off[g]) - e0);
        const float *WT = m.WT[depth];
        // this warp's share of K
        const int kc = (K + kBandWarps - 1) / kBandWarps;
        const int k0 = warp * kc, k1 = min(K, k0 + kc);
        T acc[kBandE];
#pragma unroll
        for (int e = 0; e < kBandE; ++e) acc[e] = 0;
        if (o < N) {
            if (depth == 0) {
                const float *xr[kBandE];
#pragma unroll
                for (int e = 0; e < kBandE; ++e)
                    xr[e] = X + (size_t)list[(size_t)g * d.cap + e0 + (e < ne ? e : 0)] * d.dim;
#pragma unroll 4
                for (int k = k0; k < k1; ++k) {
                    const T wk = (T)WT[(size_t)k * N + o];
#pragma unroll
                    for (int e = 0; e < kBandE; ++e)
                        if (e < ne) acc[e] += wk * (T)xr[e][k];
                }
            } else {
                const T *xr[kBandE];
#pragma unroll
                for (int e = 0; e < kBandE; ++e) xr[e] = in_act + (size_t)(off[g] + e0 + (e < ne ? e : 0)) * ld;
#pragma unroll 4
                for (int k = k0; k < k1; ++k) {
                    const T wk = (T)WT[(size_t)k * N + o];
#pragma unroll
                    for (int e = 0; e < kBandE; ++e)
                        if (e < ne) acc[e] += wk * xr[e][k];
                }
            }
        }
#pragma unroll
        for (int e = 0; e < kBandE; ++e) part[warp][e][lane] = acc[e];
        __syncthreads();
        // warp w sums entries w, w + 8 over the 8 warps' shares
        for (int e = warp; e < ne; e += kBandWarps) {
            T s = 0;
#pragma unroll
            for (int w2 = 0; w2 < kBandWarps; ++w2) s += part[w2][e][lane];
            if (o < N) {
                s += (T)m.b[depth][o];
                out_act[(size_t)(off[g] + e0 + e) * ld + o] = s > (T)0 ? s : (T)0;
            }
        }
        __syncthreads();
    }
}

// For bands of a few entries (the FP64 level): a warp per (output neuron,
// block of up to kWpnE entries), spreading even one entry's layer over all
// SMs; each weight row is read once per block.
constexpr int kWpnE = 8;

__device__ __forceinline__ void wpn_offsets(const MqDev &d, const GroupedMlps &mlps, int level, int cap_lv,
                                             int depth, int *off, int *wstart) {
    const int *cnts = d.rc->n[level];
    off[0] = 0;
    wstart[0] = 0;
    for (int g = 0; g < d.G; ++g) {
        const int lim = max(0, min(cnts[g], cap_lv - off[g]));
        off[g + 1] = off[g] + lim;
        const MlpDev &m = mlps.m[g];
        const int blocks = (lim + kWpnE - 1) / kWpnE;
        wstart[g + 1] = wstart[g] + (depth >= 0 && depth + 1 < m.n_layers ? blocks * m.dims[depth + 1] : 0);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_mq_band_layer_wpn(MqDev d, GroupedMlps mlps, int level, int depth, T *act0,
                                                       T *act1, int ld, int cap_lv) {
    int off[kMqPool + 1], wstart[kMqPool + 1];
    wpn_offsets(d, mlps, level, cap_lv, depth, off, wstart);
    const T *in_act = (depth & 1) ? act0 : act1;   // depth - 1 wrote act[(depth - 1) & 1]
    T *out_act = (depth & 1) ? act1 : act0;
    const float *X = d.hdr->X;
    const int *list = d.list[level];
    const int lane = lane_id();
    for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < wstart[d.G]; w += (gridDim.x * blockDim.x) >> 5) {
        int g = 0;
        while (w >= wstart[g + 1]) ++g;
        const MlpDev &m = mlps.m[g];
        const int N = m.dims[depth + 1], K = m.dims[depth];
        const int local = w - wstart[g];
        const int o = local % N, e0 = (local / N) * kWpnE;
        const int ne = min(kWpnE, (off[g + 1] - off[g]) - e0);
        const float *wr = m.W[depth] + (size_t)o * K;
        const void *xr[kWpnE];
#pragma unroll
        for (int e = 0; e < kWpnE; ++e) {
            const int el = e0 + (e < ne ? e : 0);
            xr[e] = depth == 0 ? (const void *)(X + (size_t)list[(size_t)g * d.cap + el] * d.dim)
                               : (const void *)(in_act + (size_t)(off[g] + el) * ld);
        }
        T acc[kWpnE];
#pragma unroll
        for (int e = 0; e < kWpnE; ++e) acc[e] = 0;
        if ((K & 127) == 0) {
#pragma unroll 2
            for (int k = 4 * lane; k < K; k += 128) {
                float wv[4];
                load4(wr + k, wv);
#pragma unroll
                for (int e = 0; e < kWpnE; ++e) {
                    if (e >= ne) break;
                    T xv[4];
                    if (depth == 0) load4(static_cast<const float *>(xr[e]) + k, xv);
                    else load4(static_cast<const T *>(xr[e]) + k, xv);
#pragma unroll
                    for (int i = 0; i < 4; ++i) acc[e] += (T)wv[i] * xv[i];
                }
            }
        } else {
            for (int k = lane; k < K; k += 32) {
                const T wk = (T)wr[k];
#pragma unroll
                for (int e = 0; e < kWpnE; ++e) {
                    if (e >= ne) break;
                    const T xk = depth == 0 ? (T) static_cast<const float *>(xr[e])[k] : static_cast<const T *>(xr[e])[k];
                    acc[e] += wk * xk;
                }
            }
        }
        const T bo = (T)m.b[depth][o];
#pragma unroll
        for (int e = 0; e < kWpnE; ++e) {
            if (e >= ne) break;
            T s = acc[e];
#pragma unroll
            for (int dd = 16; dd > 0; dd >>= 1) s += __shfl_xor_sync(0xffffffffu, s, dd);
            s += bo;
            if (lane == 0) out_act[(size_t)(off[g] + e0 + e) * ld + o] = s > (T)0 ? s : (T)0;
        }
    }
}

// The one-output last layer, a warp per entry, and the verdict.  FP32 level:
// decided unless within margin_fp32 of the threshold, else on to the FP64
// level (whose condition `next` the last block sets).  FP64 level: exact.
template <typename T>
__global__ void __launch_bounds__(256) k_mq_band_final(MqDev d, GroupedMlps mlps, int level, int r, T *act0,
                                                       T *act1, int ld, int cap_lv, Cond next) {
    int off[kMqPool + 1], wstart[kMqPool + 1];
    band_offsets(d, mlps, level, cap_lv, -1, off, wstart);
    const float *X = d.hdr->X;
    const int *list = d.list[level];
    for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < off[d.G]; j += (gridDim.x * blockDim.x) >> 5) {
        int g = 0;
        while (j >= off[g + 1]) ++g;
        const MlpDev &m = mlps.m[g];
        const int L = m.n_layers, K = m.dims[L - 1];
        const int el = j - off[g];
        const int e = list[(size_t)g * d.cap + el];
        const float *wr = m.W[L - 1];
        T s = L == 1 ? lane_dot<T>(wr, X + (size_t)e * d.dim, K)
                     : lane_dot<T>(wr, (((L - 2) & 1) ? act1 : act0) + (size_t)j * ld, K);
#pragma unroll
        for (int dd = 16; dd > 0; dd >>= 1) s += __shfl_xor_sync(0xffffffffu, s, dd);
        if (lane_id() != 0) continue;
        s += (T)m.b[L - 1][0];
        const int q = d.qid[e];
        const int slot = slot_of(d, e, q, r);
        const double t = d.thr[rq(d, q) * kMqSlots + slot];
        StatRow *row = d.rows + q * kMqSlots + slot;
        bool pass;
        if (sizeof(T) == 4) {
            // FP32: the float score, then the FP32 test
            const double sf = (double)(float)s;
            atomicAdd(ctr(row, F_R32), 1ull);
            if (fabs(sf - t) <= (double)d.margin[LV_F32][g]) {
                const int pos = atomicAdd(&d.rc->n[LV_F64][g], 1);
                d.list[LV_F64][(size_t)g * d.cap + pos] = e;
                continue;
            }
            pass = sf > t;
        } else {
            pass = (double)s > t;
            atomicAdd(ctr(row, F_R64), 1ull);
        }
        d.ok[e] = (unsigned char)pass;
        if (pass) {
            d.label[e] |= (unsigned char)(1u << slot);
            atomicAdd(ctr(row, F_PASS), 1ull);
        }
    }
    if (next.flag && last_block(&d.rc->ticket[level]) && threadIdx.x == 0) {
        __threadfence();
        int tot = 0;
        for (int g = 0; g < d.G; ++g) tot += *((volatile int *)&d.rc->n[LV_F64][g]);
        set_cond(next, tot > 0);
    }
}

// FP64 level, entries beyond the first cap64 (counted over all groups): a
// block per entry runs its UDF in FP64 from the tuple and decides exactly.
__global__ void __launch_bounds__(256) k_mq_band64(MqDev d, int r, GroupedMlps mlps) {
    extern __shared__ unsigned char smem_raw[];
    double *h = reinterpret_cast<double *>(smem_raw);
    double *g2 = h + mlps.max_width;
    int off[kMqPool + 1];
    off[0] = 0;
    for (int g = 0; g < d.G; ++g) off[g + 1] = off[g] + d.rc->n[LV_F64][g];
    const int lane = lane_id(), warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const float *X = d.hdr->X;
    for (int j = d.cap64 + blockIdx.x; j < off[d.G]; j += gridDim.x) {
        int g = 0;
        while (j >= off[g + 1]) ++g;
        const int e = d.list[LV_F64][(size_t)g * d.cap + (j - off[g])];
        const MlpDev &mlp = mlps.m[g];
        const float *x = X + (size_t)e * d.dim;
        for (int k = threadIdx.x; k < mlp.dims[0]; k += blockDim.x) h[k] = (double)x[k];
        __syncthreads();
        double *cur = h, *nxt = g2;
        for (int l = 0; l < mlp.n_layers; ++l) {
            const int fi = mlp.dims[l], fo = mlp.dims[l + 1];
            const bool last = l + 1 == mlp.n_layers;
            for (int o = warp; o < fo; o += nwarps) {
                const float *wr = mlp.W[l] + (size_t)o * fi;
                double s = 0;
                for (int k = lane; k < fi; k += 32) s += (double)wr[k] * cur[k];
#pragma unroll
                for (int dd = 16; dd > 0; dd >>= 1) s += __shfl_xor_sync(0xffffffffu, s, dd);
                if (lane == 0) {
                    s += (double)mlp.b[l][o];
                    nxt[o] = (!last && s < 0.0) ? 0.0 : s;
                }
            }
            __syncthreads();
            double *tmp = cur;
            cur = nxt;
            nxt = tmp;
        }
        if (threadIdx.x == 0) {
            const int q = d.qid[e];
            const int slot = slot_of(d, e, q, r);
            const bool pass = cur[0] > d.thr[rq(d, q) * kMqSlots + slot];
            d.ok[e] = (unsigned char)pass;
            StatRow *row = d.rows + q * kMqSlots + slot;
            if (pass) {
                d.label[e] |= (unsigned char)(1u << slot);
                atomicAdd(ctr(row, F_PASS), 1ull);
            }
            atomicAdd(ctr(row, F_R64), 1ull);
        }
        __syncthreads();
    }
}

// Next alive list: tuples that passed (or whose query is in a warmup batch)
// and have a slot left.  Clears the round's queue and band counters.
__global__ void __launch_bounds__(256) k_mq_survivors(MqDev d, int r, Cond next_round) {
    const int cur = r & 1;
    const int n = d.rc->alive[cur];
    // every level of this round is done: clear the level lists for the next round
    if (blockIdx.x == 0 && threadIdx.x < LV_N * kMqPool) (&d.rc->n[0][0])[threadIdx.x] = 0;
    for (int m0 = blockIdx.x * blockDim.x; m0 < n; m0 += gridDim.x * blockDim.x) {
        const int m = m0 + threadIdx.x;
        bool keep = false;
        int e = 0;
        if (m < n) {
            e = d.alive[cur][m];
            const int q = d.qid[e];
            keep = (d.ok[e] || d.evall[q]) && r + 1 < d.np[rq(d, q)];
        }
        const int pos = warp_append(keep ? &d.rc->alive[cur ^ 1] : nullptr, keep);
        if (keep) d.alive[cur ^ 1][pos] = e;
    }
    if (next_round.flag && last_block(&d.rc->ticket[LV_N]) && threadIdx.x == 0) {
        __threadfence();
        set_cond(next_round, *((volatile int *)&d.rc->alive[cur ^ 1]) > 0);
    }
}


// Result bitmap (bit e: every slot of e's query passed) and passes per query.
__global__ void __launch_bounds__(256) k_mq_result(MqDev d, unsigned int *bitmap) {
    const int n = min(d.off[d.Q], d.cap);
    const int words = (n + 31) / 32;
    for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < words; w += gridDim.x * blockDim.x) {
        unsigned int bits = 0;
        for (int j = 0; j < 32; ++j) {
            const int e = w * 32 + j;
            if (e >= n) break;
            const int q = d.qid[e];
            const unsigned full = (1u << d.np[rq(d, q)]) - 1u;
            if (((unsigned)d.label[e] & full) == full) {
                bits |= 1u << j;
                atomicAdd(reinterpret_cast<unsigned long long *>(&d.npass[q]), 1ull);
            }
        }
        bitmap[w] = bits;
    }
}

// Statistics of the step into each query's history, and the step's
// per-query report into the result slot.
__global__ void k_mq_commit(MqDev d, MqHist h, StatRow *res_rows, unsigned char *res_order, unsigned char *res_evall,
                            long long *res_bidx, long long *res_npass, int *res_total, int *res_gates) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *res_total = d.off[d.Q];
    if (i < kMqGates) res_gates[i] = d.gates[i];
    if (i >= d.Q * kMqSlots) return;
    const int q = i / kMqSlots, slot = i % kMqSlots;
    const long long b = d.bidx[q];
    const StatRow row = d.rows[i];
    res_rows[i] = row;
    res_order[i] = d.order[i];
    if (slot == 0) {
        res_evall[q] = d.evall[q];
        res_bidx[q] = b;
        res_npass[q] = d.npass[q];
    }
    if (b < 0) return;
    const int qq = rq(d, q);
    h.ring[((size_t)qq * h.R + (size_t)(b % h.R)) * kMqSlots + slot] = row;
    if (b < h.warmup) h.warm[((size_t)qq * h.warmup + b) * kMqSlots + slot] = row;
    if (slot == 0) atomicMax(reinterpret_cast<unsigned long long *>(&h.bdone[qq]), (unsigned long long)(b + 1));
}

__global__ void __launch_bounds__(256) k_mq_tuple_order(MqDev d, const float *logits, int ldz, const int *ready) {
    const int n = min(d.off[d.Q], d.cap);
    const bool use_proxy = logits && ready && *ready;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int q = d.qid[e];
        const int qq = rq(d, q);
        const int P = d.np[qq];
        unsigned char *o = d.order_t + (size_t)e * kMqSlots;
        if (d.evall[q] || !use_proxy) {
            for (int k = 0; k < kMqSlots; ++k) o[k] = d.evall[q] ? (unsigned char)k : d.order[q * kMqSlots + k];
            continue;
        }
        float key[kMqSlots];
        for (int i = 0; i < P; ++i) {
            const float z = fminf(fmaxf(logits[(size_t)e * ldz + i], -30.f), 30.f);
            key[i] = (float)d.cost[qq * kMqSlots + i] * (1.f + expf(z));
        }
        for (int i = 0; i < P; ++i) {
            int pos = 0;
            for (int j = 0; j < P; ++j) pos += (key[j] < key[i] || (key[j] == key[i] && j < i)) ? 1 : 0;
            o[pos] = (unsigned char)i;
        }
        for (int k = P; k < kMqSlots; ++k) o[k] = (unsigned char)k;
    }
}

// Learned sessions, proxy output layer from the BF16 hidden activations of
// the tensor-core first layer: Z[e][i] = b2[i] + sum_h W2[i][h] Hb[e][h] for
// e < *count, a thread per row (H % 8 == 0, P <= 8; W2 staged in shared memory).
__global__ void __launch_bounds__(256) k_mq_proxy_out(const int *count, const __nv_bfloat16 *Hb, int H,
                                                      const float *W2, const float *b2, int P, float *Z, int ldz) {
    extern __shared__ float w2s[];
    for (int i = threadIdx.x; i < P * H; i += blockDim.x) w2s[i] = W2[i];
    __syncthreads();
    const int n = *count;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        float acc[kMqSlots];
#pragma unroll
        for (int i = 0; i < kMqSlots; ++i) acc[i] = i < P ? b2[i] : 0.f;
        const uint4 *row = reinterpret_cast<const uint4 *>(Hb + (size_t)e * H);
        for (int c = 0; c < H / 8; ++c) {
            const uint4 v = row[c];
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float h0 = __uint_as_float(w[j] << 16), h1 = __uint_as_float(w[j] & 0xFFFF0000u);
                const int h = c * 8 + 2 * j;
#pragma unroll
                for (int i = 0; i < kMqSlots; ++i)
                    if (i < P) acc[i] = fmaf(w2s[i * H + h + 1], h1, fmaf(w2s[i * H + h], h0, acc[i]));
            }
        }
        for (int i = 0; i < P; ++i) Z[(size_t)e * ldz + i] = acc[i];
    }
}

// FP64 scores of one MLP on n rows (calibration).
__global__ void __launch_bounds__(256) k_mq_scores_f64(MlpDev mlp, int max_width, const float *X, int ldx, int n,
                                                       double *out) {
    extern __shared__ unsigned char smem_raw[];
    double *h = reinterpret_cast<double *>(smem_raw);
    double *g2 = h + max_width;
    const int lane = lane_id(), warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int j = blockIdx.x; j < n; j += gridDim.x) {
        const float *x = X + (size_t)j * ldx;
        for (int k = threadIdx.x; k < mlp.dims[0]; k += blockDim.x) h[k] = (double)x[k];
        __syncthreads();
        double *cur = h, *nxt = g2;
        for (int l = 0; l < mlp.n_layers; ++l) {
            const int fi = mlp.dims[l], fo = mlp.dims[l + 1];
            const bool last = l + 1 == mlp.n_layers;
            for (int o = warp; o < fo; o += nwarps) {
                const float *wr = mlp.W[l] + (size_t)o * fi;
                double s = 0;
                for (int k = lane; k < fi; k += 32) s += (double)wr[k] * cur[k];
#pragma unroll
                for (int dd = 16; dd > 0; dd >>= 1) s += __shfl_xor_sync(0xffffffffu, s, dd);
                if (lane == 0) {
                    s += (double)mlp.b[l][o];
                    nxt[o] = (!last && s < 0.0) ? 0.0 : s;
                }
            }
            __syncthreads();
            double *tmp = cur;
            cur = nxt;
            nxt = tmp;
        }
        if (threadIdx.x == 0) out[j] = cur[0];
        __syncthreads();
    }
}

}  // namespace

void mq_launch_init(const MqDev &d, cudaStream_t st, int sms, Cond round0) {
    k_mq_init<<<grid_for(d.cap, 256, sms, 4), 256, 0, st>>>(d, round0);
}

void mq_launch_router(const MqDev &d, const MqHist &h, cudaStream_t st) {
    k_mq_router<<<(d.Q * 32 + 255) / 256, 256, 0, st>>>(d, h);
}

void mq_launch_partition(const MqDev &d, int r, cudaStream_t st, int sms) {
    k_mq_partition<<<grid_for(d.cap, 256, sms, 2), 256, 0, st>>>(d, r);
}

void mq_launch_layers_f32(const MqLayers &L, cudaStream_t st, int sms) {
    k_mq_layer_f32<<<sms * 4, 256, 0, st>>>(L);
}

void mq_launch_dots_f32(const MqLayers &L, float *score, int sstride, cudaStream_t st, int sms) {
    k_mq_dot_f32<<<sms * 8, 256, 0, st>>>(L, score, sstride);
}

void mq_launch_classify(const MqDev &d, int r, int in, int out, cudaStream_t st, int sms, Cond next, int next_min,
                        const TcHeads *heads, const float *partials, int pstride) {
    TcHeads h{};
    if (heads) h = *heads;
    k_mq_classify<<<grid_for(d.cap, 256, sms, 2), 256, 0, st>>>(d, r, in, out, next, next_min, h,
                                                                partials, pstride);
}

void mq_launch_band32(const MqDev &d, int r, const GroupedMlps &mlps, int max_hidden, float *act0, float *act1,
                      int ld, cudaStream_t st, int sms, Cond next) {
    for (int depth = 0; depth < max_hidden; ++depth)
        k_mq_band_layer<float><<<sms * 4, 32 * kBandWarps, 0, st>>>(d, mlps, LV_F32, depth, act0, act1, ld, d.cap);
    k_mq_band_final<float><<<sms * 2, 256, 0, st>>>(d, mlps, LV_F32, r, act0, act1, ld, d.cap, next);
}

void mq_launch_band64(const MqDev &d, int r, const GroupedMlps &mlps, int max_hidden, cudaStream_t st, int sms) {
    for (int depth = 0; depth < max_hidden; ++depth)
        k_mq_band_layer_wpn<double><<<sms * 8, 256, 0, st>>>(d, mlps, LV_F64, depth, d.act64[0], d.act64[1], d.ld64,
                                                             d.cap64);
    k_mq_band_final<double><<<sms * 2, 256, 0, st>>>(d, mlps, LV_F64, r, d.act64[0], d.act64[1], d.ld64, d.cap64,
                                                     Cond());
    const size_t smem = sizeof(double) * 2 * (size_t)mlps.max_width;
    k_mq_band64<<<sms, 256, smem, st>>>(d, r, mlps);
}

void mq_launch_survivors(const MqDev &d, int r, cudaStream_t st, int sms, Cond next_round) {
    k_mq_survivors<<<grid_for(d.cap, 256, sms, 2), 256, 0, st>>>(d, r, next_round);
}

void mq_launch_result(const MqDev &d, unsigned int *bitmap, cudaStream_t st, int sms) {
    k_mq_result<<<grid_for((d.cap + 31) / 32, 256, sms, 4), 256, 0, st>>>(d, bitmap);
}

void mq_launch_commit(const MqDev &d, const MqHist &h, StatRow *res_rows, unsigned char *res_order,
                      unsigned char *res_evall, long long *res_bidx, long long *res_npass, int *res_total,
                      int *res_gates, cudaStream_t st) {
    const int n = d.Q * kMqSlots > kMqGates ? d.Q * kMqSlots : kMqGates;
    k_mq_commit<<<(n + 255) / 256, 256, 0, st>>>(d, h, res_rows, res_order, res_evall, res_bidx, res_npass, res_total,
                                                 res_gates);
}

void mq_launch_tuple_order(const MqDev &d, const float *logits, int ldz, const int *ready, cudaStream_t st, int sms) {
    k_mq_tuple_order<<<grid_for(d.cap, 256, sms, 4), 256, 0, st>>>(d, logits, ldz, ready);
}

void mq_launch_proxy_out(const int *count, const __nv_bfloat16 *Hb, int H, const float *W2, const float *b2, int P,
                         float *Z, int ldz, int max_rows, cudaStream_t st, int sms) {
    k_mq_proxy_out<<<grid_for(max_rows, 256, sms, 2), 256, sizeof(float) * (size_t)P * H, st>>>(count, Hb, H, W2, b2,
                                                                                                P, Z, ldz);
}

cudaError_t mq_band_smem_setup(int max_width) {
    const int smem = (int)(sizeof(double) * 2 * (size_t)max_width);
    cudaError_t e = cudaFuncSetAttribute(k_mq_band64, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_mq_scores_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

void mq_launch_scores_f64(const MlpDev &mlp, int max_width, const float *X, int ldx, int n, double *out,
                          cudaStream_t st, int sms) {
    const size_t smem = sizeof(double) * 2 * (size_t)max_width;
    k_mq_scores_f64<<<grid_for(n, 1, sms, 4), 256, smem, st>>>(mlp, max_width, X, ldx, n, out);
}

}  // namespace hydro
