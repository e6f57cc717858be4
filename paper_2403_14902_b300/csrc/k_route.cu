// Routing-side kernels: alive lists, threshold test with recheck bands,
// order-preserving compaction (eager dropping of failing tuples, Sec. 3.3),
// per-batch statistics (Sec. 3.3 "Metadata for Data Routing"), the pass
// bitmap, and the rank router (Sec. 4.1 "Cost-Driven Routing Policy").
//
// Alive lists hold tuple indices within the batch (int32, ascending).  Every
// kernel reads its element count from device memory, so a batch's whole
// stage sequence is enqueued without a host round trip.
#include "common.cuh"
#include "internal.h"

namespace hydro {

constexpr int kScanThreads = 1024;
// Chunks of kScanThreads entries whose loads a thread issues before the first
// of their scans, so a batch of up to 4,096 entries waits for its global loads
// once instead of once per chunk.
constexpr int kScanChunks = 4;

__global__ void k_init_alive(int *alive, int *count, int n, unsigned char *acc) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        alive[i] = i;
        if (acc) acc[i] = 1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *count = n;
}

// Threshold test of the working-precision scores of one stage.  Position m
// (0 <= m < *count_in) holds tuple alive_in[m] and score scores[m].  A score
// within `margin` of t goes to the recheck band (ordered); otherwise
// pass[m] = score > t.
template <typename S>
__global__ void __launch_bounds__(kScanThreads)
k_classify(const int *count_in, const int *alive_in, const S *scores, double t, double margin,
           unsigned char *pass, int *band_m, int *band_tuple, int *band_count, int band_cap,
           unsigned int *err) {
    const int n = *count_in;
    int base = 0;
    for (int m0 = 0; m0 < n; m0 += kScanChunks * kScanThreads) {
        S sv[kScanChunks];
#pragma unroll
        for (int k = 0; k < kScanChunks; ++k) {
            const int m = m0 + k * kScanThreads + threadIdx.x;
            sv[k] = m < n ? scores[m] : S(0);
        }
#pragma unroll
        for (int k = 0; k < kScanChunks; ++k) {
            const int m = m0 + k * kScanThreads + threadIdx.x;
            int inband = 0;
            if (m < n) {
                const double s = (double)sv[k];
                inband = fabs(s - t) <= margin;
                pass[m] = (!inband && s > t) ? 1 : 0;
            }
            int total;
            const int pos = base + block_scan_flags_1024(inband, &total);
            if (inband) {
                if (pos < band_cap) {
                    band_m[pos] = m;
                    band_tuple[pos] = alive_in[m];
                } else {
                    atomicOr(err, ERR_BAND_OVERFLOW);
                }
            }
            base += total;
        }
    }
    if (threadIdx.x == 0) *band_count = base < band_cap ? base : band_cap;
}

// Decide the band entries from their recheck scores.  If margin_next >= 0,
// entries still within margin_next of t go on to the next band (next
// precision); otherwise they are decided here.
template <typename S>
__global__ void __launch_bounds__(kScanThreads)
k_recheck_classify(const int *band_count_in, const int *band_m_in, const int *band_tuple_in,
                   const S *scores_r, double t, double margin_next, unsigned char *pass,
                   int *next_m, int *next_tuple, int *next_count, int next_cap, unsigned int *err) {
    const int n = *band_count_in;
    int base = 0;
    for (int j0 = 0; j0 < n; j0 += kScanThreads) {
        const int j = j0 + threadIdx.x;
        int fwd = 0;
        if (j < n) {
            const double s = (double)scores_r[j];
            fwd = margin_next >= 0.0 && fabs(s - t) <= margin_next;
            if (!fwd) pass[band_m_in[j]] = s > t ? 1 : 0;
        }
        int total;
        const int pos = base + block_scan_flags_1024(fwd, &total);
        if (fwd) {
            if (pos < next_cap) {
                next_m[pos] = band_m_in[j];
                next_tuple[pos] = band_tuple_in[j];
            } else {
                atomicOr(err, ERR_BAND_OVERFLOW);
            }
        }
        base += total;
    }
    if (threadIdx.x == 0 && next_count) *next_count = base < next_cap ? base : next_cap;
}

__device__ __forceinline__ long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return (long long)t;
}

__global__ void k_stage_start(StatRow *row) { row->ns = global_ns(); }

// Close a stage: record statistics and either drop the failing tuples
// (short-circuit) or AND the stage's verdict into the all-evaluate
// accumulator.  row/rrow: this predicate's statistics in the ring and in the
// batch's result block; warm: the warmup copy (nullable).
__global__ void __launch_bounds__(kScanThreads)
k_compact(const int *count_in, const int *alive_in, const unsigned char *pass, int *alive_out,
          int *count_out, unsigned char *acc, const int *bandt_count, const int *band32_count,
          const int *band64_count, const int *miss_count, StatRow *row, StatRow *rrow, StatRow *warm,
          int measure) {
    const int n = *count_in;
    int base = 0;
    for (int m0 = 0; m0 < n; m0 += kScanChunks * kScanThreads) {
        int pv[kScanChunks], tv[kScanChunks];
#pragma unroll
        for (int k = 0; k < kScanChunks; ++k) {
            const int m = m0 + k * kScanThreads + threadIdx.x;
            pv[k] = m < n ? (int)pass[m] : 0;
            tv[k] = m < n ? alive_in[m] : 0;
        }
#pragma unroll
        for (int k = 0; k < kScanChunks; ++k) {
            const int m = m0 + k * kScanThreads + threadIdx.x;
            const int p = pv[k];
            int total;
            const int pos = base + block_scan_flags_1024(p, &total);
            if (acc) {
                if (m < n && !p) acc[tv[k]] = 0;
            } else if (p) {
                alive_out[pos] = tv[k];
            }
            base += total;
        }
    }
    if (threadIdx.x == 0) {
        if (!acc) *count_out = base;
        StatRow r;
        r.evaluated = n;
        r.passed = base;
        r.recheck_tf32 = bandt_count ? *bandt_count : 0;
        r.recheck32 = band32_count ? *band32_count : 0;
        r.recheck64 = band64_count ? *band64_count : 0;
        r.hits = miss_count ? (long long)n - *miss_count : 0;
        // measured: the stage's start stamp (k_stage_start) to now
        r.ns = measure ? global_ns() - row->ns : 0;
        *row = r;
        *rrow = r;
        if (warm) *warm = r;
    }
}

// All-evaluate close: the final alive list is the accumulator's 1 entries.
__global__ void __launch_bounds__(kScanThreads)
k_acc_to_alive(const unsigned char *acc, int n, int *alive_out, int *count_out) {
    int base = 0;
    for (int m0 = 0; m0 < n; m0 += kScanThreads) {
        const int m = m0 + threadIdx.x;
        const int p = (m < n) ? (int)acc[m] : 0;
        int total;
        const int pos = base + block_scan_flags_1024(p, &total);
        if (p) alive_out[pos] = m;
        base += total;
    }
    if (threadIdx.x == 0) *count_out = base;
}

// Pass bitmap (LSB first) from the final alive list, plus n_pass.
__global__ void __launch_bounds__(kScanThreads)
k_result(const int *count, const int *alive, int n, unsigned int *bitmap, long long *n_pass) {
    const int words = (n + 31) >> 5;
    for (int w = threadIdx.x; w < words; w += blockDim.x) bitmap[w] = 0u;
    __syncthreads();
    const int c = *count;
    for (int m = threadIdx.x; m < c; m += blockDim.x) {
        const int j = alive[m];
        atomicOr(&bitmap[j >> 5], 1u << (j & 31));
    }
    if (threadIdx.x == 0) *n_pass = c;
}

// Router: one warp, lane i scores predicate i.  The order is built greedily:
// each position takes the remaining predicate that no other remaining one
// goes before (exact integer comparisons; ties to the lower id).  A head on a
// shared upstream UDF pays the upstream's cost for the batch's uncached ids
// only while no head of its group is placed yet: a later head of the group
// finds every tuple that reaches it cached by the earlier one (without groups
// the greedy order is the plain ascending order of the keys).  Statistics are
// the sums over visible batches [lo, last] of the ring; a predicate with no
// evaluations there falls back to the warmup batches' statistics.
__global__ void k_router(const StatRow *ring, int ring_len, const StatRow *warm, int n_warm_visible,
                         long long lo, long long last, int P, int policy, RouterCosts costs, const int *vmiss,
                         int *order_out) {
    const int i = threadIdx.x;
    long long E = 0, Pp = 0, NS = 0;
    // per-batch cost scaled by the batch size: c*n, plus misses * upstream cost while the
    // group's upstream is not yet computed by an earlier head
    unsigned long long base = 0, extra = 0;
    const int grp = i < P ? costs.group[i] : -1;
    if (i < P) {
        const long long nn = costs.n > 0 ? costs.n : 1;
        base = (unsigned long long)costs.c[i] * (unsigned long long)nn;
        if (grp >= 0 && vmiss && costs.n > 0)
            extra = (unsigned long long)vmiss[grp] * (unsigned long long)costs.cemb[grp];
    }
    if (i < P) {
        for (long long b = lo; b <= last; ++b) {
            const StatRow r = ring[(b % ring_len) * kMaxPred + i];
            E += r.evaluated;
            Pp += r.passed;
            NS += r.ns;
        }
        if (E == 0) {
            for (int w = 0; w < n_warm_visible; ++w) {
                E += warm[w * kMaxPred + i].evaluated;
                Pp += warm[w * kMaxPred + i].passed;
                NS += warm[w * kMaxPred + i].ns;
            }
        }
    }
    // measured cost per tuple (ns); a predicate without evaluations costs 0
    const double cm = costs.measured && E > 0 ? (double)NS / (double)E : 0.0;
    unsigned placed = 0, done_groups = 0;
    for (int k = 0; k < P; ++k) {
        const unsigned long long cost =
            base + ((grp >= 0 && !((done_groups >> grp) & 1u)) ? extra : 0ull);
        const bool mine = i < P && !((placed >> i) & 1u);
        bool first = mine;   // no other remaining predicate goes before i
        for (int j = 0; j < P; ++j) {
            const long long Ej = __shfl_sync(0xffffffffu, E, j);
            const long long Pj = __shfl_sync(0xffffffffu, Pp, j);
            const unsigned long long cj = __shfl_sync(0xffffffffu, cost, j);
            const double cmj = __shfl_sync(0xffffffffu, cm, j);
            if (!mine || j == i || ((placed >> j) & 1u)) continue;
            const unsigned long long ci = cost;
            bool before;   // does j go before i?
            if (costs.measured && policy == 0) {
                // measured rank c/(1-s) in double (the costs are measurements, not exact integers)
                const double rj = cmj * (double)(Ej + 2) / (double)(Ej - Pj + 1);
                const double ri = cm * (double)(E + 2) / (double)(E - Pp + 1);
                before = rj < ri || (rj == ri && j < i);
            } else if (costs.measured && policy == 1) {
                before = cmj < cm || (cmj == cm && j < i);
            } else if (policy == 0) {
                // rank c/(1-s), s = (p+1)/(e+2): c(e+2)/(e-p+1)
                const unsigned __int128 lhs = (unsigned __int128)cj * (unsigned long long)(Ej + 2) *
                                              (unsigned long long)(E - Pp + 1);
                const unsigned __int128 rhs = (unsigned __int128)ci * (unsigned long long)(E + 2) *
                                              (unsigned long long)(Ej - Pj + 1);
                before = lhs < rhs || (lhs == rhs && j < i);
            } else if (policy == 1) {
                before = cj < ci || (cj == ci && j < i);
            } else {
                // selectivity (p+1)/(e+2)
                const unsigned __int128 lhs = (unsigned __int128)(unsigned long long)(Pj + 1) * (unsigned long long)(E + 2);
                const unsigned __int128 rhs = (unsigned __int128)(unsigned long long)(Pp + 1) * (unsigned long long)(Ej + 2);
                before = lhs < rhs || (lhs == rhs && j < i);
            }
            if (before) first = false;
        }
        const unsigned m = __ballot_sync(0xffffffffu, first);
        const int pick = m ? __ffs(m) - 1 : 0;   // exactly one lane: the order is total
        if (i == 0) order_out[k] = pick;
        placed |= 1u << pick;
        const int gp = __shfl_sync(0xffffffffu, grp, pick);
        if (gp >= 0) done_groups |= 1u << gp;
    }
}

// ------------------------------------------------------------ band staging and gates
// Recheck band staging: the band's tuples (rows or frames of the batch) are
// copied into a fixed per-lane buffer, entry j to slot j, and the band's
// tuple index becomes j.  The recheck levels then read only buffers whose
// addresses never change, so they can replay from a captured graph while
// every batch brings its own tuple pointer.  One CTA per entry, 16-byte
// copies when the batch and the tuple size allow it.
__global__ void __launch_bounds__(256)
k_band_stage(const int *band_count, int *band_tuple, const unsigned char *tuples, long long tuple_bytes,
             unsigned char *staging) {
    const int n = *band_count;
    const bool v16 = ((reinterpret_cast<uintptr_t>(tuples) | (uintptr_t)tuple_bytes) & 15u) == 0;
    for (int j = blockIdx.x; j < n; j += gridDim.x) {
        const long long t = band_tuple[j];
        const unsigned char *src = tuples + t * tuple_bytes;
        unsigned char *dst = staging + (long long)j * tuple_bytes;
        if (v16) {
            const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
            uint4 *d4 = reinterpret_cast<uint4 *>(dst);
            for (long long k = threadIdx.x; k < tuple_bytes / 16; k += blockDim.x) d4[k] = s4[k];
        } else {
            for (long long k = threadIdx.x; k < tuple_bytes; k += blockDim.x) dst[k] = src[k];
        }
        __syncthreads();   // every thread has read band_tuple[j] before it is rewritten
        if (threadIdx.x == 0) band_tuple[j] = j;
    }
}

// Gate of a conditional recheck level inside a captured graph: the level's
// body runs iff its band is not empty.  An empty band zeroes the band counts
// of the later levels (their bodies will not run to write them), and a body
// that runs adds its kernel count to the launch counter.
__global__ void k_gate(const int *count, unsigned long long handle, int *zero0, int *zero1,
                       unsigned long long *launch_ctr, const int *body_kernels) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const bool on = *count > 0;
    cudaGraphSetConditional((cudaGraphConditionalHandle)handle, on ? 1u : 0u);
    if (!on) {
        if (zero0) *zero0 = 0;
        if (zero1) *zero1 = 0;
    } else if (launch_ctr && body_kernels) {
        atomicAdd(launch_ctr, (unsigned long long)*body_kernels);
    }
}


// ------------------------------------------------------------ device-dispatched batches
// A routed batch can replay from a graph captured once per stream lane: the
// batch's tuples are first copied into the lane's buffer and its size into
// *n_dev, the router writes the lane's order, and the graph's first kernel
// turns the order into the values of one SWITCH node per position.

__global__ void k_set_int(int *dst, int v) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *dst = v;
}

__global__ void k_init_alive_dev(int *alive, int *count, const int *n_dev) {
    const int n = *n_dev;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) alive[i] = i;
    if (blockIdx.x == 0 && threadIdx.x == 0) *count = n;
}

// Position k's SWITCH selects the body of predicate order[k]; the bodies'
// kernel counts go to the launch counter; the order goes to the result block.
__global__ void k_dispatch(const int *order, SwitchHandles h, int P, const int *body_n, unsigned long long *ctr,
                           int *order_out) {
    const int k = threadIdx.x;
    if (blockIdx.x != 0 || k >= P) return;
    const int i = order[k];
    const int v = (i >= 0 && i < P) ? i : 0;
    cudaGraphSetConditional((cudaGraphConditionalHandle)h.h[k], (unsigned)v);
    if (order_out) order_out[k] = i;
    if (ctr && body_n) atomicAdd(ctr, (unsigned long long)body_n[k * P + v]);
}

__global__ void __launch_bounds__(kScanThreads)
k_result_dev(const int *count, const int *alive, const int *n_dev, unsigned int *bitmap, long long *n_pass) {
    const int n = *n_dev;
    const int words = (n + 31) >> 5;
    for (int w = threadIdx.x; w < words; w += blockDim.x) bitmap[w] = 0u;
    __syncthreads();
    const int c = *count;
    for (int m = threadIdx.x; m < c; m += blockDim.x) {
        const int j = alive[m];
        atomicOr(&bitmap[j >> 5], 1u << (j & 31));
    }
    if (threadIdx.x == 0) *n_pass = c;
}

// The batch's statistics rows into its slot of the ring (the router's source).
__global__ void k_commit_rows(const StatRow *src, StatRow *dst, int P) {
    const int i = threadIdx.x;
    if (blockIdx.x == 0 && i < P) dst[i] = src[i];
}

// ------------------------------------------------------------ launchers

void launch_init_alive(int *alive, int *count, int n, unsigned char *acc, cudaStream_t st) {
    const int blocks = n > 0 ? (n + 255) / 256 : 1;
    k_init_alive<<<blocks, 256, 0, st>>>(alive, count, n, acc);
}

void launch_classify_f32(const int *count_in, const int *alive_in, const float *scores, double t,
                         double margin, unsigned char *pass, int *band_m, int *band_tuple,
                         int *band_count, int band_cap, unsigned int *err, cudaStream_t st) {
    k_classify<float><<<1, kScanThreads, 0, st>>>(count_in, alive_in, scores, t, margin, pass, band_m,
                                                  band_tuple, band_count, band_cap, err);
}

void launch_recheck_classify_f32(const int *band_count_in, const int *band_m_in, const int *band_tuple_in,
                                 const float *scores_r, double t, double margin_next,
                                 unsigned char *pass, int *next_m, int *next_tuple, int *next_count,
                                 int next_cap, unsigned int *err, cudaStream_t st) {
    k_recheck_classify<float><<<1, kScanThreads, 0, st>>>(band_count_in, band_m_in, band_tuple_in,
                                                          scores_r, t, margin_next, pass, next_m,
                                                          next_tuple, next_count, next_cap, err);
}

void launch_recheck_classify_f64(const int *band_count_in, const int *band_m_in, const int *band_tuple_in,
                                 const double *scores_r, double t, unsigned char *pass,
                                 unsigned int *err, cudaStream_t st) {
    k_recheck_classify<double><<<1, kScanThreads, 0, st>>>(band_count_in, band_m_in, band_tuple_in,
                                                           scores_r, t, -1.0, pass, nullptr, nullptr,
                                                           nullptr, 0, err);
}

void launch_compact(const int *count_in, const int *alive_in, const unsigned char *pass, int *alive_out,
                    int *count_out, unsigned char *acc, const int *bandt_count, const int *band32_count,
                    const int *band64_count, const int *miss_count, StatRow *row, StatRow *rrow, StatRow *warm,
                    cudaStream_t st, int measure) {
    k_compact<<<1, kScanThreads, 0, st>>>(count_in, alive_in, pass, alive_out, count_out, acc, bandt_count,
                                          band32_count, band64_count, miss_count, row, rrow, warm, measure);
}

void launch_stage_start(StatRow *row, cudaStream_t st) { k_stage_start<<<1, 1, 0, st>>>(row); }

void launch_band_stage(const int *band_count, int *band_tuple, const void *tuples, long long tuple_bytes,
                       void *staging, int max_entries, int sms, cudaStream_t st) {
    const int grid = max_entries < 4 * sms ? (max_entries > 0 ? max_entries : 1) : 4 * sms;
    k_band_stage<<<grid, 256, 0, st>>>(band_count, band_tuple, static_cast<const unsigned char *>(tuples),
                                       tuple_bytes, static_cast<unsigned char *>(staging));
}

void launch_gate(const int *count, unsigned long long handle, int *zero0, int *zero1, unsigned long long *launch_ctr,
                 const int *body_kernels, cudaStream_t st) {
    k_gate<<<1, 32, 0, st>>>(count, handle, zero0, zero1, launch_ctr, body_kernels);
}

void launch_acc_to_alive(const unsigned char *acc, int n, int *alive_out, int *count_out, cudaStream_t st) {
    k_acc_to_alive<<<1, kScanThreads, 0, st>>>(acc, n, alive_out, count_out);
}

void launch_result(const int *count, const int *alive, int n, unsigned int *bitmap, long long *n_pass,
                   cudaStream_t st) {
    k_result<<<1, kScanThreads, 0, st>>>(count, alive, n, bitmap, n_pass);
}

void launch_set_int(int *dst, int v, cudaStream_t st) { k_set_int<<<1, 32, 0, st>>>(dst, v); }

void launch_init_alive_dev(int *alive, int *count, const int *n_dev, int max_n, cudaStream_t st) {
    const int blocks = max_n > 0 ? (max_n + 255) / 256 : 1;
    k_init_alive_dev<<<blocks < 1024 ? blocks : 1024, 256, 0, st>>>(alive, count, n_dev);
}

void launch_dispatch(const int *order, const SwitchHandles &h, int P, const int *body_n, unsigned long long *ctr,
                     int *order_out, cudaStream_t st) {
    k_dispatch<<<1, 32, 0, st>>>(order, h, P, body_n, ctr, order_out);
}

void launch_result_dev(const int *count, const int *alive, const int *n_dev, unsigned int *bitmap, long long *n_pass,
                       cudaStream_t st) {
    k_result_dev<<<1, kScanThreads, 0, st>>>(count, alive, n_dev, bitmap, n_pass);
}

void launch_commit_rows(const StatRow *src, StatRow *dst, int P, cudaStream_t st) {
    k_commit_rows<<<1, 32, 0, st>>>(src, dst, P);
}

void launch_router(const StatRow *ring, int ring_len, const StatRow *warm, int n_warm_visible,
                   long long lo, long long last, int P, int policy, const RouterCosts &costs, const int *vmiss,
                   int *order_out, cudaStream_t st) {
    k_router<<<1, 32, 0, st>>>(ring, ring_len, warm, n_warm_visible, lo, last, P, policy, costs, vmiss, order_out);
}

}  // namespace hydro
