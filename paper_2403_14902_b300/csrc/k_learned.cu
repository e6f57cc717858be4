// Per-tuple routing by a learned proxy (content-based routing, Sec. 2.2
// "Content-based Routing"): a small MLP predicts every predicate's pass
// probability p_i(x) from the tuple itself; each tuple visits the predicates
// in ascending c_i / (1 - p_i(x)), the rank of Sec. 4.1 with its own
// selectivity estimate.  Execution runs in rounds: in round r every alive
// tuple evaluates the r-th predicate of its own order, so the alive tuples
// split into one queue per predicate; one grouped launch drains all queues
// of a layer depth.  A tuple that fails is dropped at once (Sec. 3.3).
// The proxy is trained online on the outcomes the rounds produce (masked
// binary cross-entropy over the (tuple, predicate) pairs actually
// evaluated).
#include <math.h>

#include "common.cuh"
#include "internal.h"
#include "simt_tile.cuh"

namespace hydro {

constexpr int kLThreads = 1024;

// ------------------------------------------------------------ orders

// Per-tuple order for tuples 0..n-1: ascending c_i * (1 + exp(z_i)) =
// c_i / (1 - sigmoid(z_i)), ties to the lower predicate id.  With logits ==
// nullptr every tuple takes `fallback` (the batch's rank order).
__global__ void k_tuple_order(int n, int P, const float *logits, int ldz, RouterCosts costs, const int *fallback,
                              unsigned char *order) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        unsigned char *o = order + (size_t)t * kMaxPred;
        if (!logits) {
            for (int k = 0; k < P; ++k) o[k] = (unsigned char)fallback[k];
            continue;
        }
        double key[kMaxPred];
        int idx[kMaxPred];
        for (int i = 0; i < P; ++i) {
            const double z = fmin((double)logits[(size_t)t * ldz + i], 60.0);
            key[i] = (double)costs.c[i] * (1.0 + exp(z));
            idx[i] = i;
        }
        for (int a = 1; a < P; ++a) {   // insertion sort, stable: ties keep the lower id first
            const double kv = key[a];
            const int iv = idx[a];
            int b = a - 1;
            while (b >= 0 && key[b] > kv) {
                key[b + 1] = key[b];
                idx[b + 1] = idx[b];
                --b;
            }
            key[b + 1] = kv;
            idx[b + 1] = iv;
        }
        for (int k = 0; k < P; ++k) o[k] = (unsigned char)idx[k];
    }
}

// Round r: split the alive list into one queue per predicate (the r-th entry
// of each tuple's order), each queue in alive-list order.
__global__ void __launch_bounds__(kLThreads)
k_partition(const int *count, const int *alive, const unsigned char *order, int r, int P, int *queues, int qstride,
            int *qcount) {
    const int n = *count;
    int base[kMaxPred];
    for (int p = 0; p < P; ++p) base[p] = 0;
    for (int m0 = 0; m0 < n; m0 += kLThreads) {
        const int m = m0 + threadIdx.x;
        int pred = -1, t = 0;
        if (m < n) {
            t = alive[m];
            pred = order[(size_t)t * kMaxPred + r];
        }
        for (int p = 0; p < P; ++p) {
            int total;
            const int pos = base[p] + block_scan_flags_1024(pred == p, &total);
            if (pred == p) queues[(size_t)p * qstride + pos] = t;
            base[p] += total;
        }
    }
    if (threadIdx.x < P) qcount[threadIdx.x] = base[threadIdx.x];
}

// ------------------------------------------------------------ grouped layers

// All groups' hidden layers of one depth in one launch: tiles are numbered
// group by group and walked grid-stride, so uneven queues share the SMs.
__global__ void __launch_bounds__(256) k_grouped_layer_f32(GroupedLayers g) {
    __shared__ __align__(16) float As[2][16][68];
    __shared__ __align__(16) float Ws[2][16][68];
    int tiles[kMaxPred], start[kMaxPred + 1];
    start[0] = 0;
    for (int i = 0; i < g.n; ++i) {
        const int M = *g.l[i].count;
        tiles[i] = ((M + 63) / 64) * ((g.l[i].N + 63) / 64);
        start[i + 1] = start[i] + tiles[i];
    }
    for (int tile = blockIdx.x; tile < start[g.n]; tile += gridDim.x) {
        int i = 0;
        while (tile >= start[i + 1]) ++i;
        const GroupLayer &L = g.l[i];
        const int local = tile - start[i];
        const int tn = (L.N + 63) / 64;
        mlp_tile_f32(*L.count, (local / tn) * 64, (local % tn) * 64, L.rows, L.X, L.ldx, L.W, L.b, L.Y, L.N, L.K,
                     L.N, L.relu, As, Ws);
    }
}

// Every group's last layer (one output) in one launch: warp per row.
__global__ void __launch_bounds__(256) k_grouped_dot_f32(GroupedLayers g, float *score, int sstride) {
    const int lane = threadIdx.x & 31;
    int start[kMaxPred + 1];
    start[0] = 0;
    for (int i = 0; i < g.n; ++i) start[i + 1] = start[i] + *g.l[i].count;
    for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < start[g.n]; w += (gridDim.x * blockDim.x) >> 5) {
        int i = 0;
        while (w >= start[i + 1]) ++i;
        const GroupLayer &L = g.l[i];
        const int m = w - start[i];
        const float *x = L.X + (size_t)(L.rows ? L.rows[m] : m) * L.ldx;
        float s = 0.f;
        for (int k = lane; k < L.K; k += 32) s = fmaf(x[k], L.W[k], s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) score[(size_t)i * sstride + m] = s + L.bconst;
    }
}

// Decide every queue entry of the round: pass/fail into per-tuple flags
// (ok, label and visited bits), or the FP64 band (entries of all groups, in
// group then queue order).  Statistics are added into the batch's rows.
__global__ void __launch_bounds__(kLThreads)
k_grouped_classify(int P, const int *qcount, const int *queues, int qstride, const float *score, int sstride,
                   RoundTests tests, unsigned char *ok, unsigned char *label, unsigned char *visited, int *band_g,
                   int *band_t, int *band_count, int band_cap, StatRow *row, StatRow *rrow, unsigned int *err) {
    int base = 0;
    for (int p = 0; p < P; ++p) {
        const int n = qcount[p];
        int passed = 0;
        for (int m0 = 0; m0 < n; m0 += kLThreads) {
            const int m = m0 + threadIdx.x;
            int inband = 0, pass = 0;
            if (m < n) {
                const int t = queues[(size_t)p * qstride + m];
                const double s = (double)score[(size_t)p * sstride + m];
                inband = fabs(s - tests.t[p]) <= tests.margin[p];
                pass = !inband && s > tests.t[p];
                ok[t] = (unsigned char)pass;
                visited[t] |= (unsigned char)(1u << p);
                if (pass) label[t] |= (unsigned char)(1u << p);
                if (inband) {
                    // filled by the FP64 recheck
                }
            }
            int tot_b, tot_p;
            const int pos = base + block_scan_flags_1024(inband, &tot_b);
            (void)block_scan_flags_1024(pass, &tot_p);
            if (inband) {
                if (pos < band_cap) {
                    band_g[pos] = p;
                    band_t[pos] = queues[(size_t)p * qstride + m];
                } else {
                    atomicOr(err, ERR_BAND_OVERFLOW);
                }
            }
            base += tot_b;
            passed += tot_p;
        }
        if (threadIdx.x == 0) {
            row[p].evaluated += n;
            row[p].passed += passed;
            rrow[p].evaluated += n;
            rrow[p].passed += passed;
        }
    }
    if (threadIdx.x == 0) *band_count = base < band_cap ? base : band_cap;
}

// FP64 recheck of the round's band: block per entry, the whole MLP of its
// predicate in FP64 from the tuple; the verdict lands in ok/label and the
// statistics (passed, recheck64).
__global__ void __launch_bounds__(256)
k_grouped_band_f64(const int *band_count, const int *band_g, const int *band_t, const float *X, int ldx,
                   GroupedMlps mlps, RoundTests tests, unsigned char *ok, unsigned char *label, StatRow *row,
                   StatRow *rrow) {
    extern __shared__ unsigned char smem_raw[];
    double *h = reinterpret_cast<double *>(smem_raw);
    double *g = h + mlps.max_width;
    const int n = *band_count;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int j = blockIdx.x; j < n; j += gridDim.x) {
        const int p = band_g[j], t = band_t[j];
        const MlpDev &mlp = mlps.m[p];
        const float *x = X + (size_t)t * ldx;
        for (int k = threadIdx.x; k < mlp.dims[0]; k += blockDim.x) h[k] = (double)x[k];
        __syncthreads();
        double *cur = h, *nxt = g;
        for (int l = 0; l < mlp.n_layers; ++l) {
            const int fi = mlp.dims[l], fo = mlp.dims[l + 1];
            const bool last = l + 1 == mlp.n_layers;
            for (int o = warp; o < fo; o += nwarps) {
                const float *wr = mlp.W[l] + (size_t)o * fi;
                double s = 0;
                for (int k = lane; k < fi; k += 32) s += (double)wr[k] * cur[k];
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
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
            const bool pass = cur[0] > tests.t[p];
            ok[t] = (unsigned char)pass;
            if (pass) {
                label[t] |= (unsigned char)(1u << p);
                atomicAdd(reinterpret_cast<unsigned long long *>(&row[p].passed), 1ull);
                atomicAdd(reinterpret_cast<unsigned long long *>(&rrow[p].passed), 1ull);
            }
            atomicAdd(reinterpret_cast<unsigned long long *>(&row[p].recheck64), 1ull);
            atomicAdd(reinterpret_cast<unsigned long long *>(&rrow[p].recheck64), 1ull);
        }
        __syncthreads();
    }
}

// Next round's alive list: this round's tuples that passed, in order.
__global__ void __launch_bounds__(kLThreads)
k_survivors(const int *count_in, const int *alive_in, const unsigned char *ok, int *alive_out, int *count_out) {
    const int n = *count_in;
    int base = 0;
    for (int m0 = 0; m0 < n; m0 += kLThreads) {
        const int m = m0 + threadIdx.x;
        const int p = m < n ? (int)ok[alive_in[m]] : 0;
        int total;
        const int pos = base + block_scan_flags_1024(p, &total);
        if (p) alive_out[pos] = alive_in[m];
        base += total;
    }
    if (threadIdx.x == 0) *count_out = base;
}

__global__ void k_zero_rows(StatRow *row, StatRow *rrow, int P, unsigned char *visited, unsigned char *label, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < P) {
        row[i] = StatRow{};
        rrow[i] = StatRow{};
    }
    for (int t = i; t < n; t += gridDim.x * blockDim.x) {
        visited[t] = 0;
        label[t] = 0;
    }
}

// ------------------------------------------------------------ training

// dZ[m][p] = (sigmoid(z) - y) / count over evaluated pairs, 0 elsewhere
// (masked binary cross-entropy; count = evaluated pairs of the minibatch).
__global__ void k_bce_grad(int M, int P, const float *Z, const unsigned char *label, const unsigned char *mask,
                           const float *inv_pairs, float *dZ) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M * P; i += gridDim.x * blockDim.x) {
        const int m = i / P, p = i % P;
        const bool ev = (mask[m] >> p) & 1;
        const float y = (float)((label[m] >> p) & 1);
        const float s = 1.f / (1.f + expf(-Z[i]));
        dZ[i] = ev ? (s - y) * (*inv_pairs) : 0.f;
    }
}

__global__ void k_inv_pairs(int M, const unsigned char *mask, float *inv_pairs) {
    __shared__ int tot;
    if (threadIdx.x == 0) tot = 0;
    __syncthreads();
    int c = 0;
    for (int m = threadIdx.x; m < M; m += blockDim.x) c += __popc((unsigned)mask[m]);
    atomicAdd(&tot, c);
    __syncthreads();
    if (threadIdx.x == 0) *inv_pairs = tot > 0 ? 1.f / (float)tot : 0.f;
}

// Weight and bias gradients G[a][b] = sum_m A[m][a] * B[m][b] and
// gb[a] = sum_m A[m][a] (A [M x NA], B [M x NB]) in two deterministic steps.
// Step 1, one CTA per 64x64 output tile and chunk of kGChunk rows:
// Gp[c][a][b] and gbp[c][a] over the rows of chunk c (16-row slices staged in
// shared memory, 4x4 outputs per thread).  Step 2 sums the chunks in order.
constexpr int kGChunk = 256;

__global__ void __launch_bounds__(256)
k_grad_outer_part(int M, int NA, int NB, const float *__restrict__ A, const float *__restrict__ B, float *Gp,
                  float *gbp) {
    __shared__ __align__(16) float As[16][64];
    __shared__ __align__(16) float Bs[16][64];
    const int a0 = blockIdx.y * 64, b0 = blockIdx.x * 64, c = blockIdx.z;
    const int m0 = c * kGChunk, m1 = min(M, m0 + kGChunk);
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    float acc[4][4] = {};
    float colsum = 0.f;
    for (int k0 = m0; k0 < m1; k0 += 16) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int idx = t + e * 256, r = idx >> 6, col = idx & 63, m = k0 + r;
            As[r][col] = (m < m1 && a0 + col < NA) ? A[(size_t)m * NA + a0 + col] : 0.f;
            Bs[r][col] = (m < m1 && b0 + col < NB) ? B[(size_t)m * NB + b0 + col] : 0.f;
        }
        __syncthreads();
        if (gbp && blockIdx.x == 0 && t < 64)
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) colsum += As[kk][t];
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            const float4 a = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
            const float4 b = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
    float *G = Gp + (size_t)c * NA * NB;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int a = a0 + ty * 4 + i;
        if (a >= NA) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int b = b0 + tx * 4 + j;
            if (b < NB) G[(size_t)a * NB + b] = acc[i][j];
        }
    }
    if (gbp && blockIdx.x == 0 && t < 64 && a0 + t < NA) gbp[(size_t)c * NA + a0 + t] = colsum;
}

__global__ void k_sum_chunks(int chunks, int n, const float *__restrict__ part, float *out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int c = 0; c < chunks; ++c) s += part[(size_t)c * n + i];
        out[i] = s;
    }
}


// dH[m][j] = (H[m][j] > 0) * sum_p dZ[m][p] * W2[p][j]
__global__ void k_grad_hidden(int M, int P, int Hd, const float *dZ, const float *W2, const float *H, float *dH) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M * Hd; i += gridDim.x * blockDim.x) {
        const int m = i / Hd, j = i % Hd;
        float s = 0.f;
        for (int p = 0; p < P; ++p) s = fmaf(dZ[(size_t)m * P + p], W2[(size_t)p * Hd + j], s);
        dH[i] = H[i] > 0.f ? s : 0.f;
    }
}

// Adam step on n parameters (bias-corrected with step count t).
__global__ void k_adam(int n, float *w, const float *g, float *m1, float *m2, float lr, int t) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        m1[i] = b1 * m1[i] + (1.f - b1) * gi;
        m2[i] = b2 * m2[i] + (1.f - b2) * gi * gi;
        w[i] -= lr * (m1[i] / c1) / (sqrtf(m2[i] / c2) + eps);
    }
}

// ------------------------------------------------------------ launchers

static int lgrid(long long work, int per_block, int sms, int per_sm) {
    long long g = (work + per_block - 1) / per_block;
    if (g > (long long)sms * per_sm) g = (long long)sms * per_sm;
    return g < 1 ? 1 : (int)g;
}

void launch_tuple_order(int n, int P, const float *logits, int ldz, const RouterCosts &costs, const int *fallback,
                        unsigned char *order, int sms, cudaStream_t st) {
    k_tuple_order<<<lgrid(n, 256, sms, 4), 256, 0, st>>>(n, P, logits, ldz, costs, fallback, order);
}

void launch_partition(const int *count, const int *alive, const unsigned char *order, int r, int P, int *queues,
                      int qstride, int *qcount, cudaStream_t st) {
    k_partition<<<1, kLThreads, 0, st>>>(count, alive, order, r, P, queues, qstride, qcount);
}

void launch_grouped_layer_f32(const GroupedLayers &g, int max_tiles, int sms, cudaStream_t st) {
    k_grouped_layer_f32<<<lgrid(max_tiles, 1, sms, 4), 256, 0, st>>>(g);
}

void launch_grouped_dot_f32(const GroupedLayers &g, float *score, int sstride, int max_rows, int sms,
                            cudaStream_t st) {
    k_grouped_dot_f32<<<lgrid((long long)max_rows * 32, 256, sms, 8), 256, 0, st>>>(g, score, sstride);
}

void launch_grouped_classify(int P, const int *qcount, const int *queues, int qstride, const float *score,
                             int sstride, const RoundTests &tests, unsigned char *ok, unsigned char *label,
                             unsigned char *visited, int *band_g, int *band_t, int *band_count, int band_cap,
                             StatRow *row, StatRow *rrow, unsigned int *err, cudaStream_t st) {
    k_grouped_classify<<<1, kLThreads, 0, st>>>(P, qcount, queues, qstride, score, sstride, tests, ok, label, visited,
                                                band_g, band_t, band_count, band_cap, row, rrow, err);
}

void launch_grouped_band_f64(const int *band_count, const int *band_g, const int *band_t, const float *X, int ldx,
                             const GroupedMlps &mlps, const RoundTests &tests, unsigned char *ok,
                             unsigned char *label, StatRow *row, StatRow *rrow, int sms, cudaStream_t st) {
    const size_t smem = sizeof(double) * 2 * (size_t)mlps.max_width;
    k_grouped_band_f64<<<sms * 2, 256, smem, st>>>(band_count, band_g, band_t, X, ldx, mlps, tests, ok, label, row,
                                                     rrow);
}

cudaError_t grouped_band_smem_setup(int max_width) {
    return cudaFuncSetAttribute(k_grouped_band_f64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(double) * 2 * (size_t)max_width));
}

void launch_survivors(const int *count_in, const int *alive_in, const unsigned char *ok, int *alive_out,
                      int *count_out, cudaStream_t st) {
    k_survivors<<<1, kLThreads, 0, st>>>(count_in, alive_in, ok, alive_out, count_out);
}

void launch_zero_rows(StatRow *row, StatRow *rrow, int P, unsigned char *visited, unsigned char *label, int n,
                      cudaStream_t st) {
    k_zero_rows<<<lgrid(n > P ? n : P, 256, 148, 4), 256, 0, st>>>(row, rrow, P, visited, label, n);
}

// acc[t] = 1 iff tuple t passed every predicate (all-evaluate batches).
__global__ void k_full_label_acc(const unsigned char *label, int n, int P, unsigned char *acc) {
    const unsigned full = (1u << P) - 1u;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x)
        acc[t] = ((unsigned)label[t] & full) == full;
}

void launch_full_label_acc(const unsigned char *label, int n, int P, unsigned char *acc, cudaStream_t st) {
    k_full_label_acc<<<lgrid(n, 256, 148, 4), 256, 0, st>>>(label, n, P, acc);
}

void grad_outer(int M, int NA, int NB, const float *A, const float *B, float *G, float *gb, float *part,
                int sms, cudaStream_t st) {
    const int chunks = (M + kGChunk - 1) / kGChunk;
    float *gbp = part + (size_t)chunks * NA * NB;
    k_grad_outer_part<<<dim3((NB + 63) / 64, (NA + 63) / 64, chunks), 256, 0, st>>>(M, NA, NB, A, B, part, gbp);
    k_sum_chunks<<<lgrid((long long)NA * NB, 256, sms, 4), 256, 0, st>>>(chunks, NA * NB, part, G);
    k_sum_chunks<<<1, 256, 0, st>>>(chunks, NA, gbp, gb);
}

void launch_proxy_train_step(const ProxyTrain &pt, cudaStream_t st) {
    const int M = pt.M, P = pt.P, Hd = pt.H, D = pt.D;
    k_inv_pairs<<<1, 256, 0, st>>>(M, pt.mask, pt.inv_pairs);
    k_bce_grad<<<lgrid((long long)M * P, 256, pt.sms, 8), 256, 0, st>>>(M, P, pt.Z, pt.label, pt.mask, pt.inv_pairs,
                                                                       pt.dZ);
    grad_outer(M, P, Hd, pt.dZ, pt.Hact, pt.gW2, pt.gb2, pt.part, pt.sms, st);
    k_grad_hidden<<<lgrid((long long)M * Hd, 256, pt.sms, 8), 256, 0, st>>>(M, P, Hd, pt.dZ, pt.W2, pt.Hact, pt.dH);
    grad_outer(M, Hd, D, pt.dH, pt.X, pt.gW1, pt.gb1, pt.part, pt.sms, st);
    k_adam<<<lgrid(Hd * D, 256, pt.sms, 4), 256, 0, st>>>(Hd * D, pt.W1, pt.gW1, pt.mW1, pt.vW1, pt.lr, pt.t);
    k_adam<<<1, 256, 0, st>>>(Hd, pt.b1, pt.gb1, pt.mb1, pt.vb1, pt.lr, pt.t);
    k_adam<<<lgrid(P * Hd, 256, pt.sms, 4), 256, 0, st>>>(P * Hd, pt.W2, pt.gW2, pt.mW2, pt.vW2, pt.lr, pt.t);
    k_adam<<<1, 32, 0, st>>>(P, pt.b2, pt.gb2, pt.mb2, pt.vb2, pt.lr, pt.t);
}

}  // namespace hydro
