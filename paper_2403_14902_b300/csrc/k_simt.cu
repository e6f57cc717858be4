// SIMT (CUDA-core) UDF kernels: FP32 inference (static FP32 evaluation and
// the FP32 recheck band), FP64 inference (FP64 recheck band, calibration),
// and a BF16-operand SIMT conv used as the tensor-core kernel's comparator.
//
// UDF definitions (Sec. 4.2 "Predicate Implementation" uses off-the-shelf
// models; the workloads here use random-init MLP and CNN UDFs):
//   MLP: h_{l+1} = W_l h_l + b_l, ReLU on hidden layers, 1 output = score.
//   CNN: x/255 -> [conv3x3 pad 1 + bias + ReLU]* -> global average pool ->
//        linear head = score.
//
// Every kernel takes its row/frame count from device memory and walks its
// tiles with a grid-stride loop, so launches need no host knowledge of how
// many tuples survived.
#include "common.cuh"
#include "internal.h"

namespace hydro {

// ---------------------------------------------------------------- MLP FP32

// Y[m][n] = act(sum_k X[row(m)][k] * W[n][k] + b[n]) for m < *count, with
// row(m) = rows[m] when rows != nullptr, and ids[rows[m]] when ids is given
// too (rows of a cache indexed by tuple id).  64x64 output tiles, 16-deep K
// slices, 4x4 outputs per thread.  The K slices are double-buffered in shared
// memory and the next slice's global loads (16 bytes per row when vec4: K and
// ldx multiples of 4) are in flight while the current one is multiplied; the
// multiply-adds of every output run in k order, as with one buffer.
__global__ void __launch_bounds__(256)
k_mlp_layer_f32(const int *count, const int *rows, const float *X, int ldx, const float *W,
                const float *b, float *Y, int K, int N, int relu, const long long *ids, int vec4) {
    __shared__ __align__(16) float As[2][16][64 + 4];
    __shared__ __align__(16) float Ws[2][16][64 + 4];
    const int M = *count;
    const int tiles_m = (M + 63) / 64, tiles_n = (N + 63) / 64;
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    const int lr = t >> 2, lk = (t & 3) * 4;   // loader: row / k offset
    for (int tile = blockIdx.x; tile < tiles_m * tiles_n; tile += gridDim.x) {
        const int m0 = (tile / tiles_n) * 64, n0 = (tile % tiles_n) * 64;
        float acc[4][4] = {};
        const int am = m0 + lr;
        const float *arow = nullptr;
        if (am < M) {
            const long long r = rows ? (ids ? ids[rows[am]] : (long long)rows[am]) : (long long)am;
            arow = X + (size_t)r * ldx;
        }
        const int wn = n0 + lr;
        const float *wrow = wn < N ? W + (size_t)wn * K : nullptr;
        float ra[4], rw[4];
        auto fetch = [&](int k0) {
            const int k = k0 + lk;
            if (vec4) {
                // K % 4 == 0: the four k of this thread are all in range or all out
                const float4 a4 = (arow && k < K) ? *reinterpret_cast<const float4 *>(arow + k) : make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 w4 = (wrow && k < K) ? *reinterpret_cast<const float4 *>(wrow + k) : make_float4(0.f, 0.f, 0.f, 0.f);
                ra[0] = a4.x, ra[1] = a4.y, ra[2] = a4.z, ra[3] = a4.w;
                rw[0] = w4.x, rw[1] = w4.y, rw[2] = w4.z, rw[3] = w4.w;
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    ra[e] = (arow && k + e < K) ? arow[k + e] : 0.f;
                    rw[e] = (wrow && k + e < K) ? wrow[k + e] : 0.f;
                }
            }
        };
        fetch(0);
        int buf = 0;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            As[0][lk + e][lr] = ra[e];
            Ws[0][lk + e][lr] = rw[e];
        }
        __syncthreads();
        for (int k0 = 0; k0 < K; k0 += 16) {
            const bool more = k0 + 16 < K;
            if (more) fetch(k0 + 16);
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) {
                float a[4], w[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = As[buf][kk][ty * 4 + i];
#pragma unroll
                for (int j = 0; j < 4; ++j) w[j] = Ws[buf][kk][tx * 4 + j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], w[j], acc[i][j]);
            }
            if (more) {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    As[buf ^ 1][lk + e][lr] = ra[e];
                    Ws[buf ^ 1][lk + e][lr] = rw[e];
                }
            }
            __syncthreads();
            buf ^= 1;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int m = m0 + ty * 4 + i;
            if (m >= M) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int n = n0 + tx * 4 + j;
                if (n >= N) continue;
                float v = acc[i][j] + b[n];
                if (relu && v < 0.f) v = 0.f;
                Y[(size_t)m * N + n] = v;
            }
        }
    }
}

// Last MLP layer (one output): score[m] = b + sum_k X[row(m)][k] * w[k].
// One warp per row; fixed lane-strided order and a butterfly reduction.
__global__ void __launch_bounds__(256)
k_mlp_dot_f32(const int *count, const int *rows, const float *X, int ldx, const float *w, float bias,
              int K, float *score, const long long *ids) {
    const int M = *count;
    const int lane = threadIdx.x & 31;
    for (int m = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; m < M; m += (gridDim.x * blockDim.x) >> 5) {
        const long long r = rows ? (ids ? ids[rows[m]] : (long long)rows[m]) : (long long)m;
        const float *x = X + (size_t)r * ldx;
        float s = 0.f;
        for (int k = lane; k < K; k += 32) s = fmaf(x[k], w[k], s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) score[m] = s + bias;
    }
}

// Whole MLP on a band list, one block per tuple, activations in shared
// memory, in precision T (float: FP32 recheck; double: FP64 recheck).
template <typename T>
__global__ void __launch_bounds__(256)
k_mlp_band(const int *band_count, const int *band_tuple, const float *X, int ldx, MlpDev mlp, T *score_out) {
    extern __shared__ unsigned char smem_raw[];
    T *h = reinterpret_cast<T *>(smem_raw);
    T *g = h + mlp.max_width;
    const int n = *band_count;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int j = blockIdx.x; j < n; j += gridDim.x) {
        const float *x = X + (size_t)band_tuple[j] * ldx;
        for (int k = threadIdx.x; k < mlp.dims[0]; k += blockDim.x) h[k] = (T)x[k];
        __syncthreads();
        T *cur = h, *nxt = g;
        for (int l = 0; l < mlp.n_layers; ++l) {
            const int fi = mlp.dims[l], fo = mlp.dims[l + 1];
            const float *W = mlp.W[l];
            const float *bb = mlp.b[l];
            const bool last = l + 1 == mlp.n_layers;
            for (int o = warp; o < fo; o += nwarps) {
                const float *wr = W + (size_t)o * fi;
                T s = 0;
                for (int k = lane; k < fi; k += 32) s += (T)wr[k] * cur[k];
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
                if (lane == 0) {
                    s += (T)bb[o];
                    nxt[o] = (!last && s < (T)0) ? (T)0 : s;
                }
            }
            __syncthreads();
            T *tmp = cur; cur = nxt; nxt = tmp;
        }
        if (threadIdx.x == 0) score_out[j] = cur[0];
        __syncthreads();
    }
}

// ---------------------------------------------------------------- CNN

// relu(acc) for COUT channels stored as 16-byte vectors (COUT * sizeof(Tout)
// is a multiple of 16 and o is aligned to it).
template <typename T, typename Tout, int COUT>
__device__ __forceinline__ void store_relu_row(const T (&acc)[COUT], Tout *o) {
    if constexpr (sizeof(Tout) == 2) {
        uint32_t pk[COUT / 2];
#pragma unroll
        for (int j = 0; j < COUT / 2; ++j) {
            const float a = acc[2 * j] > 0 ? (float)acc[2 * j] : 0.f;
            const float b = acc[2 * j + 1] > 0 ? (float)acc[2 * j + 1] : 0.f;
            const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
            pk[j] = *reinterpret_cast<const uint32_t *>(&v);
        }
        uint4 *d = reinterpret_cast<uint4 *>(o);
#pragma unroll
        for (int j = 0; j < COUT / 8; ++j) d[j] = make_uint4(pk[4 * j], pk[4 * j + 1], pk[4 * j + 2], pk[4 * j + 3]);
    } else if constexpr (sizeof(Tout) == 4) {
        float4 *d = reinterpret_cast<float4 *>(o);
#pragma unroll
        for (int j = 0; j < COUT / 4; ++j) {
            float4 v;
            v.x = acc[4 * j] > 0 ? (float)acc[4 * j] : 0.f;
            v.y = acc[4 * j + 1] > 0 ? (float)acc[4 * j + 1] : 0.f;
            v.z = acc[4 * j + 2] > 0 ? (float)acc[4 * j + 2] : 0.f;
            v.w = acc[4 * j + 3] > 0 ? (float)acc[4 * j + 3] : 0.f;
            d[j] = v;
        }
    } else {
        double2 *d = reinterpret_cast<double2 *>(o);
#pragma unroll
        for (int j = 0; j < COUT / 2; ++j) {
            double2 v;
            v.x = acc[2 * j] > 0 ? (double)acc[2 * j] : 0.0;
            v.y = acc[2 * j + 1] > 0 ? (double)acc[2 * j + 1] : 0.0;
            d[j] = v;
        }
    }
}

// relu(acc) for COUT channels in the FP32-accurate split form the tensor-core
// kernel reads: [hi(COUT) | lo(COUT)], hi = the value rounded to TF32, lo =
// the remainder rounded to TF32.
template <int COUT>
__device__ __forceinline__ void store_relu_row_split(const float (&acc)[COUT], __nv_bfloat16 *o) {
    // split-BF16 planes: hi = bf16(value), lo = bf16(value - hi); 8 values per 16-byte store
    static_assert(COUT % 8 == 0, "16-byte stores of 8 BF16 values");
#pragma unroll
    for (int j = 0; j < COUT; j += 8) {
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float v0 = acc[j + 2 * e] > 0.f ? acc[j + 2 * e] : 0.f;
            const float v1 = acc[j + 2 * e + 1] > 0.f ? acc[j + 2 * e + 1] : 0.f;
            const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
            const __nv_bfloat162 l = __floats2bfloat162_rn(v0 - __low2float(h), v1 - __high2float(h));
            hi[e] = *reinterpret_cast<const uint32_t *>(&h);
            lo[e] = *reinterpret_cast<const uint32_t *>(&l);
        }
        *reinterpret_cast<uint4 *>(o + j) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4 *>(o + COUT + j) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
}

template <int COUT>
__device__ __forceinline__ void store_relu_row_split(const float (&acc)[COUT], float *o) {
#pragma unroll
    for (int j = 0; j < COUT; j += 4) {
        float hi[4], lo[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float v = acc[j + e] > 0.f ? acc[j + e] : 0.f;
            hi[e] = tf32_rne(v);
            lo[e] = tf32_rne(v - hi[e]);
        }
        *reinterpret_cast<float4 *>(o + j) = make_float4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<float4 *>(o + COUT + j) = make_float4(lo[0], lo[1], lo[2], lo[3]);
    }
}

// First conv layer straight from the uint8 CHW frames (gathered through
// `list`): out[m][p][co] = relu(b[co] + sum_{ci,ky,kx} W * x/255), NHWC.
// One thread computes PX consecutive pixels of a row for all COUT channels,
// so every weight read from shared memory feeds PX multiply-adds.
template <typename T, typename Tout, int COUT, int PX, bool SPLIT = false>
__global__ void __launch_bounds__(256)
k_conv1_u8(const int *count, const int *list, const unsigned char *frames, int C0, int H, int Wd,
           const float *W, const float *bias, Tout *out) {
    __shared__ T Ws[8 * 9][COUT];   // [ci*9 + ky*3 + kx][co], C0 <= 8
    __shared__ T Bs[COUT];
    const int M = *count;
    // an empty band (the usual case of the recheck levels) leaves before staging the weights;
    // M is the same for every thread, so no thread skips the barrier below alone
    if (M == 0) return;
    for (int i = threadIdx.x; i < C0 * 9 * COUT; i += blockDim.x) {
        const int co = i % COUT, r = i / COUT;   // r = ci*9 + tap
        Ws[r][co] = (T)W[(size_t)co * C0 * 9 + r];
    }
    for (int i = threadIdx.x; i < COUT; i += blockDim.x) Bs[i] = (T)bias[i];
    __syncthreads();
    const int HW = H * Wd;
    const int per_block = 256 * PX;
    const int blocks_per_frame = (HW + per_block - 1) / per_block;
    const T inv255 = (T)1 / (T)255;
    for (int w = blockIdx.x; w < M * blocks_per_frame; w += gridDim.x) {
        const int m = w / blocks_per_frame;
        const int p = (w % blocks_per_frame) * per_block + threadIdx.x * PX;
        if (p >= HW) continue;
        const int y = p / Wd, x0 = p % Wd;   // Wd % PX == 0: the PX pixels share row y
        const unsigned char *f = frames + (size_t)list[m] * C0 * HW;
        T acc[PX][COUT];
#pragma unroll
        for (int i = 0; i < PX; ++i)
#pragma unroll
            for (int co = 0; co < COUT; ++co) acc[i][co] = Bs[co];
        for (int ci = 0; ci < C0; ++ci)
#pragma unroll
            for (int ky = 0; ky < 3; ++ky) {
                const int yy = y + ky - 1;
                if (yy < 0 || yy >= H) continue;
                const unsigned char *row = f + (size_t)ci * HW + (size_t)yy * Wd;
                T v[PX + 2];
#pragma unroll
                for (int j = 0; j < PX + 2; ++j) {
                    const int xx = x0 - 1 + j;
                    v[j] = (xx >= 0 && xx < Wd) ? (T)row[xx] * inv255 : (T)0;
                }
#pragma unroll
                for (int kx = 0; kx < 3; ++kx) {
                    const T *wr = Ws[ci * 9 + ky * 3 + kx];
#pragma unroll
                    for (int co = 0; co < COUT; ++co) {
                        const T wv = wr[co];
#pragma unroll
                        for (int i = 0; i < PX; ++i) acc[i][co] += wv * v[i + kx];
                    }
                }
            }
#pragma unroll
        for (int i = 0; i < PX; ++i) {
            if constexpr (SPLIT) {
                store_relu_row_split<COUT>(acc[i], out + ((size_t)m * HW + p + i) * (2 * COUT));
            } else {
                store_relu_row<T, Tout, COUT>(acc[i], out + ((size_t)m * HW + p + i) * COUT);
            }
        }
    }
}

template <typename T> __device__ __forceinline__ T ld_as(const float *p) { return (T)(*p); }
template <typename T> __device__ __forceinline__ T ld_as(const double *p) { return (T)(*p); }
template <typename T> __device__ __forceinline__ T ld_as(const __nv_bfloat16 *p) { return (T)__bfloat162float(*p); }
template <typename Tout, typename T> __device__ __forceinline__ Tout st_as(T v) { return (Tout)v; }
template <> __device__ __forceinline__ __nv_bfloat16 st_as<__nv_bfloat16, float>(float v) { return __float2bfloat16_rn(v); }

// conv3x3 (stride 1, zero pad 1) + bias + ReLU on NHWC activations of the
// first *count frames, as an implicit GEMM on CUDA cores:
//   out[m][p][co] = relu(b[co] + sum_{tap, ci} in[m][p + shift(tap)][ci] * Wt[tap][ci][co])
// Tiles of PX (128 or 64) pixels x 64 output channels; K walks (tap, 16 input
// channels), so a tile's latency is its K loop: recheck bands of a few frames
// take 64-pixel tiles (half the work per step, twice the CTAs; 32-pixel tiles
// measured no faster on the CNN workload's FP32 bands).
// KS = 3 or 9 (bands only): when *count <= split_frames, the K loop is split by
// kernel row (KS = 3: taps 3j..3j+2 for split j) or by tap (KS = 9), so a band of a
// few frames has KS times the CTAs with 1/KS of the K loop each.  Each split writes
// its raw sums to plane j of a partial buffer placed after the first split_frames
// frames of `out` ([KS][split_frames][H*W][Cout] elements of T, so `out` must hold
// (KS + 1) x split_frames frames); k_conv_splitk_sum adds the planes in order 0, 1,
// ..., then the bias, and applies the ReLU.  Above split_frames the kernel runs
// unsplit.
// Requires Cin % 16 == 0, Cout % 64 == 0, H*W % 128 == 0.
template <int PX, int KS, typename Tin, typename Tw, typename T, typename Tout>
__global__ void __launch_bounds__(256)
k_conv3x3_simt(const int *count, const Tin *in, int Cin, int H, int Wd, const Tw *Wt, const float *bias,
               int Cout, Tout *out, int split_frames) {
    static_assert(KS == 1 || KS == 3 || KS == 9, "K splits: 1, 3 (one kernel row each) or 9 (one tap each)");
    constexpr int RI = PX / 16;       // output pixels per thread, A elements per loader thread
    constexpr int APT = 16 / RI;      // loader threads per pixel
    // 16-byte aligned rows (PX + 4 and 68 elements): a thread's RI A values and 4 B values
    // of a K row are contiguous and aligned, so they can be read with vector loads
    __shared__ __align__(16) T As[16][PX + 4];
    __shared__ __align__(16) T Bs[16][64 + 4];
    const int M = *count;
    const int ks = (KS > 1 && M <= split_frames) ? KS : 1;
    const int HW = H * Wd;
    const int tiles_p = HW / PX, tiles_c = Cout / 64;
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    const int apx = t / APT, ach = (t % APT) * RI;   // A loader: pixel, channel offset
    const int bk = t >> 4, bn = (t & 15) * 4;    // B loader: k row, channel offset
    for (long long tile = blockIdx.x; tile < (long long)M * tiles_p * tiles_c * ks; tile += gridDim.x) {
        const int j = (int)(tile % ks);
        const long long u = tile / ks;
        const int m = (int)(u / (tiles_p * tiles_c));
        const int r = (int)(u % (tiles_p * tiles_c));
        const int p0 = (r / tiles_c) * PX, co0 = (r % tiles_c) * 64;
        const Tin *fin = in + (size_t)m * HW * Cin;
        const int ap = p0 + apx, ay = ap / Wd, ax = ap % Wd;
        T acc[RI][4];
#pragma unroll
        for (int i = 0; i < RI; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = (T)0;
        // K steps (tap, 16 input channels); the next step's operands are loaded
        // into registers while this step's multiply-adds run (latency hiding)
        const int csteps = Cin / 16, tap0 = j * (9 / ks), nsteps = (9 / ks) * csteps;
        T ra[RI], rw[4];
        auto fetch = [&](int s) {
            const int tap = tap0 + s / csteps, ci0 = (s % csteps) * 16;
            const int yy = ay + tap / 3 - 1, xx = ax + tap % 3 - 1;
            const bool inb = yy >= 0 && yy < H && xx >= 0 && xx < Wd;
            const Tin *src = fin + ((size_t)(inb ? yy : 0) * Wd + (inb ? xx : 0)) * Cin + ci0 + ach;
#pragma unroll
            for (int e = 0; e < RI; ++e) ra[e] = inb ? ld_as<T>(src + e) : (T)0;
            const Tw *wsrc = Wt + ((size_t)tap * Cin + ci0 + bk) * Cout + co0 + bn;
#pragma unroll
            for (int e = 0; e < 4; ++e) rw[e] = ld_as<T>(wsrc + e);
        };
        fetch(0);
        for (int s = 0; s < nsteps; ++s) {
#pragma unroll
            for (int e = 0; e < RI; ++e) As[ach + e][apx] = ra[e];
#pragma unroll
            for (int e = 0; e < 4; ++e) Bs[bk][bn + e] = rw[e];
            __syncthreads();
            if (s + 1 < nsteps) fetch(s + 1);
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) {
                T a[RI], w[4];
#pragma unroll
                for (int i = 0; i < RI; ++i) a[i] = As[kk][ty * RI + i];
#pragma unroll
                for (int j = 0; j < 4; ++j) w[j] = Bs[kk][tx * 4 + j];
#pragma unroll
                for (int i = 0; i < RI; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * w[j];
            }
            __syncthreads();
        }
        if constexpr (KS > 1) {
            if (ks > 1) {
                T *o = reinterpret_cast<T *>(out) + ((size_t)(j + 1) * split_frames + m) * HW * Cout +
                       (size_t)(p0 + ty * RI) * Cout + co0 + tx * 4;
#pragma unroll
                for (int i = 0; i < RI; ++i)
#pragma unroll
                    for (int e = 0; e < 4; ++e) o[(size_t)i * Cout + e] = acc[i][e];
                continue;
            }
        }
        Tout *o = out + ((size_t)m * HW + p0 + ty * RI) * Cout + co0 + tx * 4;
#pragma unroll
        for (int i = 0; i < RI; ++i)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                T v = acc[i][e] + (T)bias[co0 + tx * 4 + e];
                if (v < (T)0) v = (T)0;
                o[(size_t)i * Cout + e] = st_as<Tout, T>(v);
            }
    }
}

// Second half of a K-split band conv: out[m][p][co] = relu(P0 + P1 + ... + b[co]) with the
// planes added in order 0, 1, ..., ks-1; does nothing when *count > split_frames (the conv ran
// unsplit).  Each thread takes 16 bytes (4 floats or 2 doubles) of every plane with one load.
template <typename T> struct Vec16;
template <> struct Vec16<float> { using V = float4; static constexpr int N = 4; };
template <> struct Vec16<double> { using V = double2; static constexpr int N = 2; };

template <typename T>
__global__ void __launch_bounds__(256)
k_conv_splitk_sum(const int *count, int HW, int Cout, const float *bias, T *out, int split_frames, int ks) {
    using V = typename Vec16<T>::V;
    constexpr int N = Vec16<T>::N;
    const int M = *count;
    if (M > split_frames) return;
    const size_t plane = (size_t)split_frames * HW * Cout, nv = (size_t)M * HW * Cout / N;
    const T *part = out + plane;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (size_t)gridDim.x * blockDim.x) {
        T acc[N];
        {
            const V v = reinterpret_cast<const V *>(part)[i];
            const T *e = reinterpret_cast<const T *>(&v);
#pragma unroll
            for (int k = 0; k < N; ++k) acc[k] = e[k];
        }
        for (int j = 1; j < ks; ++j) {
            const V v = reinterpret_cast<const V *>(part + j * plane)[i];
            const T *e = reinterpret_cast<const T *>(&v);
#pragma unroll
            for (int k = 0; k < N; ++k) acc[k] += e[k];
        }
        V o;
        T *oe = reinterpret_cast<T *>(&o);
        const int co = (int)((i * N) % Cout);
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const T v = acc[k] + (T)bias[co + k];
            oe[k] = v < (T)0 ? (T)0 : v;
        }
        reinterpret_cast<V *>(out)[i] = o;
    }
}

// Global average pool + linear head: score[m] = hb + sum_c hw[c] * mean_p act[m][p][c].
// One block per frame; fixed-order partial sums (deterministic).
constexpr int kPoolThreads = 1024;   // per frame: C channels x (1024 / C) pixel groups

// The FP32 / FP64 recheck levels pool a band of a few frames (often one): one block per frame
// reads its 1-2 MB with too few loads in flight, so these levels split each frame by 32-channel
// group and by PS pixel ranges of HW / PS pixels.
// k_pool_sum: per (frame, channel group, pixel range j), 32 channels x 32 pixel groups sum in a
// fixed order and leave the range's channel sums in place of the range's first pixel j * HW / PS
// (only this block reads those channels of that range); k_head_dot: one warp per frame,
// hb + sum_c hw[c] * (sum over j = 0 .. PS-1 in order of the range sums) / HW with a fixed
// butterfly order.  Both deterministic; C a multiple of 32, HW a multiple of 32 * PS.
template <typename T>
__global__ void __launch_bounds__(1024) k_pool_sum(const int *count, T *act, int HW, int C, int ps) {
    __shared__ T part[32][33];
    const int M = *count, G = C / 32, R = HW / ps;
    const int c = threadIdx.x & 31, g = threadIdx.x >> 5;
    for (long long u = blockIdx.x; u < (long long)M * G * ps; u += gridDim.x) {
        const int j = (int)(u % ps);
        const long long v = u / ps;
        const int m = (int)(v / G), cg = (int)(v % G);
        T *a = act + ((size_t)m * HW + (size_t)j * R) * C + cg * 32 + c;
        T s = (T)0;
#pragma unroll 8
        for (int p = g; p < R; p += 32) s += a[(size_t)p * C];
        part[g][c] = s;
        __syncthreads();
        if (g == 0) {
            T tot = (T)0;
            for (int q = 0; q < 32; ++q) tot += part[q][c];
            a[0] = tot;
        }
        __syncthreads();
    }
}

template <typename T, typename S>
__global__ void k_head_dot(const int *count, const T *act, int HW, int C, int ps, const float *hw, double hb,
                           S *score) {
    const int M = *count;
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const size_t range = (size_t)(HW / ps) * C;
    for (int m = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; m < M; m += warps) {
        const T *pooled = act + (size_t)m * HW * C;
        T r = (T)0;
        for (int c = lane; c < C; c += 32) {
            // the range sums' loads issue together; the adds stay in order j = 0 .. ps-1
            T v[16];
            T sc = (T)0;
            for (int j0 = 0; j0 < ps; j0 += 16) {
                const int nj = ps - j0 < 16 ? ps - j0 : 16;
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = j < nj ? pooled[(j0 + j) * range + c] : (T)0;
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (j < nj) sc += v[j];
            }
            r += (T)hw[c] * (sc / (T)HW);
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) r += __shfl_xor_sync(0xffffffffu, r, d);
        if (lane == 0) score[m] = (S)((T)hb + r);
    }
}

template <typename Tin, typename T, typename S>
__global__ void __launch_bounds__(kPoolThreads)
k_pool_head(const int *count, const Tin *act, int HW, int C, const float *hw, double hb, S *score) {
    __shared__ T part[kPoolThreads];
    __shared__ T pooled[256];
    const int M = *count;
    const int groups = kPoolThreads / C;
    const int c = threadIdx.x % C, g = threadIdx.x / C;
    for (int m = blockIdx.x; m < M; m += gridDim.x) {
        const Tin *a = act + (size_t)m * HW * C;
        T s = (T)0;
        if (g < groups)
#pragma unroll 8
            for (int p = g; p < HW; p += groups) s += ld_as<T>(a + (size_t)p * C + c);
        part[threadIdx.x] = s;
        __syncthreads();
        if (threadIdx.x < C) {
            T tot = (T)0;
            for (int q = 0; q < groups; ++q) tot += part[q * C + threadIdx.x];
            pooled[threadIdx.x] = tot / (T)HW;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            T r = (T)hb;
            for (int q = 0; q < C; ++q) r += (T)hw[q] * pooled[q];
            score[m] = (S)r;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- launchers

static int grid_for(int sms, int per_sm) { return sms * per_sm; }

void launch_mlp_layer_f32(const int *count, const int *rows, const float *X, int ldx, const float *W,
                          const float *b, float *Y, int K, int N, int relu, int max_rows, int sms,
                          cudaStream_t st, const long long *ids) {
    const int tiles = ((max_rows + 63) / 64) * ((N + 63) / 64);
    int grid = tiles < grid_for(sms, 4) ? tiles : grid_for(sms, 4);
    if (grid < 1) grid = 1;
    const int vec4 = (K % 4 == 0 && ldx % 4 == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0 &&
                      (reinterpret_cast<uintptr_t>(W) & 15) == 0) ? 1 : 0;
    k_mlp_layer_f32<<<grid, 256, 0, st>>>(count, rows, X, ldx, W, b, Y, K, N, relu, ids, vec4);
}

void launch_mlp_dot_f32(const int *count, const int *rows, const float *X, int ldx, const float *w,
                        float bias, int K, float *score, int max_rows, int sms, cudaStream_t st,
                        const long long *ids) {
    int grid = (max_rows + 7) / 8;
    if (grid > grid_for(sms, 8)) grid = grid_for(sms, 8);
    if (grid < 1) grid = 1;
    k_mlp_dot_f32<<<grid, 256, 0, st>>>(count, rows, X, ldx, w, bias, K, score, ids);
}

void launch_mlp_band_f32(const int *band_count, const int *band_tuple, const float *X, int ldx,
                         const MlpDev &mlp, float *score_out, int sms, cudaStream_t st) {
    const size_t smem = sizeof(float) * 2 * mlp.max_width;
    k_mlp_band<float><<<grid_for(sms, 2), 256, smem, st>>>(band_count, band_tuple, X, ldx, mlp, score_out);
}

void launch_mlp_band_f64(const int *band_count, const int *band_tuple, const float *X, int ldx,
                         const MlpDev &mlp, double *score_out, int sms, cudaStream_t st) {
    const size_t smem = sizeof(double) * 2 * mlp.max_width;
    k_mlp_band<double><<<grid_for(sms, 2), 256, smem, st>>>(band_count, band_tuple, X, ldx, mlp, score_out);
}

cudaError_t mlp_band_smem_setup(int max_width) {
    const size_t s64 = sizeof(double) * 2 * (size_t)max_width;
    const size_t s32 = sizeof(float) * 2 * (size_t)max_width;
    cudaError_t e = cudaFuncSetAttribute(k_mlp_band<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s64);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_mlp_band<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s32);
}

template <typename T, typename Tout, int PX, bool SPLIT = false>
static void conv1_dispatch(const int *count, const int *list, const unsigned char *frames, int C0, int H,
                           int Wd, const float *W, const float *bias, int Cout, Tout *out, int max_frames, int sms,
                           cudaStream_t st) {
    const int work = max_frames * ((H * Wd + 256 * PX - 1) / (256 * PX));
    int grid = work < grid_for(sms, 8) ? work : grid_for(sms, 8);
    if (grid < 1) grid = 1;
    constexpr int PX64 = PX > 2 ? 2 : PX;   // 64 channels: fewer pixels per thread (registers)
    switch (Cout) {
        case 16: k_conv1_u8<T, Tout, 16, PX, SPLIT><<<grid, 256, 0, st>>>(count, list, frames, C0, H, Wd, W, bias, out); break;
        case 32: k_conv1_u8<T, Tout, 32, PX, SPLIT><<<grid, 256, 0, st>>>(count, list, frames, C0, H, Wd, W, bias, out); break;
        default: {
            const int work64 = max_frames * ((H * Wd + 256 * PX64 - 1) / (256 * PX64));
            int g64 = work64 < grid_for(sms, 8) ? work64 : grid_for(sms, 8);
            if (g64 < 1) g64 = 1;
            k_conv1_u8<T, Tout, 64, PX64, SPLIT><<<g64, 256, 0, st>>>(count, list, frames, C0, H, Wd, W, bias, out);
            break;
        }
    }
}

void launch_conv1(int prec, const int *count, const int *list, const unsigned char *frames, int C0, int H,
                  int Wd, const float *W, const float *bias, int Cout, void *out, int max_frames, int sms,
                  cudaStream_t st, bool band) {
    // a recheck band (often one frame) takes one pixel per thread: four times the threads
    const bool px4 = Wd % 4 == 0 && !band;
    if (prec == PREC_F64)
        conv1_dispatch<double, double, 1>(count, list, frames, C0, H, Wd, W, bias, Cout, (double *)out, max_frames,
                                          sms, st);
    else if (prec == PREC_F32) {
        if (px4)
            conv1_dispatch<float, float, 4>(count, list, frames, C0, H, Wd, W, bias, Cout, (float *)out, max_frames,
                                            sms, st);
        else
            conv1_dispatch<float, float, 1>(count, list, frames, C0, H, Wd, W, bias, Cout, (float *)out, max_frames,
                                            sms, st);
    } else {
        if (px4)
            conv1_dispatch<float, __nv_bfloat16, 4>(count, list, frames, C0, H, Wd, W, bias, Cout,
                                                    (__nv_bfloat16 *)out, max_frames, sms, st);
        else
            conv1_dispatch<float, __nv_bfloat16, 1>(count, list, frames, C0, H, Wd, W, bias, Cout,
                                                    (__nv_bfloat16 *)out, max_frames, sms, st);
    }
}

void launch_conv1_split(const int *count, const int *list, const unsigned char *frames, int C0, int H, int Wd,
                        const float *W, const float *bias, int Cout, void *out, int max_frames, int sms,
                        cudaStream_t st, bool bf16_planes) {
    if (bf16_planes) {
        // the split-BF16 level runs on recheck bands of a few dozen frames: two pixels per
        // thread give twice the threads of four, with the same weight reads per multiply-add
        // pair
        __nv_bfloat16 *o = (__nv_bfloat16 *)out;
        if (Wd % 2 == 0)
            conv1_dispatch<float, __nv_bfloat16, 2, true>(count, list, frames, C0, H, Wd, W, bias, Cout, o, max_frames,
                                                          sms, st);
        else
            conv1_dispatch<float, __nv_bfloat16, 1, true>(count, list, frames, C0, H, Wd, W, bias, Cout, o, max_frames,
                                                          sms, st);
        return;
    }
    float *o = (float *)out;
    if (Wd % 4 == 0)
        conv1_dispatch<float, float, 4, true>(count, list, frames, C0, H, Wd, W, bias, Cout, o, max_frames, sms, st);
    else
        conv1_dispatch<float, float, 1, true>(count, list, frames, C0, H, Wd, W, bias, Cout, o, max_frames, sms, st);
}

int launch_conv3x3_simt(int prec, const int *count, const void *in, int Cin, int H, int Wd, const void *Wt,
                        const float *bias, int Cout, void *out, int max_frames, int sms, cudaStream_t st, bool band) {
    const int px = band ? 64 : 128;
    // FP32 / FP64 bands of up to split_frames frames split the K loop; the partial planes live
    // in `out` behind the first split_frames frames ((ks + 1) x split_frames <= max_frames)
    // (FP32: nine splits, one tap each; FP64: three)
    const int ks_want = prec == PREC_F32 ? 9 : 3;
    const int split_frames =
        band && (prec == PREC_F64 || prec == PREC_F32) ? std::min(8, max_frames / (ks_want + 1)) : 0;
    const int ks = split_frames > 0 ? ks_want : 1;
    const long long tiles = (long long)std::max(max_frames, ks * split_frames) * (H * Wd / px) * (Cout / 64);
    int grid = tiles < grid_for(sms, 4) ? (int)tiles : grid_for(sms, 4);
    if (grid < 1) grid = 1;
    auto run = [&](auto kern, const auto *xin, const auto *w, auto *xout) {
        kern<<<grid, 256, 0, st>>>(count, xin, Cin, H, Wd, w, bias, Cout, xout, split_frames);
    };
    auto finish = [&](auto *xout) {
        const long long n = (long long)split_frames * H * Wd * Cout / 4;   // 16-byte vectors of floats
        const int g = (int)std::min<long long>((n + 255) / 256, grid_for(sms, 8));
        k_conv_splitk_sum<<<g, 256, 0, st>>>(count, H * Wd, Cout, bias, xout, split_frames, ks);
        return 2;
    };
    if (prec == PREC_F64) {
        if (ks > 1) {
            run(k_conv3x3_simt<64, 3, double, float, double, double>, (const double *)in, (const float *)Wt,
                (double *)out);
            return finish((double *)out);
        }
        if (band)
            run(k_conv3x3_simt<64, 1, double, float, double, double>, (const double *)in, (const float *)Wt,
                (double *)out);
        else
            run(k_conv3x3_simt<128, 1, double, float, double, double>, (const double *)in, (const float *)Wt,
                (double *)out);
    } else if (prec == PREC_F32) {
        if (ks > 1) {
            run(k_conv3x3_simt<64, 9, float, float, float, float>, (const float *)in, (const float *)Wt, (float *)out);
            return finish((float *)out);
        }
        if (band)
            run(k_conv3x3_simt<64, 1, float, float, float, float>, (const float *)in, (const float *)Wt, (float *)out);
        else
            run(k_conv3x3_simt<128, 1, float, float, float, float>, (const float *)in, (const float *)Wt, (float *)out);
    } else {
        run(k_conv3x3_simt<128, 1, __nv_bfloat16, __nv_bfloat16, float, __nv_bfloat16>, (const __nv_bfloat16 *)in,
            (const __nv_bfloat16 *)Wt, (__nv_bfloat16 *)out);
    }
    return 1;
}

int launch_pool_head(int prec, const int *count, void *act, int HW, int C, const float *hw, double hb,
                     void *score, int max_frames, int sms, cudaStream_t st) {
    int grid = max_frames < grid_for(sms, 2) ? max_frames : grid_for(sms, 2);
    if (grid < 1) grid = 1;
    if ((prec == PREC_F64 || prec == PREC_F32) && C % 32 == 0) {
        const int ps = HW % (32 * 16) == 0 ? 16 : 1;   // pixel ranges per (frame, channel group)
        const long long units = (long long)max_frames * (C / 32) * ps;
        const int g1 = (int)(units < grid_for(sms, 2) ? (units < 1 ? 1 : units) : grid_for(sms, 2));
        int g2 = (max_frames + 7) / 8;
        if (g2 > grid_for(sms, 4)) g2 = grid_for(sms, 4);
        if (g2 < 1) g2 = 1;
        if (prec == PREC_F64) {
            k_pool_sum<double><<<g1, 1024, 0, st>>>(count, (double *)act, HW, C, ps);
            k_head_dot<double, double><<<g2, 256, 0, st>>>(count, (const double *)act, HW, C, ps, hw, hb,
                                                           (double *)score);
        } else {
            k_pool_sum<float><<<g1, 1024, 0, st>>>(count, (float *)act, HW, C, ps);
            k_head_dot<float, float><<<g2, 256, 0, st>>>(count, (const float *)act, HW, C, ps, hw, hb,
                                                         (float *)score);
        }
        return 2;
    }
    if (prec == PREC_F64)
        k_pool_head<double, double, double><<<grid, kPoolThreads, 0, st>>>(count, (const double *)act, HW, C, hw, hb,
                                                                           (double *)score);
    else if (prec == PREC_F32)
        k_pool_head<float, float, float><<<grid, kPoolThreads, 0, st>>>(count, (const float *)act, HW, C, hw, hb,
                                                                        (float *)score);
    else
        k_pool_head<__nv_bfloat16, float, float><<<grid, kPoolThreads, 0, st>>>(count, (const __nv_bfloat16 *)act,
                                                                                HW, C, hw, hb, (float *)score);
    return 1;
}

}  // namespace hydro
