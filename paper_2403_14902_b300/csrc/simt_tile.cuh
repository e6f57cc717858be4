// FP32 CUDA-core GEMM tile shared by the grouped (per-predicate queue) layer
// kernels.
#pragma once

#include <cuda_runtime.h>

namespace hydro {

// One tile of Y = act(X[rows] W^T + b): 64x64 outputs, K in slices of 16,
// 4x4 outputs per thread (256 threads).  Row m of the tile reads X row
// rows[m] (rows nullable: row m) and writes Y row m (row stride ldy).
static __device__ __forceinline__ void mlp_tile_f32(int M, int m0, int n0, const int *rows, const float *X, int ldx,
                                             const float *W, const float *b, float *Y, int ldy, int K, int N, int relu,
                                             float (&As)[16][68], float (&Ws)[16][68]) {
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    const int lr = t >> 2, lk = (t & 3) * 4;
    float acc[4][4] = {};
    const int am = m0 + lr;
    const float *arow = am < M ? X + (size_t)(rows ? rows[am] : am) * ldx : nullptr;
    const int wn = n0 + lr;
    const float *wrow = wn < N ? W + (size_t)wn * K : nullptr;
    for (int k0 = 0; k0 < K; k0 += 16) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int k = k0 + lk + e;
            As[lk + e][lr] = (arow && k < K) ? arow[k] : 0.f;
            Ws[lk + e][lr] = (wrow && k < K) ? wrow[k] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], w[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) w[j] = Ws[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], w[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty * 4 + i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx * 4 + j;
            if (n >= N) continue;
            float v = acc[i][j] + (b ? b[n] : 0.f);
            if (relu && v < 0.f) v = 0.f;
            Y[(size_t)m * ldy + n] = v;
        }
    }
}

}  // namespace hydro
