// FP32 CUDA-core GEMM tile shared by the grouped (per-predicate queue) layer
// kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hydro {

// Four consecutive k (from k0 + lk) of an X row and a W row, zero past K or for a missing row.
// vec4: K % 4 == 0 with 16-byte aligned rows, so the four are all in range or all out.
static __device__ __forceinline__ void mlp_tile_fetch(const float *arow, const float *wrow, int K, int lk, int k0,
                                                      bool vec4, float4 &ra, float4 &rw) {
    const int k = k0 + lk;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    if (vec4) {
        ra = (arow && k < K) ? *reinterpret_cast<const float4 *>(arow + k) : z;
        rw = (wrow && k < K) ? *reinterpret_cast<const float4 *>(wrow + k) : z;
    } else {
        ra = make_float4((arow && k < K) ? arow[k] : 0.f, (arow && k + 1 < K) ? arow[k + 1] : 0.f,
                         (arow && k + 2 < K) ? arow[k + 2] : 0.f, (arow && k + 3 < K) ? arow[k + 3] : 0.f);
        rw = make_float4((wrow && k < K) ? wrow[k] : 0.f, (wrow && k + 1 < K) ? wrow[k + 1] : 0.f,
                         (wrow && k + 2 < K) ? wrow[k + 2] : 0.f, (wrow && k + 3 < K) ? wrow[k + 3] : 0.f);
    }
}

// The fetched k of row lr into column lr of a K slice (transposed, k-major in shared memory).
static __device__ __forceinline__ void mlp_tile_put(float (&As)[16][68], float (&Ws)[16][68], int lk, int lr,
                                                    const float4 &ra, const float4 &rw) {
    As[lk][lr] = ra.x, As[lk + 1][lr] = ra.y, As[lk + 2][lr] = ra.z, As[lk + 3][lr] = ra.w;
    Ws[lk][lr] = rw.x, Ws[lk + 1][lr] = rw.y, Ws[lk + 2][lr] = rw.z, Ws[lk + 3][lr] = rw.w;
}

// One tile of Y = act(X[rows] W^T + b): 64x64 outputs, K in slices of 16,
// 4x4 outputs per thread (256 threads).  Row m of the tile reads X row
// rows[m] (rows nullable: row m) and writes Y row m (row stride ldy).  The
// K slices alternate between two shared buffers and the next slice's global
// loads (16 bytes per row when K, ldx and the bases allow) are in flight while
// the current slice is multiplied; every output's multiply-adds run in k order.
static __device__ __forceinline__ void mlp_tile_f32(int M, int m0, int n0, const int *rows, const float *X, int ldx,
                                             const float *W, const float *b, float *Y, int ldy, int K, int N, int relu,
                                             float (&As)[2][16][68], float (&Ws)[2][16][68]) {
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    const int lr = t >> 2, lk = (t & 3) * 4;
    float acc[4][4] = {};
    const int am = m0 + lr;
    const float *arow = am < M ? X + (size_t)(rows ? rows[am] : am) * ldx : nullptr;
    const int wn = n0 + lr;
    const float *wrow = wn < N ? W + (size_t)wn * K : nullptr;
    const bool vec4 = K % 4 == 0 && ldx % 4 == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0 &&
                      (reinterpret_cast<uintptr_t>(W) & 15) == 0;
    float4 ra, rw;   // this thread's four k of its X row and W row for the next slice
    mlp_tile_fetch(arow, wrow, K, lk, 0, vec4, ra, rw);
    mlp_tile_put(As[0], Ws[0], lk, lr, ra, rw);
    __syncthreads();
    int buf = 0;
    for (int k0 = 0; k0 < K; k0 += 16) {
        const bool more = k0 + 16 < K;
        if (more) mlp_tile_fetch(arow, wrow, K, lk, k0 + 16, vec4, ra, rw);
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
        if (more) mlp_tile_put(As[buf ^ 1], Ws[buf ^ 1], lk, lr, ra, rw);
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
            float v = acc[i][j] + (b ? b[n] : 0.f);
            if (relu && v < 0.f) v = 0.f;
            Y[(size_t)m * ldy + n] = v;
        }
    }
}

}  // namespace hydro
