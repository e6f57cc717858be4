// Tensor-core (tcgen05, TMA-fed) BF16 MLP layers and the BF16 row gather.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/hydro.h"

namespace hydro {

// Layer shape K -> N runs on the tensor cores (K, N multiples of 64).
bool tc_gemm_supported(int K, int N);
// Look up the tensor-map encoder and set kernel attributes (once per query).
hydro_status tc_gemm_init(void **encode);
// Y[m] = relu(X[m] W^T + bias) (bf16, [rows][N]) for m < *count; X is bf16
// [max_rows][K], W bf16 [N][K].  With head_w (the UDF's one-output last layer,
// fp32 [N]) nothing is stored to Y: partials[m * tc_gemm_col_tiles(N) + j]
// receives head_w . relu(...) over column tile j.
hydro_status tc_gemm_run(void *encode, const int *count, const __nv_bfloat16 *X, int K, const __nv_bfloat16 *W,
                         const float *bias, int N, __nv_bfloat16 *Y, int max_rows, int sms, cudaStream_t st,
                         unsigned int *err, const float *head_w = nullptr, float *partials = nullptr);
int tc_gemm_col_tiles(int N);
// out[m] = bf16(X[rows[m]]) for m < *count (K % 8 == 0, 16-byte aligned rows).
void launch_gather_bf16(const int *count, const int *rows, const float *X, int ldx, int K, __nv_bfloat16 *out,
                        int max_rows, int sms, cudaStream_t st);
const char *tc_gemm_last_error();

}  // namespace hydro
