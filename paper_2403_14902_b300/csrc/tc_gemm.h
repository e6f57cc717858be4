// Tensor-core (tcgen05, TMA-fed) BF16 MLP layers and the BF16 row gather.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/hydro.h"

namespace hydro {

constexpr int kMaxGroups = 8;

// One layer of one group of a grouped launch.  The group's rows are stacked
// after the earlier groups' rows (row offset = sum of the earlier counts).
struct TcGemmGroup {
    const int *count;            // rows of the group (device)
    const __nv_bfloat16 *X;      // stacked operand, row stride ldx elements (multiple of 8)
    int ldx;
    long long x_rows;            // rows of X's allocation
    const __nv_bfloat16 *W;      // [N][K]
    const float *bias;           // [N]
    const float *head_w;         // [N] one-output head folded into the epilogue, or nullptr (store Y)
    int K, N;
    int nt;                      // column-tile width 64/128/256 dividing N; 0: the widest that divides
    // FP8 (E4M3) group: with W8 set, the layer reads X8 (stacked E4M3 rows,
    // row stride ldx bytes, K % 128 == 0) and W8 (E4M3 [N][K]) instead of X
    // and W, and the epilogue scales the accumulator of row m, column n by
    // ascale[m] * wscale[n] (m: stacked row) before the bias.
    const unsigned char *X8 = nullptr;
    const unsigned char *W8 = nullptr;
    const float *ascale = nullptr;
    const float *wscale = nullptr;
};
// A group with W == nullptr (and W8 == nullptr) contributes only its row
// count to the stacking.

struct TcHeads {                 // per group: head bias and head partials per row of the last hidden layer
    float b[kMaxGroups];
    int tiles[kMaxGroups];
};

// Layer shape K -> N runs on the tensor cores (K, N multiples of 64; FP8
// layers also need K % 128 == 0).
bool tc_gemm_supported(int K, int N);
bool tc_gemm_fp8_supported(int K, int N);
// Look up the tensor-map encoder and set kernel attributes (once per query).
hydro_status tc_gemm_init(void **encode);
// Y[m] = relu(X[m] W^T + bias) (bf16, [rows][N]) for m < *count; X is bf16
// [max_rows][K], W bf16 [N][K].  With head_w (the UDF's one-output last layer,
// fp32 [N]) nothing is stored to Y: partials[m * tc_gemm_col_tiles(N) + j]
// receives head_w . relu(...) over column half-tile j.
hydro_status tc_gemm_run(void *encode, const int *count, const __nv_bfloat16 *X, int K, const __nv_bfloat16 *W,
                         const float *bias, int N, __nv_bfloat16 *Y, int max_rows, int sms, cudaStream_t st,
                         unsigned int *err, const float *head_w = nullptr, float *partials = nullptr);
// Head partials per row of a fused-head layer of width N (two per column
// tile: the epilogue's column halves); nt as in TcGemmGroup.
int tc_gemm_col_tiles(int N);
int tc_gemm_head_parts(int N, int nt);
// Tile scheduling of a grouped launch.  data_aware: tiles numbered heaviest
// first (K x column-tile width) and claimed one at a time by the CTA that is
// ready for one, through counters (two ints, zero before the first launch;
// the launch leaves them zero); else static round robin in group order.
// rec (nullable): per CTA the global-timer ns of its first and last work,
// [grid][2] (CTAs without tiles leave theirs untouched).
struct TcSched {
    int data_aware = 0;
    int *counters = nullptr;
    unsigned long long *rec = nullptr;
};
// All groups' layers of one depth in one persistent launch.  Y (stacked,
// row stride ldy) receives the groups without a head; partials (stacked, row
// stride pstride) the head partials of the others.
// split3: store Y rows as [hi | hi | lo] BF16 splits (3N columns, ldy >= 3N)
// for a split-BF16 next layer.  min_rows: with fewer stacked rows than this
// (read on the device) the launch does nothing.
hydro_status tc_gemm_grouped_run(void *encode, const TcGemmGroup *groups, int n, __nv_bfloat16 *Y, int ldy,
                                 float *partials, int pstride, int sms, cudaStream_t st, unsigned int *err,
                                 bool split3 = false, int min_rows = 0, const TcSched *sched = nullptr);
// out[off_g + m] = bf16(X[queues[g * qstride + m]]) for m < counts[g], X = *Xp
// (read on the device, so a captured launch follows the pointer's updates).
void launch_gather_grouped_bf16(int n, const int *counts, const int *queues, int qstride, const float *const *Xp,
                                int ldx, int K, __nv_bfloat16 *out, int max_rows, int sms, cudaStream_t st);
// Split-BF16 rows: out[off_g + m] = [hi | hi | lo] of X[queues[g * qstride + m]]
// (3K columns), hi = bf16(x), lo = bf16(x - hi).
void launch_gather_grouped_bf16x3(int n, const int *counts, const int *queues, int qstride, const float *const *Xp,
                                  int ldx, int K, __nv_bfloat16 *out, int max_rows, int sms, cudaStream_t st,
                                  int min_rows = 0);
// score[g * sstride + m] = heads.b[g] + sum_j partials[(off_g + m) * pstride + j], j < heads.tiles[g].
void launch_head_finalize_grouped(int n, const int *counts, const TcHeads &heads, const float *partials, int pstride,
                                  float *score, int sstride, int max_rows, int sms, cudaStream_t st,
                                  int min_rows = 0);
// Level-0 operand of a session whose groups in q8_mask run their first layer
// in FP8: stacked row e of group g (source X[queues[g * qstride + m]]) goes
// to out8 as E4M3 codes of x / ascale[e], ascale[e] = max_k |x_k| / 448, when
// bit g of q8_mask is set, else to out16 as BF16.  K % 128 == 0.
void launch_gather_grouped_mixed(int n, const int *counts, const int *queues, int qstride, const float *const *Xp,
                                 int ldx, int K, unsigned q8_mask, __nv_bfloat16 *out16, unsigned char *out8,
                                 float *ascale, int max_rows, int sms, cudaStream_t st);
// Per-row E4M3 quantisation of a fp32 [rows][K] matrix (K % 128 == 0):
// scale[r] = max_k |X[r][k]| / 448 and out[r][k] = e4m3(X[r][k] / scale[r])
// (saturating; an all-zero row gets scale 0 and zero codes).
void launch_quant_rows_e4m3(const float *X, int rows, int K, unsigned char *out, float *scale, int sms,
                            cudaStream_t st);
// out[m] = bf16(X[rows[m]]) for m < *count (K % 8 == 0, 16-byte aligned rows).
void launch_gather_bf16(const int *count, const int *rows, const float *X, int ldx, int K, __nv_bfloat16 *out,
                        int max_rows, int sms, cudaStream_t st);
const char *tc_gemm_last_error();

}  // namespace hydro
