// Device side of multi-query sessions: one step = every query's next chunk
// of tuples, stacked query after query, routed per query and evaluated in
// rounds of grouped launches (one group per pool UDF).
#pragma once

#include <cuda_runtime.h>

#include "../../include/hydro.h"
#include "common.cuh"
#include "internal.h"
#include "tc_gemm.h"

namespace hydro {

constexpr int kMqMaxQ = HYDRO_MAX_QUERIES;
constexpr int kMqPool = HYDRO_MAX_POOL;
constexpr int kMqSlots = HYDRO_MAX_PREDICATES;

// What the host sends per step (one H2D copy from pinned memory).
struct StepHdr {
    const float *X;            // stacked fp32 rows of the step
    int counts[kMqMaxQ];       // rows per query
};

// Precision levels of a round.  Every entry of a level's lists is decided
// there or sent to the next level's list of the same group.
//   BF16 sessions: 0 BF16 -> 1 split BF16 (tensor cores) -> 2 FP32 -> 3 FP64
//   FP8 sessions:  0 FP8 first layer (UDFs in the FP8 set) or BF16 (the
//                  others) -> 1 BF16 (FP8 set only; the others skip to 2)
//                  -> 2 FP32 -> 3 FP64
//   FP32 sessions: 0 FP32 -> 3 FP64
enum { LV_MAIN = 0, LV_X3 = 1, LV_F32 = 2, LV_F64 = 3, LV_N = 4 };

// The split-BF16 level runs only on bands of at least this many rows (all
// groups together); smaller bands go straight to the FP32 level, whose
// layer-parallel kernels finish a few rows sooner than one tensor-core tile
// pass over K x 3.
constexpr int kMinSplitRows = 256;

// Round counters of one step, device.
struct RoundCounters {
    int alive[2];              // alive list sizes (ping-pong)
    int n[LV_N][kMqPool];      // per level and group: list length
    int ticket[LV_N + 1];      // last-block detection of the classify (per input level) and survivors kernels
};

// Condition of a captured step's IF node: the handle (0: launched without a
// graph) and a device flag that records the value for the launch count.
// A kernel's last block sets the condition of the node that follows it.
struct Cond {
    unsigned long long h = 0;
    int *flag = nullptr;
};
constexpr int kMqMaxRounds = kMqSlots;
constexpr int kMqGates = 4 * kMqMaxRounds;   // per round: round, split, FP32 band, FP64 band

// Device tables and per-step buffers of a session.  A step holds up to K
// routing batches of each query: "virtual query" v = q * K + k is query q's
// k-th batch of the step; per-step arrays are indexed by v (Q of them),
// the query tables and histories by q = v / K.
struct MqDev {
    int Q, G, cap, dim;
    int K;                         // batches per query per step
    const StepHdr *hdr;
    int *off;                      // [Q+1] stacked offsets of the step
    unsigned short *qid;           // [cap] virtual query of each stacked tuple
    const unsigned char *np;       // [Q / K] predicates per query
    const unsigned char *udf;      // [Q / K][8] pool UDF of each slot
    const double *thr;             // [Q / K][8] thresholds
    const long long *cost;         // [Q / K][8] model cost of each slot's UDF
    unsigned char *order;          // [Q][8] slot order of each batch of the step
    unsigned char *evall;          // [Q] 1: warmup batch (every slot on every tuple)
    long long *bidx;               // [Q] the batch's number in its query (-1: no tuples)
    StatRow *rows;                 // [Q][8] step statistics per slot
    long long *npass;              // [Q]
    unsigned char *visited, *label, *ok;   // [cap] per tuple
    int *alive[2];                 // [cap]
    int *list[LV_N];               // per level [G][cap]: round queues (level 0) and band lists
    RoundCounters *rc;
    float *score[LV_F64];          // per level below FP64: [G][cap] scores of the level's lists
    const float *margin[LV_F64];   // per level below FP64: [G] margins (absolute score units)
    double *act64[2];              // FP64 band activations [cap64][max width]
    int cap64, ld64;               // FP64 band entries handled layer-parallel per round; row stride
    unsigned int *err;
    int *gates;                    // [kMqGates] condition values of the step (0 unless set)
    unsigned char *order_t;        // learned sessions: [cap][8] slot order of each tuple (else nullptr)
    unsigned lv1_skip;             // groups whose undecided level-0 entries go straight to the FP32 level
};

// Per-query statistics history (device).
struct MqHist {
    StatRow *ring;                 // [queries][R][8]
    int R;
    StatRow *warm;                 // [queries][warmup][8]
    int warmup, window;
    int lag;                       // batch b is routed on batches <= b - 1 - lag
    long long *bdone;              // [queries] batches completed
    int static_order;              // 1: every batch in declared slot order, no warmup batches
};

// One depth of the stacked grouped FP32 layers.  Group g's rows are
// [off_g, off_g + count_g) of the stacked buffers, off_g = sum of the earlier
// groups' counts.  in_rows (depth 0): queue list of the group (rows of X).
struct MqLayer {
    const float *W, *b;            // W == nullptr: group has no layer at this depth
    float bconst;                  // one-output last layer: its bias
    const float *in;               // stacked input (depth >= 1), row stride ldin
    int ldin;
    int K, N;
    int norelu;                    // 1: no ReLU (logits)
};
struct MqLayers {
    MqLayer l[kMqPool];
    int n;                         // groups
    const int *counts;             // [n] rows per group
    const int *rows;               // [n][cap] queue lists or nullptr (stacked input)
    int cap;
    const StepHdr *hdr;            // X of depth 0 (rows given) comes from the step header
    int ldx;
    float *Y;                      // stacked output, row stride ldy
    int ldy;
};

// h_round0: set to (step has tuples).
void mq_launch_init(const MqDev &d, cudaStream_t st, int sms, Cond round0 = Cond());
void mq_launch_router(const MqDev &d, const MqHist &h, cudaStream_t st);
void mq_launch_partition(const MqDev &d, int r, cudaStream_t st, int sms);
void mq_launch_layers_f32(const MqLayers &L, cudaStream_t st, int sms);
void mq_launch_dots_f32(const MqLayers &L, float *score, int sstride, cudaStream_t st, int sms);
// Decide the entries of level `in` with that level's scores and margins;
// undecided entries go to level `out`'s lists.
// next: set to (level `out` holds at least next_min entries).  With
// partials (tensor-core levels) the scores are summed from the GEMM's head
// partials (heads: per group bias and partials per row) in this kernel.
void mq_launch_classify(const MqDev &d, int r, int in, int out, cudaStream_t st, int sms, Cond next = Cond(),
                        int next_min = 1, const TcHeads *heads = nullptr, const float *partials = nullptr,
                        int pstride = 0);
// The FP64 level: every entry's UDF in FP64, its layers spread over all SMs
// (a warp per output neuron), the first cap64 entries of the round; the rest
// a block per entry.  Decides exactly.
void mq_launch_band64(const MqDev &d, int r, const GroupedMlps &mlps, int max_hidden, cudaStream_t st, int sms);
// The FP32 level of BF16 sessions, layer-parallel like the FP64 level, with
// its own test (margin_fp32; undecided entries go to the FP64 level, whose
// condition `next` it sets; act0/act1: [cap][ld] floats).
void mq_launch_band32(const MqDev &d, int r, const GroupedMlps &mlps, int max_hidden, float *act0, float *act1,
                      int ld, cudaStream_t st, int sms, Cond next = Cond());
// h_next_round: set to (the next alive list is not empty).
void mq_launch_survivors(const MqDev &d, int r, cudaStream_t st, int sms, Cond next_round = Cond());
void mq_launch_result(const MqDev &d, unsigned int *bitmap, cudaStream_t st, int sms);
void mq_launch_commit(const MqDev &d, const MqHist &h, StatRow *res_rows, unsigned char *res_order,
                      unsigned char *res_evall, long long *res_bidx, long long *res_npass, int *res_total,
                      int *res_gates, cudaStream_t st);
cudaError_t mq_band_smem_setup(int max_width);
// Learned sessions: each tuple's slot order.  Warmup batch: declared order;
// proxy trained (*ready): slots by c_i (1 + e^{z_i}) of the tuple's logits
// z (row stride ldz), ties to the lower slot; else the query's rank order.
void mq_launch_tuple_order(const MqDev &d, const float *logits, int ldz, const int *ready, cudaStream_t st, int sms);
// Learned sessions: proxy logits Z (row stride ldz) of the first *count rows
// from their BF16 hidden activations Hb [rows][H] (H % 8 == 0, P <= 8).
void mq_launch_proxy_out(const int *count, const __nv_bfloat16 *Hb, int H, const float *W2, const float *b2, int P,
                         float *Z, int ldz, int max_rows, cudaStream_t st, int sms);
// FP64 scores of one UDF on n rows of X (block per row), for calibration.
void mq_launch_scores_f64(const MlpDev &mlp, int max_width, const float *X, int ldx, int n, double *out,
                          cudaStream_t st, int sms);

}  // namespace hydro
