// Device side of multi-query sessions: one step = every query's next chunk
// of tuples, stacked query after query, routed per query and evaluated in
// rounds of grouped launches (one group per pool UDF).
#pragma once

#include <cuda_runtime.h>

#include "../../include/hydro.h"
#include "common.cuh"
#include "internal.h"

namespace hydro {

constexpr int kMqMaxQ = HYDRO_MAX_QUERIES;
constexpr int kMqPool = HYDRO_MAX_POOL;
constexpr int kMqSlots = HYDRO_MAX_PREDICATES;

// What the host sends per step (one H2D copy from pinned memory).
struct StepHdr {
    const float *X;            // stacked fp32 rows of the step
    int counts[kMqMaxQ];       // rows per query
};

// Round counters of one step, device.
struct RoundCounters {
    int alive[2];              // alive list sizes (ping-pong)
    int q[kMqPool];            // per group: queue length of the round
    int b32[kMqPool];          // per group: FP32 band (BF16 sessions)
    int b64[kMqPool];          // per group: FP64 band
};

// Device tables and per-step buffers of a session.
struct MqDev {
    int Q, G, cap, dim;
    const StepHdr *hdr;
    int *off;                      // [Q+1] stacked offsets of the step
    unsigned char *qid;            // [cap] query of each stacked tuple
    const unsigned char *np;       // [Q] predicates per query
    const unsigned char *udf;      // [Q][8] pool UDF of each slot
    const double *thr;             // [Q][8] thresholds
    const long long *cost;         // [Q][8] model cost of each slot's UDF
    unsigned char *order;          // [Q][8] slot order of the step
    unsigned char *evall;          // [Q] 1: warmup batch (every slot on every tuple)
    long long *bidx;               // [Q] the query's batch number this step (-1: no tuples)
    StatRow *rows;                 // [Q][8] step statistics per slot
    long long *npass;              // [Q]
    unsigned char *visited, *label, *ok;   // [cap] per tuple
    int *alive[2];                 // [cap]
    int *queues;                   // [G][cap] round queues
    int *bq32, *bq64;              // [G][cap] band queues
    RoundCounters *rc;
    float *score;                  // [G][cap] working-precision scores of the round's queues
    float *rscore;                 // [G][cap] FP32 scores of the FP32 band
    const float *margin_lowp;      // [G]
    const float *margin_fp32;      // [G]
    unsigned int *err;
};

// Per-query statistics history (device).
struct MqHist {
    StatRow *ring;                 // [Q][R][8]
    int R;
    StatRow *warm;                 // [Q][warmup][8]
    int warmup, window;
    long long *bdone;              // [Q] batches completed
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

void mq_launch_init(const MqDev &d, cudaStream_t st, int sms);
void mq_launch_router(const MqDev &d, const MqHist &h, cudaStream_t st);
void mq_launch_partition(const MqDev &d, int r, cudaStream_t st, int sms);
void mq_launch_layers_f32(const MqLayers &L, cudaStream_t st, int sms);
void mq_launch_dots_f32(const MqLayers &L, float *score, int sstride, cudaStream_t st, int sms);
// level 0: score of the round queues vs margin_lowp (BF16) or margin_fp32 (FP32
// sessions); level 1: FP32 band scores vs margin_fp32.
void mq_launch_classify(const MqDev &d, int r, int level, bool bf16, cudaStream_t st, int sms);
void mq_launch_band64(const MqDev &d, int r, const GroupedMlps &mlps, cudaStream_t st, int sms);
void mq_launch_survivors(const MqDev &d, int r, cudaStream_t st, int sms);
void mq_launch_result(const MqDev &d, unsigned int *bitmap, cudaStream_t st, int sms);
void mq_launch_commit(const MqDev &d, const MqHist &h, StatRow *res_rows, unsigned char *res_order,
                      unsigned char *res_evall, long long *res_bidx, long long *res_npass, int *res_total,
                      cudaStream_t st);
cudaError_t mq_band_smem_setup(int max_width);
// FP64 scores of one UDF on n rows of X (block per row), for calibration.
void mq_launch_scores_f64(const MlpDev &mlp, int max_width, const float *X, int ldx, int n, double *out,
                          cudaStream_t st, int sms);

}  // namespace hydro
