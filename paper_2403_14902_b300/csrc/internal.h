// Internal launch interface between the host runtime (hydro_api.cu) and the
// kernel files.  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hydro {

struct StatRow;

enum { PREC_F32 = 0, PREC_BF16 = 1, PREC_F64 = 2, PREC_TF32X3 = 3, PREC_BF16X3 = 4 };

constexpr int kMaxLayers = 16;

// Device view of an MLP UDF (fp32 weights as given: W[l] is [dims[l+1]][dims[l]]).
struct MlpDev {
    int n_layers;
    int max_width;
    int dims[kMaxLayers + 1];
    const float *W[kMaxLayers];
    const float *b[kMaxLayers];
    const float *WT[kMaxLayers];   // transposed weights [in][out] (sessions' band levels), else nullptr
};

// Router costs: c[i] is the per-tuple cost of predicate i (for a predicate
// on a shared embedding, its head's cost); group[i] >= 0 names the embedding
// whose per-batch misses add miss * cemb[group] (reuse-aware cost).
struct RouterCosts {
    long long c[8];
    int group[8];
    long long cemb[8];
    long long n;   // tuples in the batch
    int measured;  // 1: c_i = the window's stage time / tuples evaluated (ignores c, cemb)
};

// k_route.cu
void launch_init_alive(int *alive, int *count, int n, unsigned char *acc, cudaStream_t st);
void launch_classify_f32(const int *count_in, const int *alive_in, const float *scores, double t, double margin,
                         unsigned char *pass, int *band_m, int *band_tuple, int *band_count, int band_cap,
                         unsigned int *err, cudaStream_t st);
void launch_recheck_classify_f32(const int *band_count_in, const int *band_m_in, const int *band_tuple_in,
                                 const float *scores_r, double t, double margin_next, unsigned char *pass,
                                 int *next_m, int *next_tuple, int *next_count, int next_cap, unsigned int *err,
                                 cudaStream_t st);
void launch_recheck_classify_f64(const int *band_count_in, const int *band_m_in, const int *band_tuple_in,
                                 const double *scores_r, double t, unsigned char *pass, unsigned int *err,
                                 cudaStream_t st);
// Measured cost: stamp the stage's start (device global timer) into its row;
// the stage's compaction (measure = 1) turns it into the stage's duration.
void launch_stage_start(StatRow *row, cudaStream_t st);
// Copy the band's tuples into a fixed staging buffer (entry j -> slot j) and
// turn the band's tuple indices into staging slots.
void launch_band_stage(const int *band_count, int *band_tuple, const void *tuples, long long tuple_bytes,
                       void *staging, int max_entries, int sms, cudaStream_t st);
// Inside a captured graph: set a conditional IF node's handle to (*count > 0);
// zero the later band counts when it is off; count the body's kernels when on.
void launch_gate(const int *count, unsigned long long handle, int *zero0, int *zero1, unsigned long long *launch_ctr,
                 const int *body_kernels, cudaStream_t st);
void launch_compact(const int *count_in, const int *alive_in, const unsigned char *pass, int *alive_out,
                    int *count_out, unsigned char *acc, const int *bandt_count, const int *band32_count,
                    const int *band64_count, const int *miss_count, StatRow *row, StatRow *rrow, StatRow *warm,
                    cudaStream_t st, int measure = 0);

// Device-dispatched batches (a graph per stream lane): the switch handles of
// the positions, the batch size on the device, the first and last kernels
// and the copy of the batch's statistics rows into the ring.
struct SwitchHandles {
    unsigned long long h[8];
};
void launch_set_int(int *dst, int v, cudaStream_t st);
void launch_init_alive_dev(int *alive, int *count, const int *n_dev, int max_n, cudaStream_t st);
void launch_dispatch(const int *order, const SwitchHandles &h, int P, const int *body_n, unsigned long long *ctr,
                     int *order_out, cudaStream_t st);
void launch_result_dev(const int *count, const int *alive, const int *n_dev, unsigned int *bitmap, long long *n_pass,
                       cudaStream_t st);
void launch_commit_rows(const StatRow *src, StatRow *dst, int P, cudaStream_t st);

// k_cache.cu: reuse cache of a shared upstream UDF's outputs, keyed by tuple id.
// tags[id]: 0 absent, -1 prefilled, b+1 computed by batch b.
void launch_cache_probe_miss(const int *count_in, const int *list_in, const long long *ids, const int *tags,
                             long long cap, int *miss_list, int *miss_count, unsigned int *err, cudaStream_t st);
void launch_cache_store(const int *miss_count, const int *miss_list, const long long *ids, const float *src, int D,
                        float *values, int *tags, int tag_value, int max_rows, int sms, cudaStream_t st);
void launch_probe_visible(const long long *ids, int n, const int *tags, long long cap, long long last,
                          int *out_miss, cudaStream_t st);
void launch_acc_to_alive(const unsigned char *acc, int n, int *alive_out, int *count_out, cudaStream_t st);
void launch_result(const int *count, const int *alive, int n, unsigned int *bitmap, long long *n_pass,
                   cudaStream_t st);
void launch_router(const StatRow *ring, int ring_len, const StatRow *warm, int n_warm_visible, long long lo,
                   long long last, int P, int policy, const RouterCosts &costs, const int *vmiss, int *order_out,
                   cudaStream_t st);

// k_simt.cu
void launch_mlp_layer_f32(const int *count, const int *rows, const float *X, int ldx, const float *W,
                          const float *b, float *Y, int K, int N, int relu, int max_rows, int sms,
                          cudaStream_t st, const long long *ids = nullptr);
void launch_mlp_dot_f32(const int *count, const int *rows, const float *X, int ldx, const float *w, float bias,
                        int K, float *score, int max_rows, int sms, cudaStream_t st,
                        const long long *ids = nullptr);
void launch_mlp_band_f32(const int *band_count, const int *band_tuple, const float *X, int ldx,
                         const MlpDev &mlp, float *score_out, int sms, cudaStream_t st);
void launch_mlp_band_f64(const int *band_count, const int *band_tuple, const float *X, int ldx,
                         const MlpDev &mlp, double *score_out, int sms, cudaStream_t st);
cudaError_t mlp_band_smem_setup(int max_width);
// band: a recheck band of a few frames (one pixel per thread instead of four)
void launch_conv1(int prec, const int *count, const int *list, const unsigned char *frames, int C0, int H,
                  int Wd, const float *W, const float *bias, int Cout, void *out, int max_frames, int sms,
                  cudaStream_t st, bool band = false);
// First conv layer (FP32) in a split form [hi(Cout) | lo(Cout)] per pixel:
// TF32 planes in fp32 (3xTF32 level), or with bf16_planes BF16 planes
// (split-BF16 level).
void launch_conv1_split(const int *count, const int *list, const unsigned char *frames, int C0, int H, int Wd,
                        const float *W, const float *bias, int Cout, void *out, int max_frames, int sms,
                        cudaStream_t st, bool bf16_planes = false);
// Returns the number of kernels launched (2 for an FP32 / FP64 band with the K-split form: the
// FP32 form's nine and the FP64 form's three partial planes use the whole of `out`, up to
// max_frames frames, as scratch, behind its first max_frames / 10 (FP64: / 4) frames).
int launch_conv3x3_simt(int prec, const int *count, const void *in, int Cin, int H, int Wd, const void *Wt,
                        const float *bias, int Cout, void *out, int max_frames, int sms, cudaStream_t st,
                        bool band = false);
// Returns the number of kernels launched.  The FP32 / FP64 forms overwrite the first pixel of
// each of the frame's pixel ranges (16 ranges when H*W is a multiple of 512) in `act` with the
// range's channel sums.
int launch_pool_head(int prec, const int *count, void *act, int HW, int C, const float *hw, double hb,
                     void *score, int max_frames, int sms, cudaStream_t st);

// k_learned.cu: per-tuple routing by a learned proxy, grouped per-predicate queues
struct GroupLayer {
    const int *count;    // rows of this group (device)
    const int *rows;     // row indices into X (nullable: rows 0..count-1)
    const float *X;
    int ldx;
    const float *W;      // [N][K]
    const float *b;      // [N] (hidden layers)
    float bconst;        // bias of a one-output last layer
    float *Y;            // [rows][N] (hidden layers)
    int K, N, relu;
};
struct GroupedLayers {
    int n;
    GroupLayer l[8];
};
struct RoundTests {
    double t[8];
    double margin[8];
};
struct GroupedMlps {
    int max_width;
    MlpDev m[8];
};
struct ProxyTrain {
    int M, P, H, D, sms, t;
    float lr;
    const float *X;            // [M][D] minibatch features
    const float *Hact;         // [M][H] hidden activations (forward)
    const float *Z;            // [M][P] logits (forward)
    float *dZ, *dH, *inv_pairs;
    float *part;               // per-chunk gradient partials, proxy_grad_part_floats(M, D, H, P)
    const unsigned char *label, *mask;   // per tuple: pass bits / evaluated bits
    float *W1, *b1, *W2, *b2;
    float *gW1, *gb1, *gW2, *gb2;
    float *mW1, *vW1, *mb1, *vb1, *mW2, *vW2, *mb2, *vb2;
};
// Floats of the per-chunk gradient partials of one training step over M rows.
inline size_t proxy_grad_part_floats(int M, int D, int H, int P) {
    const size_t chunks = (size_t)(M + 255) / 256;
    const size_t a = (size_t)H * D + H, b = (size_t)P * H + P;
    return chunks * (a > b ? a : b);
}
void launch_tuple_order(int n, int P, const float *logits, int ldz, const RouterCosts &costs, const int *fallback,
                        unsigned char *order, int sms, cudaStream_t st);
void launch_partition(const int *count, const int *alive, const unsigned char *order, int r, int P, int *queues,
                      int qstride, int *qcount, cudaStream_t st);
void launch_grouped_layer_f32(const GroupedLayers &g, int max_tiles, int sms, cudaStream_t st);
void launch_grouped_dot_f32(const GroupedLayers &g, float *score, int sstride, int max_rows, int sms,
                            cudaStream_t st);
void launch_grouped_classify(int P, const int *qcount, const int *queues, int qstride, const float *score,
                             int sstride, const RoundTests &tests, unsigned char *ok, unsigned char *label,
                             unsigned char *visited, int *band_g, int *band_t, int *band_count, int band_cap,
                             StatRow *row, StatRow *rrow, unsigned int *err, cudaStream_t st);
void launch_grouped_band_f64(const int *band_count, const int *band_g, const int *band_t, const float *X, int ldx,
                             const GroupedMlps &mlps, const RoundTests &tests, unsigned char *ok,
                             unsigned char *label, StatRow *row, StatRow *rrow, int sms, cudaStream_t st);
cudaError_t grouped_band_smem_setup(int max_width);
void launch_survivors(const int *count_in, const int *alive_in, const unsigned char *ok, int *alive_out,
                      int *count_out, cudaStream_t st);
void launch_zero_rows(StatRow *row, StatRow *rrow, int P, unsigned char *visited, unsigned char *label, int n,
                      cudaStream_t st);
void launch_full_label_acc(const unsigned char *label, int n, int P, unsigned char *acc, cudaStream_t st);
void launch_proxy_train_step(const ProxyTrain &pt, cudaStream_t st);

// hydro_api.cu: message returned by hydro_last_error() on this thread
void set_last_error(const char *msg);

// k_util.cu
void launch_f32_to_f64(const float *src, double *dst, int n, cudaStream_t st);
void launch_identity_list(int *list, int *count, int start, int n, cudaStream_t st);

}  // namespace hydro
