// Host runtime behind include/hydro.h: query state, device buffers, the
// per-batch stage sequence (Eddy routing of a batch through its predicates,
// Sec. 3.2), result slots and polling.
//
// One query drives one CUDA stream.  A batch's stages are enqueued in the
// order the router picked; counts of surviving tuples stay on the device.
// The router itself runs on a second stream: for batch b it waits for batch
// b-1-lag to finish, computes the order on the device from the statistics
// ring, and copies the P order bytes back; the host launches batch b's
// stages once that small copy lands (Sec. 3.3 "Metadata for Data Routing":
// statistics of completed batches decide the next routing).
#include <algorithm>
#include <cstdarg>
#include <random>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include <cuda.h>

#include "../../include/hydro.h"
#include "common.cuh"
#include "internal.h"
#include "tc_conv.h"
#include "tc_gemm.h"

using namespace hydro;

namespace {

thread_local std::string g_err;

hydro_status fail(hydro_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define CU(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(e_ == cudaErrorMemoryAllocation ? HYDRO_ENOMEM : HYDRO_ECUDA, "%s: %s", \
                        #call, cudaGetErrorString(e_));                                       \
    } while (0)

constexpr int kEvRing = 16;

// A shared upstream UDF whose outputs are cached per tuple id.
struct Emb {
    int n_layers = 0;
    std::vector<int> dims;
    std::vector<std::vector<float>> W, b;
    long long cap = 0;     // ids in [0, cap)
    long long cost = 1;    // flops per tuple
    std::vector<float *> dW, db;
    float *values = nullptr;   // [cap][dims.back()]
    int *tags = nullptr;       // [cap]: 0 absent, -1 prefilled, b+1 computed by batch b
};

struct Pred {
    int kind = 0;
    int n_layers = 0;
    int upstream = 0;      // 0, or 1-based embedding id; layers [0, head_start) are the embedding's
    int head_start = 0;
    std::vector<int> dims;
    std::vector<std::vector<float>> W, b;
    std::vector<float> head_w;
    double head_b = 0.0;
    double threshold = 0.0;
    double margin_lowp = 0.02;
    double margin_tf32 = -1.0;   // < 0: not set, default at finalize
    double margin_fp32 = -1.0;
    long long cost = 1;
    // device copies
    std::vector<float *> dW, db;          // as given
    std::vector<float *> dWt32;           // CNN layer l >= 1: [tap][ci][co] fp32
    std::vector<__nv_bfloat16 *> dWt16;   // CNN layer l >= 1: [tap][ci][co] bf16
    std::vector<void *> dWtc;             // CNN layer l >= 1: tensor-core layout (bf16)
    std::vector<void *> dWts;             // CNN layer l >= 1: tensor-core split-TF32 layout (fp32 hi, lo)
    std::vector<void *> dWbs;             // CNN layer l >= 1: tensor-core split-BF16 layout (bf16 hi, lo)
    bool tc_all = false;                  // every layer l >= 1 has tensor-core weights
    bool tc_conv1 = false;                // CNN, BF16: the first layer runs on the tensor cores
    __half *dWc1 = nullptr;               //   with this packed FP16 weight tile (bias folded in)
    std::vector<__nv_bfloat16 *> dW16;    // MLP hidden layers: bf16 weights for the tensor cores
    bool tc_mlp = false;                  // MLP: every hidden layer runs on the tensor cores
    float *dHead = nullptr;
    MlpDev mlp{};
};

struct Slot {
    long long batch = -1;
    int n = 0;
    bool busy = false;
    bool warmup = false;
    int order[kMaxPred] = {};
    cudaEvent_t start = nullptr, done = nullptr;
    unsigned char *dres = nullptr;   // device result block
    unsigned char *hres = nullptr;   // pinned host mirror
    bool dev = false;                // routed and dispatched on the device (order in the result header)
};

// Result block layout (device and pinned host).
struct ResHdr {
    long long n_pass;
    unsigned int err;
    unsigned int pad0;
    int order[8];        // device-dispatched batches: the order the router chose
    unsigned int pad[4];
};
static_assert(sizeof(ResHdr) == 64, "header size");
constexpr size_t kRowsOff = sizeof(ResHdr);
constexpr size_t kBitmapOff = kRowsOff + sizeof(StatRow) * kMaxPred;

// Profiling: one record per timed launch; its item count is resolved from
// the batch's statistics row when the batch is polled.
enum ProfSrc { SRC_MAIN = 0, SRC_R32 = 1, SRC_R64 = 2, SRC_RTF = 3, SRC_MISS = 4 };
struct ProfCtx {
    long long batch;
    int pred;
    int src;
};
struct ProfRec {
    int cls;
    int ev;               // events ev, ev+1 in the pool
    long long batch;
    int pred, src;
    double fpi, bpi;      // flops / bytes per item
    double fixed_bytes;   // per launch (weights)
};
const char *const kProfNames[] = {"conv3x3_bf16_tc", "conv3x3_bf16_simt", "conv3x3_f32_simt", "conv3x3_f64_simt",
                                  "conv1_u8",        "pool_head",         "mlp_layer_f32",    "mlp_dot_f32",
                                  "mlp_band_f32",    "mlp_band_f64",      "conv3x3_split_tc",  "mlp_layer_bf16_tc",
                                  "gather_rows_bf16"};
enum { PC_CONV_TC = 0, PC_CONV_BF16, PC_CONV_F32, PC_CONV_F64, PC_CONV1, PC_POOL, PC_MLP, PC_DOT, PC_BAND32,
       PC_BAND64, PC_CONV_TF32, PC_MLP_TC, PC_GATHER, PC_N };

struct Prof {
    bool on = false;
    std::vector<cudaEvent_t> ev;
    std::vector<ProfRec> recs;
    std::vector<std::vector<StatRow>> rows;   // per polled batch (index batch - base)
    long long base = 0;
};

}  // namespace

constexpr int kMaxLanes = 8;

// Per-batch scratch of one stream lane.
struct LaneBufs {
    int *alive[2] = {};
    int *ints = nullptr;
    unsigned char *pass = nullptr, *acc = nullptr;
    float *score32 = nullptr;
    int *band1_m = nullptr, *band1_t = nullptr, *band2_m = nullptr, *band2_t = nullptr;
    int *band3_m = nullptr, *band3_t = nullptr;
    float *rscore_t = nullptr, *rscore32 = nullptr;
    double *rscore64 = nullptr;
    void *act[2] = {}, *ract32[2] = {}, *ract64[2] = {};
    float *partials = nullptr;
    __nv_bfloat16 *stage16 = nullptr, *act16[2] = {};
    void *band_rows = nullptr;
    void *batch_rows = nullptr;       // device dispatch: the batch's tuples
    unsigned char *lres = nullptr;    // device dispatch: the batch's result block
    int *lord = nullptr, *ln = nullptr;   // device dispatch: router order, batch size
    int *miss_list = nullptr;             // stage probe of a cached embedding
};

struct hydro_query {
    hydro_query_config cfg{};
    std::vector<Pred> preds;
    std::vector<Emb> embs;
    std::vector<int> static_order;
    int *vmiss = nullptr;         // router probe: misses per embedding for the batch being routed
    // learned per-tuple routing (HYDRO_POLICY_LEARNED)
    unsigned char *order_t = nullptr;   // [B][8] per-tuple predicate order
    unsigned char *okf = nullptr, *label = nullptr, *visited = nullptr;   // [B] per tuple
    int *queues = nullptr, *qcount = nullptr;   // [8][B], [8]
    float *qscore = nullptr;                    // [8][B]
    int *bandg = nullptr, *bandt = nullptr;     // [B]
    std::vector<float *> gact;                  // per predicate, two [B][width] buffers
    int *d_fallback = nullptr, *h_fallback = nullptr;
    GroupedMlps gmlps{};
    int ph = 64;
    float *pW1 = nullptr, *pb1 = nullptr, *pW2 = nullptr, *pb2 = nullptr;
    float *pg = nullptr, *pm = nullptr, *pv = nullptr;   // gradients and Adam moments, same layout as params
    float *pH = nullptr, *pZ = nullptr, *pdZ = nullptr, *pdH = nullptr, *pinv = nullptr, *ppart = nullptr;
    float *ringX = nullptr;
    unsigned char *ringL = nullptr, *ringM = nullptr;
    std::vector<int> ring_n;
    bool proxy_ready = false;
    int adam_t = 0;
    long long last_learned_batch = -1;
    int last_n = 0;
    int *miss_list = nullptr;     // stage probe: alive tuples whose embedding is not cached
    bool finalized = false;
    bool dead = false;
    int sms = 148;
    cudaStream_t st = nullptr, rst = nullptr;
    bool own_stream = false;
    std::vector<void *> allocs;   // device allocations to free
    // scratch
    int *alive[2] = {};
    int *ints = nullptr;          // [0],[1]: alive counts; [2],[3],[4]: band 1, 2, 3 counts
    unsigned char *pass = nullptr, *acc = nullptr;
    float *score32 = nullptr;
    // recheck bands: entries (position in the stage, tuple in the batch)
    int *band1_m = nullptr, *band1_t = nullptr, *band2_m = nullptr, *band2_t = nullptr;
    int *band3_m = nullptr, *band3_t = nullptr;
    int cap1 = 0, cap2 = 0, cap3 = 0;   // band capacities (entries / frames)
    int ract_esz = 8;                   // bytes a channel of the CNN recheck activations
    float *rscore_t = nullptr;    // 3xTF32 recheck scores (band 1)
    float *rscore32 = nullptr;    // FP32 recheck scores
    double *rscore64 = nullptr;   // FP64 recheck scores
    void *act[2] = {};            // working precision activations
    void *ract32[2] = {};         // CNN FP32 recheck activations
    void *ract64[2] = {};         // CNN FP64 recheck activations
    float *partials = nullptr;    // BF16: fused (pool+)head partials [max_batch][tiles]
    __nv_bfloat16 *stage16 = nullptr;   // BF16 MLP: gathered first-layer operand [max_batch][dim]
    __nv_bfloat16 *act16[2] = {};       // BF16 MLP: hidden activations
    void *gemm_encode = nullptr;
    StatRow *ring = nullptr, *warm = nullptr;
    int ring_len = 0;
    int *d_order = nullptr;       // [max_in_flight][8]
    int *h_order = nullptr;       // pinned mirror
    unsigned int *d_err = nullptr;
    cudaEvent_t ev_done[kEvRing] = {};
    cudaEvent_t ev_route = nullptr;
    std::vector<Slot> slots;
    size_t res_bytes = 0;
    long long next_batch = 0;
    unsigned int latched_err = 0;
    // cumulative statistics (updated at poll)
    long long tot[kMaxPred][6] = {};
    // tensor-core conv
    TcConvPlan tc{};
    // profiling and launch count
    Prof prof;
    long long launches = 0;
    // stream lanes: batch b runs on lane b % n_lanes, each with its own scratch and stream
    int n_lanes = 1;
    LaneBufs lanes[kMaxLanes];
    cudaStream_t lane_st[kMaxLanes] = {};
    bool own_lane_st[kMaxLanes] = {};
    cudaEvent_t ev_user = nullptr;   // input-ready point on the caller's stream (the batch's lane waits on it)
    cudaStream_t home_st = nullptr;  // with two lanes: the caller's (or the library's) stream
    int cur_lane = 0;
    // recheck graphs: the recheck levels of predicate p on lane l replay from tail[l][p]
    void *band_rows = nullptr;       // current lane's staging buffer of the band's tuples [cap1][tuple bytes]
    // device-dispatched batches: each lane's batch graph (a SWITCH per position)
    void *batch_rows = nullptr;
    unsigned char *lres = nullptr;
    int *lord = nullptr, *ln = nullptr;
    cudaGraphExec_t bgraph[kMaxLanes] = {};
    int *d_switch_n = nullptr;       // [kMaxLanes][8 positions][8 predicates] kernels per switch body
    cudaGraphExec_t tail[kMaxLanes][kMaxPred] = {};
    int tail_gates[kMaxLanes][kMaxPred] = {};
    int *d_body_n = nullptr;         // [kMaxLanes][kMaxPred][3] kernels per conditional body
    unsigned long long *d_launch_ctr = nullptr;   // kernels the conditional bodies ran
    cudaStream_t cap_st = nullptr;
    cudaStream_t cap_help[3] = {};   // capture streams of nested conditional bodies
    int cap_depth = 0;
    bool capturing = false;
    cudaGraph_t cap_graph = nullptr;
    std::vector<std::pair<int *, int>> cap_body_counts;   // (device slot, kernels) of the bodies just captured
    // pipeline: order position k runs on pos_st[k] with sms_pos SMs; ev_stage[l][k] closes
    // position k of the batch on lane l
    bool pipe = false;
    int sms_full = 0, sms_pos = 0;
    cudaStream_t pos_st[kMaxPred] = {};
    cudaEvent_t ev_stage[kMaxLanes][kMaxPred] = {};
    CUgreenCtx gctx[kMaxPred] = {};   // pipeline 2: one SM partition per position
};

namespace {

int tuple_bytes(const hydro_query_config &c) {
    return c.tuple_kind == HYDRO_TUPLE_F32 ? c.dim * 4 : c.channels * c.height * c.width;
}

template <typename T>
hydro_status dalloc(hydro_query *q, T **p, size_t bytes) {
    void *v = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&v, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(HYDRO_ENOMEM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    q->allocs.push_back(v);
    *p = (T *)v;
    return HYDRO_OK;
}

#define TRY(x)                         \
    do {                               \
        hydro_status s_ = (x);         \
        if (s_ != HYDRO_OK) return s_; \
    } while (0)

template <typename T>
hydro_status upload(hydro_query *q, T **dst, const T *src, size_t count) {
    TRY(dalloc(q, dst, count * sizeof(T)));
    CU(cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice));
    return HYDRO_OK;
}

long long model_cost(const Pred &p, const hydro_query_config &c) {
    long long f = 0;
    if (p.kind == HYDRO_UDF_MLP) {
        for (int l = 0; l < p.n_layers; ++l) f += 2LL * p.dims[l] * p.dims[l + 1];
    } else {
        const long long hw = (long long)c.height * c.width;
        for (int l = 0; l < p.n_layers; ++l) f += 2LL * hw * 9 * p.dims[l] * p.dims[l + 1];
        f += 2LL * p.dims[p.n_layers];
    }
    return f;
}

// Tensor-core query: BF16 working precision, or split BF16 as the working
// precision of a frame query (FP32-class scores on the tensor cores).  Both
// prepare the same tensor-core weights and buffers.
bool tc_query(const hydro_query_config &c) {
    return c.precision == HYDRO_PREC_BF16 || c.precision == HYDRO_PREC_BF16X3;
}

bool adaptive(int policy);

// Routed batches of this query can run from a per-lane graph whose SWITCH
// nodes take the order the router writes on the device (no host round trip).
bool device_dispatch(const hydro_query *q) {
    const hydro_query_config &c = q->cfg;
    return c.recheck_graphs && !c.pipeline && q->embs.empty() &&
           (c.policy == HYDRO_POLICY_RANK || c.policy == HYDRO_POLICY_COST || c.policy == HYDRO_POLICY_SELECTIVITY);
}

bool adaptive(int policy) {
    return policy == HYDRO_POLICY_RANK || policy == HYDRO_POLICY_COST || policy == HYDRO_POLICY_SELECTIVITY ||
           policy == HYDRO_POLICY_LEARNED;
}

int max_width(const hydro_query *q) {
    int w = 1;
    for (const Pred &p : q->preds)
        for (int d : p.dims) w = std::max(w, d);
    return w;
}

hydro_status finalize_learned(hydro_query *q) {
    const hydro_query_config &c = q->cfg;
    const int B = c.max_batch, P = (int)q->preds.size(), D = c.dim;
    for (const Pred &p : q->preds)
        if (p.kind != HYDRO_UDF_MLP || p.upstream)
            return fail(HYDRO_EUNSUPPORTED, "the learned router takes MLP predicates on the tuple");
    TRY(dalloc(q, &q->order_t, (size_t)B * kMaxPred));
    TRY(dalloc(q, &q->okf, B));
    TRY(dalloc(q, &q->label, B));
    TRY(dalloc(q, &q->visited, B));
    TRY(dalloc(q, &q->queues, sizeof(int) * kMaxPred * B));
    TRY(dalloc(q, &q->qcount, sizeof(int) * kMaxPred));
    TRY(dalloc(q, &q->qscore, sizeof(float) * kMaxPred * B));
    TRY(dalloc(q, &q->bandg, sizeof(int) * B));
    TRY(dalloc(q, &q->bandt, sizeof(int) * B));
    TRY(dalloc(q, &q->d_fallback, sizeof(int) * kMaxPred));
    CU(cudaMallocHost(&q->h_fallback, sizeof(int) * kMaxPred));
    q->gact.assign(2 * P, nullptr);
    int wmax = 1;
    for (int i = 0; i < P; ++i) {
        int w = 1;
        for (int d : q->preds[i].dims) w = std::max(w, d);
        wmax = std::max(wmax, w);
        for (int k = 0; k < 2; ++k) TRY(dalloc(q, &q->gact[2 * i + k], sizeof(float) * (size_t)B * w));
        q->gmlps.m[i] = q->preds[i].mlp;
    }
    q->gmlps.max_width = wmax;
    CU(grouped_band_smem_setup(wmax));
    // proxy MLP D -> H -> P (ReLU, then logits), seeded uniform init
    const int H = q->ph = c.proxy_hidden > 0 ? c.proxy_hidden : 64;
    const size_t nparam = (size_t)H * D + H + (size_t)P * H + P;
    std::vector<float> init(nparam, 0.f);
    std::mt19937 gen((unsigned)c.proxy_seed);
    std::uniform_real_distribution<float> u1(-std::sqrt(6.f / D), std::sqrt(6.f / D));
    std::uniform_real_distribution<float> u2(-1.f / std::sqrt((float)H), 1.f / std::sqrt((float)H));
    for (size_t k = 0; k < (size_t)H * D; ++k) init[k] = u1(gen);
    for (size_t k = 0; k < (size_t)P * H; ++k) init[(size_t)H * D + H + k] = u2(gen);
    float *params = nullptr;
    TRY(dalloc(q, &params, sizeof(float) * nparam));
    CU(cudaMemcpy(params, init.data(), sizeof(float) * nparam, cudaMemcpyHostToDevice));
    q->pW1 = params;
    q->pb1 = q->pW1 + (size_t)H * D;
    q->pW2 = q->pb1 + H;
    q->pb2 = q->pW2 + (size_t)P * H;
    TRY(dalloc(q, &q->pg, sizeof(float) * nparam));
    TRY(dalloc(q, &q->pm, sizeof(float) * nparam));
    TRY(dalloc(q, &q->pv, sizeof(float) * nparam));
    CU(cudaMemset(q->pm, 0, sizeof(float) * nparam));
    CU(cudaMemset(q->pv, 0, sizeof(float) * nparam));
    TRY(dalloc(q, &q->pH, sizeof(float) * (size_t)B * H));
    TRY(dalloc(q, &q->pZ, sizeof(float) * (size_t)B * kMaxPred));
    TRY(dalloc(q, &q->pdZ, sizeof(float) * (size_t)B * kMaxPred));
    TRY(dalloc(q, &q->pdH, sizeof(float) * (size_t)B * H));
    TRY(dalloc(q, &q->ppart, sizeof(float) * proxy_grad_part_floats(B, D, H, P)));
    TRY(dalloc(q, &q->pinv, sizeof(float)));
    const int R = std::max(1, c.proxy_refresh);
    TRY(dalloc(q, &q->ringX, sizeof(float) * (size_t)R * B * D));
    TRY(dalloc(q, &q->ringL, (size_t)R * B));
    TRY(dalloc(q, &q->ringM, (size_t)R * B));
    q->ring_n.assign(R, 0);
    return HYDRO_OK;
}

// Per-batch scratch buffers of the current lane (the q-> fields).
hydro_status alloc_scratch(hydro_query *q) {
    const hydro_query_config &c = q->cfg;
    const int B = c.max_batch;
    const bool cnn = c.tuple_kind == HYDRO_TUPLE_U8_FRAME;
    const int wmax = max_width(q);
    TRY(dalloc(q, &q->alive[0], sizeof(int) * B));
    TRY(dalloc(q, &q->alive[1], sizeof(int) * B));
    TRY(dalloc(q, &q->ints, sizeof(int) * 16));
    if (!q->embs.empty()) TRY(dalloc(q, &q->miss_list, sizeof(int) * B));
    TRY(dalloc(q, &q->pass, B));
    TRY(dalloc(q, &q->acc, B));
    TRY(dalloc(q, &q->score32, sizeof(float) * B));
    // band capacities: the FP64 level of CNN UDFs is capped at 64 frames per
    // stage (ERR_BAND_OVERFLOW beyond), every other level holds a full batch
    q->cap1 = B;
    q->cap2 = B;
    q->cap3 = cnn ? std::min(B, 64) : B;
    TRY(dalloc(q, &q->band1_m, sizeof(int) * q->cap1));
    TRY(dalloc(q, &q->band1_t, sizeof(int) * q->cap1));
    TRY(dalloc(q, &q->band2_m, sizeof(int) * q->cap2));
    TRY(dalloc(q, &q->band2_t, sizeof(int) * q->cap2));
    TRY(dalloc(q, &q->band3_m, sizeof(int) * q->cap3));
    TRY(dalloc(q, &q->band3_t, sizeof(int) * q->cap3));
    TRY(dalloc(q, &q->rscore_t, sizeof(float) * q->cap1));
    TRY(dalloc(q, &q->rscore32, sizeof(float) * std::max(q->cap1, q->cap2)));
    TRY(dalloc(q, &q->rscore64, sizeof(double) * std::max(q->cap1, q->cap3)));
    if (cnn) {
        const size_t px = (size_t)c.height * c.width * wmax;
        // BF16 activations, or [hi | lo] BF16 planes (split working precision) / FP32
        const size_t esz = c.precision == HYDRO_PREC_BF16 ? 2 : 4;
        for (int k = 0; k < 2; ++k) TRY(dalloc(q, &q->act[k], esz * px * B));
        // recheck levels: split BF16 ([hi | lo] bf16, 4 B a channel) and FP32 (4 B); 3xTF32 as the
        // configured split level needs two fp32 planes (8 B)
        q->ract_esz = (c.precision == HYDRO_PREC_BF16 && c.split_precision == HYDRO_PREC_TF32X3) ? 8 : 4;
        if (tc_query(c))
            for (int k = 0; k < 2; ++k)
                TRY(dalloc(q, &q->ract32[k], (size_t)q->ract_esz * px * std::max(q->cap1, q->cap2)));
        for (int k = 0; k < 2; ++k) TRY(dalloc(q, &q->ract64[k], 8 * px * q->cap3));
        if (tc_query(c))
            TRY(dalloc(q, &q->partials, sizeof(float) * (size_t)B * tc_conv_max_head_parts(c.height, c.width)));
    } else {
        for (int k = 0; k < 2; ++k) TRY(dalloc(q, &q->act[k], sizeof(float) * (size_t)wmax * B));
        CU(mlp_band_smem_setup(wmax));
        if (c.precision == HYDRO_PREC_BF16) {
            TRY(dalloc(q, &q->stage16, sizeof(__nv_bfloat16) * (size_t)B * c.dim));
            for (int k = 0; k < 2; ++k) TRY(dalloc(q, &q->act16[k], sizeof(__nv_bfloat16) * (size_t)wmax * B));
            TRY(dalloc(q, &q->partials, sizeof(float) * (size_t)B * 2 * std::max(1, wmax / 64)));
            hydro_status s = tc_gemm_init(&q->gemm_encode);
            if (s != HYDRO_OK) return fail(s, "tensor-core GEMM init failed: %s", tc_gemm_last_error());
        }
    }
    if (c.recheck_graphs) TRY(dalloc(q, (unsigned char **)&q->band_rows, (size_t)q->cap1 * tuple_bytes(c)));
    if (device_dispatch(q)) {
        TRY(dalloc(q, (unsigned char **)&q->batch_rows, (size_t)B * tuple_bytes(c)));
        TRY(dalloc(q, &q->lres, kBitmapOff + sizeof(unsigned int) * (size_t)((B + 31) / 32)));
        TRY(dalloc(q, &q->lord, sizeof(int) * kMaxPred));
        TRY(dalloc(q, &q->ln, sizeof(int)));
        CU(cudaMemset(q->lord, 0, sizeof(int) * kMaxPred));
        CU(cudaMemset(q->ln, 0, sizeof(int)));
    }
    return HYDRO_OK;
}

void save_lane(hydro_query *q, int l) {
    LaneBufs &L = q->lanes[l];
    for (int k = 0; k < 2; ++k) {
        L.alive[k] = q->alive[k];
        L.act[k] = q->act[k];
        L.ract32[k] = q->ract32[k];
        L.ract64[k] = q->ract64[k];
        L.act16[k] = q->act16[k];
    }
    L.ints = q->ints;
    L.pass = q->pass;
    L.acc = q->acc;
    L.score32 = q->score32;
    L.band1_m = q->band1_m;
    L.band1_t = q->band1_t;
    L.band2_m = q->band2_m;
    L.band2_t = q->band2_t;
    L.band3_m = q->band3_m;
    L.band3_t = q->band3_t;
    L.rscore_t = q->rscore_t;
    L.rscore32 = q->rscore32;
    L.rscore64 = q->rscore64;
    L.partials = q->partials;
    L.stage16 = q->stage16;
    L.band_rows = q->band_rows;
    L.batch_rows = q->batch_rows;
    L.lres = q->lres;
    L.lord = q->lord;
    L.ln = q->ln;
    L.miss_list = q->miss_list;
}

// Make lane l current: its scratch and its stream.
void load_lane(hydro_query *q, int l) {
    const LaneBufs &L = q->lanes[l];
    for (int k = 0; k < 2; ++k) {
        q->alive[k] = L.alive[k];
        q->act[k] = L.act[k];
        q->ract32[k] = L.ract32[k];
        q->ract64[k] = L.ract64[k];
        q->act16[k] = L.act16[k];
    }
    q->ints = L.ints;
    q->pass = L.pass;
    q->acc = L.acc;
    q->score32 = L.score32;
    q->band1_m = L.band1_m;
    q->band1_t = L.band1_t;
    q->band2_m = L.band2_m;
    q->band2_t = L.band2_t;
    q->band3_m = L.band3_m;
    q->band3_t = L.band3_t;
    q->rscore_t = L.rscore_t;
    q->rscore32 = L.rscore32;
    q->rscore64 = L.rscore64;
    q->partials = L.partials;
    q->stage16 = L.stage16;
    q->band_rows = L.band_rows;
    q->batch_rows = L.batch_rows;
    q->lres = L.lres;
    q->lord = L.lord;
    q->ln = L.ln;
    q->miss_list = L.miss_list;
    q->st = q->lane_st[l];
    q->cur_lane = l;
}

// Every lane's work done; lane 0 current (calls that use the scratch outside batches).
hydro_status quiesce(hydro_query *q) {
    for (int l = 0; l < q->n_lanes; ++l)
        if (q->lane_st[l]) CU(cudaStreamSynchronize(q->lane_st[l]));
    for (int k = 0; k < kMaxPred; ++k)
        if (q->pos_st[k]) CU(cudaStreamSynchronize(q->pos_st[k]));
    if (q->n_lanes > 1) load_lane(q, 0);
    return HYDRO_OK;
}

// Driver entry points for SM partitions (green contexts), looked up through
// the runtime so that the library needs no link-time libcuda.
struct GreenApi {
    CUresult (*get_resource)(CUdevice, CUdevResource *, CUdevResourceType) = nullptr;
    CUresult (*split)(CUdevResource *, unsigned int *, const CUdevResource *, CUdevResource *, unsigned int,
                      unsigned int) = nullptr;
    CUresult (*gen_desc)(CUdevResourceDesc *, CUdevResource *, unsigned int) = nullptr;
    CUresult (*create)(CUgreenCtx *, CUdevResourceDesc, CUdevice, unsigned int) = nullptr;
    CUresult (*stream_create)(CUstream *, CUgreenCtx, unsigned int, int) = nullptr;
    CUresult (*destroy)(CUgreenCtx) = nullptr;
    CUresult (*stream_destroy)(CUstream) = nullptr;
};

bool green_api(GreenApi *g) {
    auto get = [](const char *name, void **fn) {
        cudaDriverEntryPointQueryResult qr;
        return cudaGetDriverEntryPointByVersion(name, fn, CUDA_VERSION, cudaEnableDefault, &qr) == cudaSuccess &&
               qr == cudaDriverEntryPointSuccess && *fn;
    };
    return get("cuDeviceGetDevResource", (void **)&g->get_resource) &&
           get("cuDevSmResourceSplitByCount", (void **)&g->split) &&
           get("cuDevResourceGenerateDesc", (void **)&g->gen_desc) && get("cuGreenCtxCreate", (void **)&g->create) &&
           get("cuGreenCtxStreamCreate", (void **)&g->stream_create) &&
           get("cuGreenCtxDestroy", (void **)&g->destroy) && get("cuStreamDestroy", (void **)&g->stream_destroy);
}

// Pipeline 2: split the device's SMs into P equal partitions (multiples of
// 8 SMs, the split granularity) and give position k a stream of partition k.
hydro_status make_partitions(hydro_query *q, int P) {
    GreenApi g;
    if (!green_api(&g)) return fail(HYDRO_EUNSUPPORTED, "SM partitions (green contexts) are not available");
    CUdevice dev = q->cfg.device;
    CUdevResource all{};
    if (g.get_resource(dev, &all, CU_DEV_RESOURCE_TYPE_SM) != CUDA_SUCCESS)
        return fail(HYDRO_ECUDA, "cuDeviceGetDevResource failed");
    const unsigned per = all.sm.smCount / (unsigned)P / 8u * 8u;
    if (per < 8) return fail(HYDRO_EUNSUPPORTED, "too few SMs for %d partitions", P);
    CUdevResource parts[kMaxPred], rest{};
    unsigned ng = (unsigned)P;
    if (g.split(parts, &ng, &all, &rest, 0, per) != CUDA_SUCCESS || ng < (unsigned)P)
        return fail(HYDRO_ECUDA, "cuDevSmResourceSplitByCount failed");
    int smin = 1 << 30;
    for (int k = 0; k < P; ++k) {
        CUdevResourceDesc desc;
        if (g.gen_desc(&desc, &parts[k], 1) != CUDA_SUCCESS ||
            g.create(&q->gctx[k], desc, dev, CU_GREEN_CTX_DEFAULT_STREAM) != CUDA_SUCCESS)
            return fail(HYDRO_ECUDA, "green context %d could not be created", k);
        CUstream st = nullptr;
        if (g.stream_create(&st, q->gctx[k], CU_STREAM_NON_BLOCKING, 0) != CUDA_SUCCESS)
            return fail(HYDRO_ECUDA, "stream of green context %d could not be created", k);
        q->pos_st[k] = (cudaStream_t)st;
        smin = std::min(smin, (int)parts[k].sm.smCount);
    }
    q->sms_pos = smin;
    return HYDRO_OK;
}

hydro_status finalize(hydro_query *q) {
    if (q->finalized) return HYDRO_OK;
    const hydro_query_config &c = q->cfg;
    if (q->preds.empty()) return fail(HYDRO_ESTATE, "query has no predicates");
    CU(cudaSetDevice(c.device));
    CU(cudaDeviceGetAttribute(&q->sms, cudaDevAttrMultiProcessorCount, c.device));
    if (c.stream) {
        q->st = (cudaStream_t)c.stream;
    } else {
        CU(cudaStreamCreateWithFlags(&q->st, cudaStreamNonBlocking));
        q->own_stream = true;
    }
    CU(cudaStreamCreateWithFlags(&q->rst, cudaStreamNonBlocking));
    for (int i = 0; i < kEvRing; ++i) CU(cudaEventCreateWithFlags(&q->ev_done[i], cudaEventDisableTiming));
    CU(cudaEventCreateWithFlags(&q->ev_route, cudaEventDisableTiming));

    const int B = c.max_batch;
    const bool cnn = c.tuple_kind == HYDRO_TUPLE_U8_FRAME;
    const int wmax = max_width(q);
    TRY(alloc_scratch(q));
    q->lane_st[0] = q->st;
    save_lane(q, 0);
    q->n_lanes = std::max(1, c.lanes);
    if (q->n_lanes > 1) {
        // embeddings: each lane probes into its own miss list; the cache itself is indexed by
        // tuple id, and batches in flight on different lanes hold different ids
        if (c.policy == HYDRO_POLICY_LEARNED) return fail(HYDRO_EUNSUPPORTED, "lanes need a policy other than LEARNED");
        for (int l = 1; l < q->n_lanes; ++l) {
            TRY(alloc_scratch(q));
            save_lane(q, l);
        }
        // every lane on a library stream; each batch waits for the caller's stream (q->st)
        for (int l = 0; l < q->n_lanes; ++l) {
            CU(cudaStreamCreateWithFlags(&q->lane_st[l], cudaStreamNonBlocking));
            q->own_lane_st[l] = true;
        }
        CU(cudaEventCreateWithFlags(&q->ev_user, cudaEventDisableTiming));
        q->home_st = q->st;
        load_lane(q, 0);
    }
    if (c.pipeline) {
        if (q->n_lanes < 2) return fail(HYDRO_EUNSUPPORTED, "pipeline needs lanes >= 2");
        const int P = (int)q->preds.size();
        q->pipe = true;
        q->sms_full = q->sms;
        if (c.pipeline == 2) {
            TRY(make_partitions(q, P));
        } else {
            q->sms_pos = std::max(1, q->sms / P);
            for (int k = 0; k < P; ++k) CU(cudaStreamCreateWithFlags(&q->pos_st[k], cudaStreamNonBlocking));
        }
        for (int l = 0; l < q->n_lanes; ++l)
            for (int k = 0; k < P; ++k) CU(cudaEventCreateWithFlags(&q->ev_stage[l][k], cudaEventDisableTiming));
    }
    q->ring_len = c.stats_window + c.route_lag + 4;
    TRY(dalloc(q, &q->ring, sizeof(StatRow) * kMaxPred * q->ring_len));
    CU(cudaMemset(q->ring, 0, sizeof(StatRow) * kMaxPred * q->ring_len));
    const int nw = std::max(1, c.warmup_batches);
    TRY(dalloc(q, &q->warm, sizeof(StatRow) * kMaxPred * nw));
    CU(cudaMemset(q->warm, 0, sizeof(StatRow) * kMaxPred * nw));
    TRY(dalloc(q, &q->d_order, sizeof(int) * kMaxPred * c.max_in_flight));
    CU(cudaMallocHost(&q->h_order, sizeof(int) * kMaxPred * c.max_in_flight));
    TRY(dalloc(q, &q->d_err, sizeof(unsigned int)));
    CU(cudaMemset(q->d_err, 0, sizeof(unsigned int)));
    TRY(dalloc(q, &q->vmiss, sizeof(int) * kMaxPred));
    if (c.recheck_graphs) {
        TRY(dalloc(q, &q->d_switch_n, sizeof(int) * kMaxLanes * kMaxPred * kMaxPred));
        CU(cudaMemset(q->d_switch_n, 0, sizeof(int) * kMaxLanes * kMaxPred * kMaxPred));
        TRY(dalloc(q, &q->d_body_n, sizeof(int) * kMaxLanes * kMaxPred * 3));
        CU(cudaMemset(q->d_body_n, 0, sizeof(int) * kMaxLanes * kMaxPred * 3));
        TRY(dalloc(q, &q->d_launch_ctr, sizeof(unsigned long long)));
        CU(cudaMemset(q->d_launch_ctr, 0, sizeof(unsigned long long)));
        CU(cudaStreamCreateWithFlags(&q->cap_st, cudaStreamNonBlocking));
        for (int k = 0; k < 3; ++k) CU(cudaStreamCreateWithFlags(&q->cap_help[k], cudaStreamNonBlocking));
    }
    for (Emb &e : q->embs) {
        e.dW.resize(e.n_layers);
        e.db.resize(e.n_layers);
        for (int l = 0; l < e.n_layers; ++l) {
            TRY(upload(q, &e.dW[l], e.W[l].data(), e.W[l].size()));
            TRY(upload(q, &e.db[l], e.b[l].data(), e.b[l].size()));
        }
        TRY(dalloc(q, &e.values, sizeof(float) * (size_t)e.cap * e.dims.back()));
        TRY(dalloc(q, &e.tags, sizeof(int) * (size_t)e.cap));
        CU(cudaMemset(e.tags, 0, sizeof(int) * (size_t)e.cap));
    }

    // result slots
    q->res_bytes = kBitmapOff + sizeof(unsigned int) * (size_t)((B + 31) / 32);
    q->slots.resize(c.max_in_flight);
    for (Slot &s : q->slots) {
        TRY(dalloc(q, &s.dres, q->res_bytes));
        CU(cudaMallocHost(&s.hres, q->res_bytes));
        CU(cudaEventCreate(&s.start));
        CU(cudaEventCreate(&s.done));
    }

    // weights
    for (Pred &p : q->preds) {
        p.dW.resize(p.n_layers);
        p.db.resize(p.n_layers);
        for (int l = 0; l < p.n_layers; ++l) {
            TRY(upload(q, &p.dW[l], p.W[l].data(), p.W[l].size()));
            TRY(upload(q, &p.db[l], p.b[l].data(), p.b[l].size()));
        }
        if (p.kind == HYDRO_UDF_MLP && c.precision == HYDRO_PREC_BF16 && !p.upstream && p.n_layers >= 2 &&
            c.dim % 8 == 0) {
            p.tc_mlp = true;
            for (int l = 0; l + 1 < p.n_layers; ++l) p.tc_mlp = p.tc_mlp && tc_gemm_supported(p.dims[l], p.dims[l + 1]);
            if (p.tc_mlp) {
                p.dW16.assign(p.n_layers, nullptr);
                for (int l = 0; l + 1 < p.n_layers; ++l) {
                    std::vector<__nv_bfloat16> w16(p.W[l].size());
                    for (size_t k = 0; k < w16.size(); ++k) w16[k] = __float2bfloat16_rn(p.W[l][k]);
                    TRY(upload(q, &p.dW16[l], w16.data(), w16.size()));
                }
            }
        }
        if (p.kind == HYDRO_UDF_MLP) {
            p.mlp.n_layers = p.n_layers;
            p.mlp.max_width = wmax;
            for (int l = 0; l <= p.n_layers; ++l) p.mlp.dims[l] = p.dims[l];
            for (int l = 0; l < p.n_layers; ++l) {
                p.mlp.W[l] = p.dW[l];
                p.mlp.b[l] = p.db[l];
            }
        } else {
            TRY(upload(q, &p.dHead, p.head_w.data(), p.head_w.size()));
            p.dWt32.assign(p.n_layers, nullptr);
            p.dWt16.assign(p.n_layers, nullptr);
            p.dWtc.assign(p.n_layers, nullptr);
            p.dWts.assign(p.n_layers, nullptr);
            p.dWbs.assign(p.n_layers, nullptr);
            p.tc_all = tc_query(c) && p.n_layers > 1;
            p.tc_conv1 = tc_query(c) &&
                         tc_conv1_supported(c.channels, c.height, c.width, p.dims[1], c.max_batch, p.W[0].data(),
                                            p.b[0].data());
            if (p.tc_conv1) {
                std::vector<__half> c1;
                tc_conv1_pack_weights(p.W[0].data(), p.b[0].data(), c.channels, c1);
                TRY(upload(q, &p.dWc1, c1.data(), c1.size()));
            }
            for (int l = 1; l < p.n_layers; ++l) {
                const int ci_n = p.dims[l], co_n = p.dims[l + 1];
                std::vector<float> t32((size_t)9 * ci_n * co_n);
                std::vector<__nv_bfloat16> t16(t32.size());
                for (int co = 0; co < co_n; ++co)
                    for (int ci = 0; ci < ci_n; ++ci)
                        for (int tap = 0; tap < 9; ++tap) {
                            const float v = p.W[l][((size_t)co * ci_n + ci) * 9 + tap];
                            const size_t o = ((size_t)tap * ci_n + ci) * co_n + co;
                            t32[o] = v;
                            t16[o] = __float2bfloat16_rn(v);
                        }
                TRY(upload(q, &p.dWt32[l], t32.data(), t32.size()));
                TRY(upload(q, &p.dWt16[l], t16.data(), t16.size()));
                if (tc_query(c) && tc_conv_supported(ci_n, co_n, c.height, c.width)) {
                    std::vector<__nv_bfloat16> tc;
                    tc_conv_pack_weights(p.W[l].data(), ci_n, co_n, tc);
                    __nv_bfloat16 *d = nullptr;
                    TRY(upload(q, &d, tc.data(), tc.size()));
                    p.dWtc[l] = d;
                    std::vector<float> ts;
                    tc_conv_pack_weights_split(p.W[l].data(), ci_n, co_n, ts);
                    float *ds = nullptr;
                    TRY(upload(q, &ds, ts.data(), ts.size()));
                    p.dWts[l] = ds;
                    std::vector<__nv_bfloat16> tb;
                    tc_conv_pack_weights_split_bf16(p.W[l].data(), ci_n, co_n, tb);
                    __nv_bfloat16 *db = nullptr;
                    TRY(upload(q, &db, tb.data(), tb.size()));
                    p.dWbs[l] = db;
                } else {
                    p.tc_all = false;
                }
            }
        }
        if (c.precision == HYDRO_PREC_BF16X3 && !p.tc_all)
            return fail(HYDRO_EUNSUPPORTED, "split-BF16 working precision needs tensor-core CNN layers");
        if (p.margin_fp32 < 0.0) p.margin_fp32 = 1e-5 * std::max(1.0, std::fabs(p.threshold));
        if (p.margin_tf32 < 0.0) p.margin_tf32 = 5e-3 * std::max(1.0, std::fabs(p.threshold));
    }
    if (cnn && tc_query(c)) {
        hydro_status s = tc_conv_init(&q->tc, c.device);
        if (s != HYDRO_OK) return fail(s, "tensor-core conv init failed: %s", tc_conv_last_error());
    }
    if (c.policy == HYDRO_POLICY_LEARNED) TRY(finalize_learned(q));
    q->finalized = true;
    return HYDRO_OK;
}

// ---------------------------------------------------------------- profiling

int prof_begin(hydro_query *q, const ProfCtx *pc, int cls, double fpi, double bpi, double fixed_bytes) {
    if (!q->prof.on || !pc) return -1;
    Prof &P = q->prof;
    const int e = (int)P.recs.size() * 2;
    while ((int)P.ev.size() < e + 2) {
        cudaEvent_t x;
        if (cudaEventCreate(&x) != cudaSuccess) return -1;
        P.ev.push_back(x);
    }
    if (cudaEventRecord(P.ev[e], q->st) != cudaSuccess) return -1;
    P.recs.push_back(ProfRec{cls, e, pc->batch, pc->pred, pc->src, fpi, bpi, fixed_bytes});
    return e;
}

void prof_end(hydro_query *q, int e) {
    if (e >= 0) cudaEventRecord(q->prof.ev[e + 1], q->st);
}

// ---------------------------------------------------------------- UDF runs

// Run predicate p's UDF at precision prec on the *count tuples listed in
// `list` (indices into `tuples`), leaving FP32 scores in score32 (FP32/BF16)
// or FP64 scores in score64.  act: two activation buffers for that precision,
// sized for max_rows rows/frames.
hydro_status run_udf(hydro_query *q, const Pred &p, int prec, const int *count, const int *list,
                     const void *tuples, int max_rows, void *const act[2], float *score32, double *score64,
                     const ProfCtx *pc = nullptr, bool band = false) {
    const hydro_query_config &c = q->cfg;
    cudaStream_t st = q->st;
    if (p.kind == HYDRO_UDF_MLP) {
        const float *X = (const float *)tuples;
        if (prec == PREC_F64) {
            const int e = prof_begin(q, pc, PC_BAND64, (double)p.cost, 8.0 * c.dim, 0);
            launch_mlp_band_f64(count, list, X, c.dim, p.mlp, score64, q->sms, st);
            prof_end(q, e);
            q->launches++;
            return HYDRO_OK;
        }
        if (prec == PREC_BF16 && p.tc_mlp && ((uintptr_t)X % 16) == 0) {
            // BF16 tensor cores: gather the rows, hidden layers on tcgen05, the
            // one-output last layer folded into the last hidden layer's epilogue
            int e = prof_begin(q, pc, PC_GATHER, 0.0, 6.0 * c.dim, 0.0);
            launch_gather_bf16(count, list, X, c.dim, c.dim, q->stage16, max_rows, q->sms, st);
            prof_end(q, e);
            q->launches++;
            const __nv_bfloat16 *in = q->stage16;
            int cur = 0;
            const int L = p.n_layers;
            for (int l = 0; l + 1 < L; ++l) {
                const bool last = l + 2 == L;
                e = prof_begin(q, pc, PC_MLP_TC, 2.0 * p.dims[l] * p.dims[l + 1],
                               2.0 * (p.dims[l] + (last ? 0 : p.dims[l + 1])), 2.0 * p.dims[l] * p.dims[l + 1]);
                hydro_status rs = tc_gemm_run(q->gemm_encode, count, in, p.dims[l], p.dW16[l], p.db[l], p.dims[l + 1],
                                              q->act16[cur], max_rows, q->sms, st, q->d_err,
                                              last ? p.dW[L - 1] : nullptr, last ? q->partials : nullptr);
                prof_end(q, e);
                if (rs != HYDRO_OK) return fail(rs, "tensor-core GEMM: %s", tc_gemm_last_error());
                q->launches++;
                in = q->act16[cur];
                cur = 1 - cur;
            }
            tc_head_finalize(count, q->partials, tc_gemm_col_tiles(p.dims[L - 1]), (double)p.b[L - 1][0], 1, score32,
                             max_rows, q->sms, st);
            q->launches++;
            return HYDRO_OK;
        }
        // FP32 on CUDA cores
        if (p.n_layers == 1) {
            const int e = prof_begin(q, pc, PC_DOT, 2.0 * p.dims[0], 4.0 * p.dims[0] + 4, 4.0 * p.dims[0]);
            launch_mlp_dot_f32(count, list, X, c.dim, p.dW[0], p.b[0][0], p.dims[0], score32, max_rows, q->sms, st);
            prof_end(q, e);
            q->launches++;
            return HYDRO_OK;
        }
        int e = prof_begin(q, pc, PC_MLP, 2.0 * p.dims[0] * p.dims[1], 4.0 * (p.dims[0] + p.dims[1]),
                           4.0 * p.dims[0] * p.dims[1]);
        launch_mlp_layer_f32(count, list, X, c.dim, p.dW[0], p.db[0], (float *)act[0], p.dims[0], p.dims[1], 1,
                             max_rows, q->sms, st);
        prof_end(q, e);
        q->launches++;
        int cur = 0;
        for (int l = 1; l + 1 < p.n_layers; ++l) {
            e = prof_begin(q, pc, PC_MLP, 2.0 * p.dims[l] * p.dims[l + 1], 4.0 * (p.dims[l] + p.dims[l + 1]),
                           4.0 * p.dims[l] * p.dims[l + 1]);
            launch_mlp_layer_f32(count, nullptr, (const float *)act[cur], p.dims[l], p.dW[l], p.db[l],
                                 (float *)act[1 - cur], p.dims[l], p.dims[l + 1], 1, max_rows, q->sms, st);
            prof_end(q, e);
            q->launches++;
            cur = 1 - cur;
        }
        const int L = p.n_layers - 1;
        e = prof_begin(q, pc, PC_DOT, 2.0 * p.dims[L], 4.0 * p.dims[L] + 4, 4.0 * p.dims[L]);
        launch_mlp_dot_f32(count, nullptr, (const float *)act[cur], p.dims[L], p.dW[L], p.b[L][0], p.dims[L],
                           score32, max_rows, q->sms, st);
        prof_end(q, e);
        q->launches++;
        return HYDRO_OK;
    }
    // CNN
    const int H = c.height, Wd = c.width;
    const double hw = (double)H * Wd;
    if (prec == PREC_TF32X3 || prec == PREC_BF16X3) {
        if (!p.tc_all || !q->partials) return fail(HYDRO_EUNSUPPORTED, "split forms need tensor-core CNN layers");
        // the first recheck level on the tensor cores: 3xTF32 or split-BF16 [hi | lo] operands
        const bool sb = prec == PREC_BF16X3;
        const unsigned char *frames = (const unsigned char *)tuples;
        const double pb = sb ? 4.0 : 8.0;   // bytes per channel of a [hi | lo] pixel
        int e = prof_begin(q, pc, PC_CONV1, 2.0 * hw * 9 * p.dims[0] * p.dims[1], hw * (p.dims[0] + pb * p.dims[1]),
                           4.0 * 9 * p.dims[0] * p.dims[1]);
        launch_conv1_split(count, list, frames, c.channels, H, Wd, p.dW[0], p.db[0], p.dims[1], act[0], max_rows,
                           q->sms, q->st, sb);
        prof_end(q, e);
        q->launches++;
        int cur = 0;
        for (int l = 1; l < p.n_layers; ++l) {
            const bool last = l + 1 == p.n_layers;
            e = prof_begin(q, pc, PC_CONV_TF32, 2.0 * hw * 9 * p.dims[l] * p.dims[l + 1],
                           hw * pb * (p.dims[l] + (last ? 0 : p.dims[l + 1])), pb * 9 * p.dims[l] * p.dims[l + 1]);
            hydro_status rs = tc_conv_run(&q->tc, count, act[cur], p.dims[l], H, Wd, sb ? p.dWbs[l] : p.dWts[l],
                                          p.db[l], p.dims[l + 1], act[1 - cur], max_rows, q->sms, q->st, q->d_err,
                                          last ? p.dHead : nullptr, last ? q->partials : nullptr, sb ? 2 : 1);
            prof_end(q, e);
            if (rs != HYDRO_OK) return fail(rs, "tensor-core conv (split): %s", tc_conv_last_error());
            q->launches++;
            cur = 1 - cur;
        }
        tc_head_finalize(count, q->partials,
                         tc_conv_head_parts(p.dims[p.n_layers - 1], p.dims[p.n_layers], H, Wd, sb ? 2 : 1), p.head_b,
                         H * Wd, score32, max_rows, q->sms, q->st);
        q->launches++;
        return HYDRO_OK;
    }
    const double esz = prec == PREC_F64 ? 8.0 : prec == PREC_F32 ? 4.0 : 2.0;
    const unsigned char *frames = (const unsigned char *)tuples;
    int e = prof_begin(q, pc, PC_CONV1, 2.0 * hw * 9 * p.dims[0] * p.dims[1], hw * (p.dims[0] + esz * p.dims[1]),
                       4.0 * 9 * p.dims[0] * p.dims[1]);
    if (prec == PREC_BF16 && p.tc_conv1) {
        hydro_status rs = launch_conv1_tc(&q->tc, count, list, frames, c.channels, H, Wd, p.dWc1,
                                          (__nv_bfloat16 *)act[0], max_rows, q->sms, q->d_err, st);
        if (rs != HYDRO_OK) return fail(rs, "tensor-core first conv layer launch failed");
    } else {
        launch_conv1(prec, count, list, frames, c.channels, H, Wd, p.dW[0], p.db[0], p.dims[1], act[0], max_rows,
                     q->sms, st, band);
    }
    prof_end(q, e);
    q->launches++;
    int cur = 0;
    bool fused_head = false;
    for (int l = 1; l < p.n_layers; ++l) {
        const double fpi = 2.0 * hw * 9 * p.dims[l] * p.dims[l + 1];
        const double bpi = hw * esz * (p.dims[l] + p.dims[l + 1]);
        const double wb = 9.0 * p.dims[l] * p.dims[l + 1] * (prec == PREC_BF16 ? 2.0 : 4.0);
        if (prec == PREC_BF16 && p.dWtc[l]) {
            // the last layer folds pooling + head into its epilogue
            const bool last = l + 1 == p.n_layers && q->partials != nullptr;
            e = prof_begin(q, pc, PC_CONV_TC, fpi, last ? hw * esz * p.dims[l] : bpi, wb);
            hydro_status rs = tc_conv_run(&q->tc, count, act[cur], p.dims[l], H, Wd, p.dWtc[l], p.db[l],
                                          p.dims[l + 1], act[1 - cur], max_rows, q->sms, st, q->d_err,
                                          last ? p.dHead : nullptr, last ? q->partials : nullptr);
            prof_end(q, e);
            if (rs != HYDRO_OK) return fail(rs, "tensor-core conv: %s", tc_conv_last_error());
            fused_head = last;
        } else {
            const int cls = prec == PREC_BF16 ? PC_CONV_BF16 : prec == PREC_F32 ? PC_CONV_F32 : PC_CONV_F64;
            e = prof_begin(q, pc, cls, fpi, bpi, wb);
            const void *w = prec == PREC_BF16 ? (const void *)p.dWt16[l] : (const void *)p.dWt32[l];
            const int nk = launch_conv3x3_simt(prec, count, act[cur], p.dims[l], H, Wd, w, p.db[l], p.dims[l + 1],
                                               act[1 - cur], max_rows, q->sms, st, band);
            prof_end(q, e);
            q->launches += nk - 1;
        }
        q->launches++;
        cur = 1 - cur;
    }
    if (fused_head) {
        tc_head_finalize(count, q->partials, tc_conv_head_parts(p.dims[p.n_layers - 1], p.dims[p.n_layers], H, Wd, 0),
                         p.head_b, H * Wd, score32, max_rows, q->sms, st);
        q->launches++;
        return HYDRO_OK;
    }
    void *score = prec == PREC_F64 ? (void *)score64 : (void *)score32;
    const int CL = p.dims[p.n_layers];
    e = prof_begin(q, pc, PC_POOL, 2.0 * hw * CL, hw * esz * CL, 4.0 * CL);
    const int nk = launch_pool_head(prec, count, act[cur], H * Wd, CL, p.dHead, p.head_b, score, max_rows, q->sms, st);
    prof_end(q, e);
    q->launches += nk;
    return HYDRO_OK;
}

// Main-path scores of a predicate on a shared embedding (FP32): the
// embedding runs only on alive tuples whose id is not cached (results are
// stored in the cache with tag_value), then the head reads every alive
// tuple's embedding from the cache.  miss_count receives the misses.
hydro_status run_grouped(hydro_query *q, const Pred &p, const int *count, const int *list, const void *tuples,
                         const long long *ids, int tag_value, int max_rows, int *miss_count, float *score32,
                         const ProfCtx *pc = nullptr) {
    ProfCtx pc_miss{0, 0, SRC_MISS};
    if (pc) pc_miss = ProfCtx{pc->batch, pc->pred, SRC_MISS};
    const hydro_query_config &c = q->cfg;
    cudaStream_t st = q->st;
    Emb &e = q->embs[p.upstream - 1];
    const int D = e.dims.back();
    float *act[2] = {(float *)q->act[0], (float *)q->act[1]};
    launch_cache_probe_miss(count, list, ids, e.tags, e.cap, q->miss_list, miss_count, q->d_err, st);
    int ev = prof_begin(q, pc ? &pc_miss : nullptr, PC_MLP, 2.0 * e.dims[0] * e.dims[1],
                        4.0 * (e.dims[0] + e.dims[1]), 4.0 * e.dims[0] * e.dims[1]);
    launch_mlp_layer_f32(miss_count, q->miss_list, (const float *)tuples, c.dim, e.dW[0], e.db[0], act[0], e.dims[0],
                         e.dims[1], 1, max_rows, q->sms, st);
    prof_end(q, ev);
    int cur = 0;
    for (int l = 1; l < e.n_layers; ++l) {
        ev = prof_begin(q, pc ? &pc_miss : nullptr, PC_MLP, 2.0 * e.dims[l] * e.dims[l + 1],
                        4.0 * (e.dims[l] + e.dims[l + 1]), 4.0 * e.dims[l] * e.dims[l + 1]);
        launch_mlp_layer_f32(miss_count, nullptr, act[cur], e.dims[l], e.dW[l], e.db[l], act[1 - cur], e.dims[l],
                             e.dims[l + 1], 1, max_rows, q->sms, st);
        prof_end(q, ev);
        cur = 1 - cur;
    }
    launch_cache_store(miss_count, q->miss_list, ids, act[cur], D, e.values, e.tags, tag_value, max_rows, q->sms,
                       st);
    q->launches += 2 + e.n_layers;
    if (!score32) return HYDRO_OK;   // prefill: no head
    const int hs = p.head_start, L = p.n_layers;
    if (L - hs == 1) {
        launch_mlp_dot_f32(count, list, e.values, D, p.dW[hs], p.b[hs][0], D, score32, max_rows, q->sms, st, ids);
        q->launches++;
        return HYDRO_OK;
    }
    ev = prof_begin(q, pc, PC_MLP, 2.0 * D * p.dims[hs + 1], 4.0 * (D + p.dims[hs + 1]), 4.0 * D * p.dims[hs + 1]);
    launch_mlp_layer_f32(count, list, e.values, D, p.dW[hs], p.db[hs], act[0], D, p.dims[hs + 1], 1, max_rows, q->sms,
                         st, ids);
    prof_end(q, ev);
    cur = 0;
    for (int l = hs + 1; l + 1 < L; ++l) {
        ev = prof_begin(q, pc, PC_MLP, 2.0 * p.dims[l] * p.dims[l + 1], 4.0 * (p.dims[l] + p.dims[l + 1]),
                        4.0 * p.dims[l] * p.dims[l + 1]);
        launch_mlp_layer_f32(count, nullptr, act[cur], p.dims[l], p.dW[l], p.db[l], act[1 - cur], p.dims[l],
                             p.dims[l + 1], 1, max_rows, q->sms, st);
        prof_end(q, ev);
        cur = 1 - cur;
    }
    launch_mlp_dot_f32(count, nullptr, act[cur], p.dims[L - 1], p.dW[L - 1], p.b[L - 1][0], p.dims[L - 1], score32,
                       max_rows, q->sms, st);
    q->launches += L - hs;
    return HYDRO_OK;
}

// One stage: evaluate predicate p on the alive list (in_list, in_count),
// decide pass/fail exactly and close the stage.  Scores within a level's
// margin of the threshold go to the next level of the cascade:
//   BF16 query, CNN UDF:       BF16 tensor cores -> split BF16 (or 3xTF32) tensor cores
//                              -> FP32 CUDA cores -> FP64
//   split-BF16 query (CNN):    split BF16 tensor cores -> FP32 CUDA cores -> FP64
//   BF16 query, MLP UDF:       BF16 tensor cores -> FP32 -> FP64
//   FP32 query:                FP32 -> FP64
// The first recheck level of BF16 tensor-core CNN UDFs (hydro_query_config.split_precision).
int split_prec(const hydro_query_config &c) {
    return c.split_precision == HYDRO_PREC_TF32X3 ? PREC_TF32X3 : PREC_BF16X3;
}

// The recheck levels of stage pi, after the working-precision classify has
// filled band 1; `bt` is what the band entries index (the batch's tuples, or
// the lane's staging buffer).  Directly: every level's kernels are launched.
// While capturing (q->capturing): each level is a gate kernel followed by an
// IF node whose body holds the level's kernels, so a level with an empty band
// costs one tiny kernel.
hydro_status enqueue_rechecks(hydro_query *q, int pi, const void *bt, long long batch) {
    const hydro_query_config &c = q->cfg;
    const Pred &p = q->preds[pi];
    const bool bf16 = tc_query(c);
    const bool cnn = p.kind == HYDRO_UDF_CNN;
    const bool tf32_level = c.precision == HYDRO_PREC_BF16 && cnn && p.tc_all && q->partials;
    int *band1_count = q->ints + 2, *band2_count = q->ints + 3, *band3_count = q->ints + 4;
    const bool cap = q->capturing;
    const ProfCtx pc_rtf{batch, pi, SRC_RTF}, pc_r32{batch, pi, SRC_R32}, pc_r64{batch, pi, SRC_R64};
    const ProfCtx *prtf = cap ? nullptr : &pc_rtf, *pr32 = cap ? nullptr : &pc_r32, *pr64 = cap ? nullptr : &pc_r64;
    int gate = 0;
    // one level: directly, or as gate + IF node (body captured on the body stream)
    auto level = [&](const int *count, int *z0, int *z1, auto body) -> hydro_status {
        if (!cap) return body();
        if (gate >= 3) return fail(HYDRO_ECUDA, "more than three recheck levels");
        cudaGraphConditionalHandle h;
        CU(cudaGraphConditionalHandleCreate(&h, q->cap_graph, 0, cudaGraphCondAssignDefault));
        int *body_n = q->d_body_n + ((size_t)q->cur_lane * kMaxPred + pi) * 3 + gate;
        launch_gate(count, (unsigned long long)h, z0, z1, q->d_launch_ctr, body_n, q->st);
        cudaStreamCaptureStatus cs;
        cudaGraph_t g = nullptr;
        const cudaGraphNode_t *deps = nullptr;
        const cudaGraphEdgeData *ed = nullptr;
        size_t nd = 0;
        CU(cudaStreamGetCaptureInfo(q->st, &cs, nullptr, &g, &deps, &ed, &nd));
        alignas(cudaGraphNodeParams) unsigned char pbuf[sizeof(cudaGraphNodeParams)];
        std::memset(pbuf, 0, sizeof pbuf);
        cudaGraphNodeParams &np = *reinterpret_cast<cudaGraphNodeParams *>(pbuf);   // zeroed, as the API requires
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeIf;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        CU(cudaGraphAddNode(&node, g, deps, ed, nd, &np));
        CU(cudaStreamUpdateCaptureDependencies(q->st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
        if (q->cap_depth >= 3) return fail(HYDRO_ECUDA, "conditional bodies nest too deep");
        const cudaStream_t hs = q->cap_help[q->cap_depth++];
        CU(cudaStreamBeginCaptureToGraph(hs, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                         cudaStreamCaptureModeThreadLocal));
        const cudaStream_t top = q->st;
        q->st = hs;
        const long long l0 = q->launches;
        hydro_status rs = body();
        const int n_body = (int)(q->launches - l0);
        cudaGraph_t out = nullptr;
        cudaError_t ee = cudaStreamEndCapture(hs, &out);
        q->cap_depth--;
        q->st = top;
        if (rs != HYDRO_OK) return rs;
        CU(ee);
        q->cap_body_counts.push_back({body_n, n_body});   // written once the capture has ended
        ++gate;
        q->launches = l0 + 1;   // at capture time only the gate is a launch of every replay
        return HYDRO_OK;
    };
    const int *b64_count = band1_count, *b64_m = q->band1_m, *b64_t = q->band1_t;
    if (bf16) {
        // FP32-level input: band 1 directly, or what the split level leaves undecided
        const int *b32_count = band1_count, *b32_m = q->band1_m, *b32_t = q->band1_t;
        if (tf32_level) {
            TRY(level(band1_count, band2_count, band3_count, [&]() -> hydro_status {
                TRY(run_udf(q, p, split_prec(c), band1_count, q->band1_t, bt, q->cap1, q->ract32, q->rscore_t,
                            nullptr, prtf));
                launch_recheck_classify_f32(band1_count, q->band1_m, q->band1_t, q->rscore_t, p.threshold,
                                            p.margin_tf32, q->pass, q->band2_m, q->band2_t, band2_count, q->cap2,
                                            q->d_err, q->st);
                q->launches++;
                return HYDRO_OK;
            }));
            b32_count = band2_count;
            b32_m = q->band2_m;
            b32_t = q->band2_t;
        }
        TRY(level(b32_count, band3_count, nullptr, [&]() -> hydro_status {
            if (!cnn && p.upstream) {
                const int e = prof_begin(q, pr32, PC_BAND32, (double)p.cost, 4.0 * c.dim, 0);
                launch_mlp_band_f32(b32_count, b32_t, (const float *)bt, c.dim, p.mlp, q->rscore32, q->sms, q->st);
                prof_end(q, e);
                q->launches++;
            } else if (!cnn) {
                // the band as a (short) GEMM: weight tiles shared by the band's rows
                TRY(run_udf(q, p, PREC_F32, b32_count, b32_t, bt, q->cap1, q->act, q->rscore32, nullptr, pr32));
            } else {
                TRY(run_udf(q, p, PREC_F32, b32_count, b32_t, bt, tf32_level ? q->cap2 : q->cap1, q->ract32,
                            q->rscore32, nullptr, pr32, true));
            }
            launch_recheck_classify_f32(b32_count, b32_m, b32_t, q->rscore32, p.threshold, p.margin_fp32, q->pass,
                                        q->band3_m, q->band3_t, band3_count, q->cap3, q->d_err, q->st);
            q->launches++;
            return HYDRO_OK;
        }));
        b64_count = band3_count;
        b64_m = q->band3_m;
        b64_t = q->band3_t;
    }
    TRY(level(b64_count, nullptr, nullptr, [&]() -> hydro_status {
        if (!cnn) {
            const int e = prof_begin(q, pr64, PC_BAND64, (double)p.cost, 4.0 * c.dim, 0);
            launch_mlp_band_f64(b64_count, b64_t, (const float *)bt, c.dim, p.mlp, q->rscore64, q->sms, q->st);
            prof_end(q, e);
            q->launches++;
        } else {
            TRY(run_udf(q, p, PREC_F64, b64_count, b64_t, bt, q->cap3, q->ract64, nullptr, q->rscore64, pr64, true));
        }
        launch_recheck_classify_f64(b64_count, b64_m, b64_t, q->rscore64, p.threshold, q->pass, q->d_err, q->st);
        q->launches++;
        return HYDRO_OK;
    }));
    return HYDRO_OK;
}

// Capture the recheck levels of predicate pi on the current lane into a graph
// (once per lane and predicate): its tuples are the lane's staging buffer.
hydro_status ensure_tail(hydro_query *q, int pi) {
    const int l = q->cur_lane;
    if (q->tail[l][pi]) return HYDRO_OK;
    const cudaStream_t saved = q->st;
    const long long l0 = q->launches;
    q->st = q->cap_st;
    q->cap_body_counts.clear();
    CU(cudaStreamBeginCapture(q->cap_st, cudaStreamCaptureModeThreadLocal));
    cudaStreamCaptureStatus cs;
    hydro_status rs = HYDRO_OK;
    if (cudaStreamGetCaptureInfo(q->cap_st, &cs, nullptr, &q->cap_graph, nullptr, nullptr, nullptr) != cudaSuccess)
        rs = fail(HYDRO_ECUDA, "capture info of the recheck graph");
    q->capturing = true;
    if (rs == HYDRO_OK) rs = enqueue_rechecks(q, pi, q->band_rows, -1);
    q->capturing = false;
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(q->cap_st, &g);
    q->st = saved;
    q->cap_graph = nullptr;
    const int gates = (int)(q->launches - l0);
    q->launches = l0;
    if (rs != HYDRO_OK) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return rs;
    }
    if (ee != cudaSuccess || !g) {
        cudaGetLastError();
        return fail(HYDRO_ECUDA, "capture of the recheck graph failed: %s", cudaGetErrorString(ee));
    }
    cudaError_t ie = cudaGraphInstantiate(&q->tail[l][pi], g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
        q->tail[l][pi] = nullptr;
        cudaGetLastError();
        return fail(HYDRO_ECUDA, "instantiating the recheck graph failed: %s", cudaGetErrorString(ie));
    }
    q->tail_gates[l][pi] = gates;
    // the bodies' kernel counts, read by the gates (nothing of this graph runs yet)
    for (const auto &bc : q->cap_body_counts) CU(cudaMemcpy(bc.first, &bc.second, sizeof(int), cudaMemcpyHostToDevice));
    q->cap_body_counts.clear();
    return HYDRO_OK;
}

// dev_rows (device-dispatched batches, while capturing the lane's batch
// graph): the stage's statistics go to the lane's result rows and its recheck
// levels become IF nodes that read the lane's copy of the batch directly.
hydro_status run_stage(hydro_query *q, int pi, const int *in_count, const int *in_list, int *out_list,
                       int *out_count, bool eval_all, const void *tuples, const long long *ids, int n,
                       long long batch, Slot *slot, StatRow *dev_rows = nullptr) {
    const hydro_query_config &c = q->cfg;
    const Pred &p = q->preds[pi];
    // split_main: split BF16 is the working precision, so the cascade is
    // split BF16 -> FP32 -> FP64 (band 1 goes straight to the FP32 level)
    const bool split_main = c.precision == HYDRO_PREC_BF16X3;
    const bool bf16 = tc_query(c);
    const bool cnn = p.kind == HYDRO_UDF_CNN;
    const bool tf32_level = c.precision == HYDRO_PREC_BF16 && cnn && p.tc_all && q->partials;
    const int wprec = split_main ? split_prec(c) : bf16 ? PREC_BF16 : PREC_F32;
    int *band1_count = q->ints + 2, *band2_count = q->ints + 3, *band3_count = q->ints + 4;
    const ProfCtx pc_main{batch, pi, SRC_MAIN};
    int *miss_count = nullptr;
    const bool measure = c.cost_source == HYDRO_COST_MEASURED;
    StatRow *row = dev_rows ? dev_rows + pi : q->ring + (batch % q->ring_len) * kMaxPred + pi;
    if (measure) {
        launch_stage_start(row, q->st);
        q->launches++;
    }
    if (p.upstream) {
        miss_count = q->ints + 5;
        TRY(run_grouped(q, p, in_count, in_list, tuples, ids, (int)(batch + 1), std::max(n, 1), miss_count,
                        q->score32, &pc_main));
    } else {
        TRY(run_udf(q, p, wprec, in_count, in_list, tuples, std::max(n, 1), q->act, q->score32, nullptr, &pc_main));
    }

    // level 0 -> band 1 (FP32 queries: band 1 is the FP64 band, capacity cap3)
    const double margin0 = split_main ? p.margin_tf32 : bf16 ? p.margin_lowp : p.margin_fp32;
    launch_classify_f32(in_count, in_list, q->score32, p.threshold, margin0, q->pass,
                        q->band1_m, q->band1_t, band1_count, bf16 ? q->cap1 : q->cap3, q->d_err, q->st);
    q->launches++;
    if (dev_rows) {
        TRY(enqueue_rechecks(q, pi, tuples, batch));
    } else if (c.recheck_graphs && !q->gctx[0]) {
        // the band's tuples to the lane's staging buffer, then the captured levels
        launch_band_stage(band1_count, q->band1_t, tuples, tuple_bytes(c), q->band_rows, bf16 ? q->cap1 : q->cap3,
                          q->sms, q->st);
        q->launches++;
        TRY(ensure_tail(q, pi));
        CU(cudaGraphLaunch(q->tail[q->cur_lane][pi], q->st));
        q->launches += q->tail_gates[q->cur_lane][pi];
    } else {
        TRY(enqueue_rechecks(q, pi, tuples, batch));
    }
    // the band counts each level saw, for the statistics row
    const int *cnt_tf = tf32_level ? band1_count : nullptr;
    const int *cnt_32 = bf16 ? (tf32_level ? band2_count : band1_count) : nullptr;
    const int *b64_count = bf16 ? band3_count : band1_count;
    StatRow *rrow = dev_rows ? row : (StatRow *)(slot->dres + kRowsOff) + pi;
    StatRow *warm = nullptr;
    if (!dev_rows && adaptive(c.policy) && batch < c.warmup_batches) warm = q->warm + batch * kMaxPred + pi;
    launch_compact(in_count, in_list, q->pass, out_list, out_count, eval_all ? q->acc : nullptr, cnt_tf, cnt_32,
                   b64_count, miss_count, row, rrow, warm, q->st, measure ? 1 : 0);
    q->launches++;
    return HYDRO_OK;
}

// Capture the current lane's batch graph (once): the initial alive list, the
// dispatch kernel (order -> SWITCH values), one SWITCH node per position with
// one body per predicate (that predicate's whole stage at that position,
// recheck levels as nested IF nodes), and the result bitmap.
hydro_status ensure_batch_graph(hydro_query *q) {
    const int l = q->cur_lane;
    if (q->bgraph[l]) return HYDRO_OK;
    const int P = (int)q->preds.size();
    const cudaStream_t saved = q->st;
    const long long l0 = q->launches;
    ResHdr *hdr = (ResHdr *)q->lres;
    int *bodyn = q->d_switch_n + (size_t)l * kMaxPred * kMaxPred;
    std::vector<int> hbody((size_t)P * P, 0);
    q->st = q->cap_st;
    q->cap_body_counts.clear();
    q->cap_depth = 0;
    CU(cudaStreamBeginCapture(q->cap_st, cudaStreamCaptureModeThreadLocal));
    hydro_status rs = HYDRO_OK;
    cudaStreamCaptureStatus cs;
    if (cudaStreamGetCaptureInfo(q->cap_st, &cs, nullptr, &q->cap_graph, nullptr, nullptr, nullptr) != cudaSuccess)
        rs = fail(HYDRO_ECUDA, "capture info of the batch graph");
    q->capturing = true;
    SwitchHandles sh{};
    for (int k = 0; k < P && rs == HYDRO_OK; ++k) {
        cudaGraphConditionalHandle h;
        if (cudaGraphConditionalHandleCreate(&h, q->cap_graph, 0, cudaGraphCondAssignDefault) != cudaSuccess)
            rs = fail(HYDRO_ECUDA, "conditional handle of position %d", k);
        sh.h[k] = (unsigned long long)h;
    }
    if (rs == HYDRO_OK) {
        launch_init_alive_dev(q->alive[0], q->ints + 0, q->ln, q->cfg.max_batch, q->st);
        launch_dispatch(q->lord, sh, P, bodyn, q->d_launch_ctr, hdr->order, q->st);
    }
    int cur = 0;
    for (int k = 0; k < P && rs == HYDRO_OK; ++k) {
        cudaGraph_t g = nullptr;
        const cudaGraphNode_t *deps = nullptr;
        const cudaGraphEdgeData *ed = nullptr;
        size_t nd = 0;
        if (cudaStreamGetCaptureInfo(q->st, &cs, nullptr, &g, &deps, &ed, &nd) != cudaSuccess) {
            rs = fail(HYDRO_ECUDA, "capture info at position %d", k);
            break;
        }
        alignas(cudaGraphNodeParams) unsigned char pbuf[sizeof(cudaGraphNodeParams)];
        std::memset(pbuf, 0, sizeof pbuf);
        cudaGraphNodeParams &np = *reinterpret_cast<cudaGraphNodeParams *>(pbuf);   // zeroed, as the API requires
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = (cudaGraphConditionalHandle)sh.h[k];
        np.conditional.type = cudaGraphCondTypeSwitch;
        np.conditional.size = (unsigned)P;
        cudaGraphNode_t node;
        if (cudaGraphAddNode(&node, g, deps, ed, nd, &np) != cudaSuccess ||
            cudaStreamUpdateCaptureDependencies(q->st, &node, nullptr, 1, cudaStreamSetCaptureDependencies) !=
                cudaSuccess) {
            rs = fail(HYDRO_ECUDA, "SWITCH node of position %d", k);
            break;
        }
        for (int i = 0; i < P && rs == HYDRO_OK; ++i) {
            const cudaStream_t hs = q->cap_help[q->cap_depth++];
            if (cudaStreamBeginCaptureToGraph(hs, np.conditional.phGraph_out[i], nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                q->cap_depth--;
                rs = fail(HYDRO_ECUDA, "capture of position %d, predicate %d", k, i);
                break;
            }
            q->st = hs;
            const long long b0 = q->launches;
            rs = run_stage(q, i, q->ints + cur, q->alive[cur], q->alive[1 - cur], q->ints + 1 - cur, false,
                           q->batch_rows, nullptr, q->cfg.max_batch, -1, nullptr, (StatRow *)(q->lres + kRowsOff));
            hbody[(size_t)k * P + i] = (int)(q->launches - b0);
            cudaGraph_t out = nullptr;
            cudaError_t ee = cudaStreamEndCapture(hs, &out);
            q->cap_depth--;
            q->st = q->cap_st;
            if (rs == HYDRO_OK && ee != cudaSuccess) rs = fail(HYDRO_ECUDA, "end of capture: %s", cudaGetErrorString(ee));
        }
        cur = 1 - cur;
    }
    if (rs == HYDRO_OK)
        launch_result_dev(q->ints + cur, q->alive[cur], q->ln, (unsigned int *)(q->lres + kBitmapOff), &hdr->n_pass,
                          q->st);
    q->capturing = false;
    cudaGraph_t graph = nullptr;
    cudaError_t ee = cudaStreamEndCapture(q->cap_st, &graph);
    q->st = saved;
    q->cap_graph = nullptr;
    q->launches = l0;
    if (rs != HYDRO_OK) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return rs;
    }
    if (ee != cudaSuccess || !graph) {
        cudaGetLastError();
        return fail(HYDRO_ECUDA, "capture of the batch graph failed: %s", cudaGetErrorString(ee));
    }
    cudaError_t ie = cudaGraphInstantiate(&q->bgraph[l], graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
        q->bgraph[l] = nullptr;
        cudaGetLastError();
        return fail(HYDRO_ECUDA, "instantiating the batch graph failed: %s", cudaGetErrorString(ie));
    }
    // kernel counts of the bodies (the dispatch kernel adds the chosen ones, the gates theirs)
    CU(cudaMemcpy(bodyn, hbody.data(), sizeof(int) * hbody.size(), cudaMemcpyHostToDevice));
    for (const auto &bc : q->cap_body_counts) CU(cudaMemcpy(bc.first, &bc.second, sizeof(int), cudaMemcpyHostToDevice));
    q->cap_body_counts.clear();
    return HYDRO_OK;
}

// A batch under the learned router: per-tuple orders (proxy, or the batch's
// rank order until the proxy is trained), then P rounds; round r splits the
// alive tuples by the r-th predicate of their order into one queue per
// predicate and evaluates all queues with grouped launches (FP32, FP64
// recheck within margin_fp32).  Leaves the final alive list in
// q->alive[*cur_out], its count in q->ints[*cur_out].
hydro_status run_batch_learned(hydro_query *q, long long b, const int *order, bool eval_all, const void *tuples,
                               int n, Slot &slot, int *cur_out) {
    const hydro_query_config &c = q->cfg;
    const int P = (int)q->preds.size(), B = c.max_batch;
    cudaStream_t st = q->st;
    const float *X = (const float *)tuples;
    int *cnt = q->ints;
    StatRow *row = q->ring + (b % q->ring_len) * kMaxPred;
    StatRow *rrow = (StatRow *)(slot.dres + kRowsOff);
    launch_zero_rows(row, rrow, P, q->visited, q->label, n, st);
    launch_init_alive(q->alive[0], cnt + 0, n, nullptr, st);
    RouterCosts costs{};
    for (int i = 0; i < P; ++i) costs.c[i] = q->preds[i].cost;
    if (q->proxy_ready && !eval_all) {
        launch_mlp_layer_f32(cnt + 0, nullptr, X, c.dim, q->pW1, q->pb1, q->pH, c.dim, q->ph, 1, std::max(n, 1),
                             q->sms, st);
        launch_mlp_layer_f32(cnt + 0, nullptr, q->pH, q->ph, q->pW2, q->pb2, q->pZ, q->ph, P, 0, std::max(n, 1),
                             q->sms, st);
        launch_tuple_order(n, P, q->pZ, P, costs, nullptr, q->order_t, q->sms, st);
        q->launches += 3;
    } else {
        for (int i = 0; i < P; ++i) q->h_fallback[i] = order[i];
        CU(cudaMemcpyAsync(q->d_fallback, q->h_fallback, sizeof(int) * P, cudaMemcpyHostToDevice, st));
        launch_tuple_order(n, P, nullptr, 0, costs, q->d_fallback, q->order_t, q->sms, st);
        q->launches++;
    }
    RoundTests tests{};
    for (int i = 0; i < P; ++i) {
        tests.t[i] = q->preds[i].threshold;
        tests.margin[i] = q->preds[i].margin_fp32;
    }
    int maxL = 0;
    for (const Pred &p : q->preds) maxL = std::max(maxL, p.n_layers);
    int cur = 0;
    for (int r = 0; r < P; ++r) {
        launch_partition(cnt + cur, q->alive[cur], q->order_t, r, P, q->queues, B, q->qcount, st);
        for (int l = 0; l + 1 < maxL; ++l) {
            GroupedLayers g{};
            int tiles = 0;
            for (int i = 0; i < P; ++i) {
                const Pred &p = q->preds[i];
                if (l + 1 >= p.n_layers) continue;
                GroupLayer &L = g.l[g.n++];
                L.count = q->qcount + i;
                L.rows = l == 0 ? q->queues + (size_t)i * B : nullptr;
                L.X = l == 0 ? X : q->gact[2 * i + (l - 1) % 2];
                L.ldx = l == 0 ? c.dim : p.dims[l];
                L.W = p.dW[l];
                L.b = p.db[l];
                L.Y = q->gact[2 * i + l % 2];
                L.K = p.dims[l];
                L.N = p.dims[l + 1];
                L.relu = 1;
                tiles += ((B + 63) / 64) * ((L.N + 63) / 64);
            }
            if (g.n) {
                launch_grouped_layer_f32(g, tiles, q->sms, st);
                q->launches++;
            }
        }
        GroupedLayers dots{};
        for (int i = 0; i < P; ++i) {
            const Pred &p = q->preds[i];
            const int L = p.n_layers - 1;
            GroupLayer &G = dots.l[dots.n++];
            G.count = q->qcount + i;
            G.rows = L == 0 ? q->queues + (size_t)i * B : nullptr;
            G.X = L == 0 ? X : q->gact[2 * i + (L - 1) % 2];
            G.ldx = L == 0 ? c.dim : p.dims[L];
            G.W = p.dW[L];
            G.bconst = p.b[L][0];
            G.K = p.dims[L];
            G.N = 1;
        }
        launch_grouped_dot_f32(dots, q->qscore, B, P * B, q->sms, st);
        launch_grouped_classify(P, q->qcount, q->queues, B, q->qscore, B, tests, q->okf, q->label, q->visited,
                                q->bandg, q->bandt, cnt + 2, B, row, rrow, q->d_err, st);
        launch_grouped_band_f64(cnt + 2, q->bandg, q->bandt, X, c.dim, q->gmlps, tests, q->okf, q->label, row, rrow,
                                q->sms, st);
        q->launches += 4;
        if (!eval_all) {
            launch_survivors(cnt + cur, q->alive[cur], q->okf, q->alive[1 - cur], cnt + 1 - cur, st);
            q->launches++;
            cur = 1 - cur;
        }
    }
    if (eval_all) {
        launch_full_label_acc(q->label, n, P, q->acc, st);
        launch_acc_to_alive(q->acc, n, q->alive[1 - cur], cnt + 1 - cur, st);
        q->launches += 2;
        cur = 1 - cur;
    }
    if (adaptive(c.policy) && b < c.warmup_batches)
        CU(cudaMemcpyAsync(q->warm + b * kMaxPred, row, sizeof(StatRow) * P, cudaMemcpyDeviceToDevice, st));
    // outcomes for the proxy's training ring
    const int R = (int)q->ring_n.size();
    const int rs = (int)(b % R);
    if (n > 0) {
        CU(cudaMemcpyAsync(q->ringX + (size_t)rs * B * c.dim, X, sizeof(float) * (size_t)n * c.dim,
                           cudaMemcpyDeviceToDevice, st));
        CU(cudaMemcpyAsync(q->ringL + (size_t)rs * B, q->label, n, cudaMemcpyDeviceToDevice, st));
        CU(cudaMemcpyAsync(q->ringM + (size_t)rs * B, q->visited, n, cudaMemcpyDeviceToDevice, st));
    }
    q->ring_n[rs] = n;
    q->last_learned_batch = b;
    q->last_n = n;
    *cur_out = cur;
    return HYDRO_OK;
}

// Retrain the proxy on the training ring (enqueued after the batch that
// filled the ring; batches submitted later use the new weights).
hydro_status train_proxy(hydro_query *q) {
    const hydro_query_config &c = q->cfg;
    const int P = (int)q->preds.size(), D = c.dim, H = q->ph, B = c.max_batch;
    const size_t nW1 = (size_t)H * D;
    for (int e = 0; e < std::max(1, c.proxy_epochs); ++e)
        for (size_t s = 0; s < q->ring_n.size(); ++s) {
            const int M = q->ring_n[s];
            if (M <= 0) continue;
            const float *Xs = q->ringX + s * (size_t)B * D;
            launch_identity_list(q->alive[0], q->ints + 7, 0, M, q->st);
            launch_mlp_layer_f32(q->ints + 7, nullptr, Xs, D, q->pW1, q->pb1, q->pH, D, H, 1, M, q->sms, q->st);
            launch_mlp_layer_f32(q->ints + 7, nullptr, q->pH, H, q->pW2, q->pb2, q->pZ, H, P, 0, M, q->sms, q->st);
            ProxyTrain pt{};
            pt.M = M;
            pt.P = P;
            pt.H = H;
            pt.D = D;
            pt.sms = q->sms;
            pt.t = ++q->adam_t;
            pt.lr = c.proxy_lr;
            pt.X = Xs;
            pt.Hact = q->pH;
            pt.Z = q->pZ;
            pt.dZ = q->pdZ;
            pt.dH = q->pdH;
            pt.part = q->ppart;
            pt.inv_pairs = q->pinv;
            pt.label = q->ringL + s * (size_t)B;
            pt.mask = q->ringM + s * (size_t)B;
            pt.W1 = q->pW1;
            pt.b1 = q->pb1;
            pt.W2 = q->pW2;
            pt.b2 = q->pb2;
            pt.gW1 = q->pg;
            pt.gb1 = q->pg + nW1;
            pt.gW2 = pt.gb1 + H;
            pt.gb2 = pt.gW2 + (size_t)P * H;
            pt.mW1 = q->pm;
            pt.mb1 = q->pm + nW1;
            pt.mW2 = pt.mb1 + H;
            pt.mb2 = pt.mW2 + (size_t)P * H;
            pt.vW1 = q->pv;
            pt.vb1 = q->pv + nW1;
            pt.vW2 = pt.vb1 + H;
            pt.vb2 = pt.vW2 + (size_t)P * H;
            launch_proxy_train_step(pt, q->st);
            q->launches += 12;
        }
    q->proxy_ready = true;
    return HYDRO_OK;
}

hydro_status wait_event(cudaEvent_t ev, long long wait_ms, bool *done) {
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess) {
            *done = true;
            return HYDRO_OK;
        }
        if (e != cudaErrorNotReady) return fail(HYDRO_ECUDA, "event query: %s", cudaGetErrorString(e));
        if (wait_ms == 0) break;
        if (wait_ms > 0) {
            auto el = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0);
            if (el.count() >= wait_ms) break;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    *done = false;
    return HYDRO_OK;
}

hydro_status check_query(hydro_query *q) {
    if (!q) return fail(HYDRO_EINVAL, "NULL query");
    if (q->dead) return fail(HYDRO_ESTATE, "query is in a failed state");
    return HYDRO_OK;
}

}  // namespace

void hydro::set_last_error(const char *msg) { g_err = msg; }

// ================================================================ C ABI

extern "C" {

const char *hydro_last_error(void) { return g_err.c_str(); }

void hydro_default_config(hydro_query_config *cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof *cfg);
    cfg->tuple_kind = HYDRO_TUPLE_F32;
    cfg->policy = HYDRO_POLICY_RANK;
    cfg->precision = HYDRO_PREC_FP32;
    cfg->cost_source = HYDRO_COST_MODEL;
    cfg->warmup_batches = 1;
    cfg->stats_window = 8;
    cfg->route_lag = 1;
    cfg->max_in_flight = 4;
    cfg->device = 0;
    cfg->stream = nullptr;
    cfg->proxy_hidden = 64;
    cfg->proxy_refresh = 16;
    cfg->proxy_epochs = 2;
    cfg->proxy_lr = 1e-3f;
    cfg->proxy_seed = 1;
    cfg->recheck_graphs = 1;
}

hydro_status hydro_create_query(const hydro_query_config *cfg, hydro_query **out) {
    g_err.clear();
    if (!cfg || !out) return fail(HYDRO_EINVAL, "NULL argument");
    *out = nullptr;
    const hydro_query_config &c = *cfg;
    if (c.tuple_kind == HYDRO_TUPLE_F32) {
        if (c.dim < 1 || c.dim > (1 << 16)) return fail(HYDRO_EINVAL, "dim out of range");
    } else if (c.tuple_kind == HYDRO_TUPLE_U8_FRAME) {
        if (c.channels < 1 || c.channels > 8 || c.height < 1 || c.width < 1 || c.height * c.width > (1 << 16))
            return fail(HYDRO_EINVAL, "frame shape out of range");
    } else {
        return fail(HYDRO_EINVAL, "unknown tuple_kind %d", c.tuple_kind);
    }
    if (c.max_batch < 1 || c.max_batch > 65536) return fail(HYDRO_EINVAL, "max_batch must be 1..65536");
    if (c.policy < 0 || c.policy > 5) return fail(HYDRO_EINVAL, "unknown policy");
    if (c.policy == HYDRO_POLICY_LEARNED) {
        if (c.tuple_kind != HYDRO_TUPLE_F32 || c.precision != HYDRO_PREC_FP32)
            return fail(HYDRO_EUNSUPPORTED, "the learned router needs F32 tuples and an FP32 query");
        if (c.proxy_hidden < 0 || c.proxy_hidden > 1024 || c.proxy_refresh < 0 || c.proxy_epochs < 0 ||
            !(c.proxy_lr >= 0.f))
            return fail(HYDRO_EINVAL, "bad proxy settings");
    }
    if (c.precision != HYDRO_PREC_FP32 && c.precision != HYDRO_PREC_BF16 && c.precision != HYDRO_PREC_BF16X3)
        return fail(HYDRO_EINVAL, "precision must be FP32, BF16 or (frame tuples) BF16X3");
    if (c.precision == HYDRO_PREC_BF16X3 && c.tuple_kind != HYDRO_TUPLE_U8_FRAME)
        return fail(HYDRO_EUNSUPPORTED, "split-BF16 working precision is built for frame (CNN) queries");
    if (c.precision == HYDRO_PREC_BF16X3 && c.split_precision == HYDRO_PREC_TF32X3)
        return fail(HYDRO_EUNSUPPORTED, "split-BF16 working precision takes split_precision BF16X3 (or 0)");

    if (c.split_precision != 0 && c.split_precision != HYDRO_PREC_TF32X3 && c.split_precision != HYDRO_PREC_BF16X3)
        return fail(HYDRO_EINVAL, "split_precision must be TF32X3 or BF16X3");
    if (c.cost_source != HYDRO_COST_MODEL && c.cost_source != HYDRO_COST_MEASURED)
        return fail(HYDRO_EINVAL, "unknown cost source");
    if (c.cost_source == HYDRO_COST_MEASURED &&
        ((c.policy != HYDRO_POLICY_RANK && c.policy != HYDRO_POLICY_COST) || c.warmup_batches < 1))
        return fail(HYDRO_EUNSUPPORTED, "measured cost needs the rank or cost policy and warmup_batches >= 1");
    if (c.warmup_batches < 0 || c.warmup_batches > 64) return fail(HYDRO_EINVAL, "warmup_batches must be 0..64");
    if (c.stats_window < 1 || c.stats_window > 1024) return fail(HYDRO_EINVAL, "stats_window must be 1..1024");
    if (c.route_lag < 0 || c.route_lag > 7) return fail(HYDRO_EINVAL, "route_lag must be 0..7");
    if (c.lanes < 0 || c.lanes > kMaxLanes) return fail(HYDRO_EINVAL, "lanes must be 1..%d", kMaxLanes);
    if (c.lanes > c.route_lag + 1) return fail(HYDRO_EINVAL, "lanes must be <= route_lag + 1");
    if (c.max_in_flight < 1 || c.max_in_flight > 64) return fail(HYDRO_EINVAL, "max_in_flight must be 1..64");
    if (c.pipeline < 0 || c.pipeline > 2) return fail(HYDRO_EINVAL, "pipeline must be 0, 1 or 2");
    if (c.pipeline && (c.lanes < 2 || c.policy == HYDRO_POLICY_LEARNED))
        return fail(HYDRO_EUNSUPPORTED, "pipeline needs lanes >= 2 and a policy other than LEARNED");
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(HYDRO_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));
    }
    if (c.device < 0 || c.device >= ndev) return fail(HYDRO_EINVAL, "device %d out of range", c.device);
    hydro_query *q = new (std::nothrow) hydro_query();
    if (!q) return fail(HYDRO_ENOMEM, "host allocation failed");
    q->cfg = c;
    *out = q;
    return HYDRO_OK;
}

hydro_status hydro_add_predicate(hydro_query *q, const hydro_udf_desc *udf, double threshold, int32_t *out_pred_id) {
    g_err.clear();
    TRY(check_query(q));
    if (!udf || !out_pred_id) return fail(HYDRO_EINVAL, "NULL argument");
    if (q->finalized) return fail(HYDRO_ESTATE, "predicates must be added before the first submit");
    if ((int)q->preds.size() >= HYDRO_MAX_PREDICATES) return fail(HYDRO_EINVAL, "at most %d predicates", HYDRO_MAX_PREDICATES);
    if (!std::isfinite(threshold)) return fail(HYDRO_EINVAL, "threshold must be finite");
    const hydro_query_config &c = q->cfg;
    const int L = udf->n_layers;
    if (L < 1 || L > HYDRO_MAX_LAYERS || !udf->dims || !udf->weights || !udf->biases)
        return fail(HYDRO_EINVAL, "bad layer description");
    Pred p;
    p.kind = udf->kind;
    p.n_layers = L;
    p.dims.assign(udf->dims, udf->dims + L + 1);
    for (int d : p.dims)
        if (d < 1 || d > 8192) return fail(HYDRO_EINVAL, "layer width out of range");
    if (p.kind == HYDRO_UDF_MLP) {
        if (c.tuple_kind != HYDRO_TUPLE_F32) return fail(HYDRO_EINVAL, "MLP UDFs need F32 tuples");
        const int up = udf->upstream;
        if (up < 0 || up > (int)q->embs.size()) return fail(HYDRO_EINVAL, "unknown embedding id %d", up);
        const int in_dim = up ? q->embs[up - 1].dims.back() : c.dim;
        if (p.dims[0] != in_dim || p.dims[L] != 1)
            return fail(HYDRO_EINVAL, "MLP dims must run from %d to 1", in_dim);
        for (int l = 0; l < L; ++l) {
            if (!udf->weights[l] || !udf->biases[l]) return fail(HYDRO_EINVAL, "NULL weights");
            p.W.emplace_back(udf->weights[l], udf->weights[l] + (size_t)p.dims[l] * p.dims[l + 1]);
            p.b.emplace_back(udf->biases[l], udf->biases[l] + p.dims[l + 1]);
        }
        if (up) {
            // the full UDF is the embedding's layers followed by the head's
            const Emb &e = q->embs[up - 1];
            if (e.n_layers + L > HYDRO_MAX_LAYERS) return fail(HYDRO_EINVAL, "embedding + head too deep");
            long long head_cost = 0;
            for (int l = 0; l < L; ++l) head_cost += 2LL * p.dims[l] * p.dims[l + 1];
            std::vector<int> dims = e.dims;
            dims.insert(dims.end(), p.dims.begin() + 1, p.dims.end());
            std::vector<std::vector<float>> W = e.W, b = e.b;
            W.insert(W.end(), p.W.begin(), p.W.end());
            b.insert(b.end(), p.b.begin(), p.b.end());
            p.dims = dims;
            p.W = W;
            p.b = b;
            p.head_start = e.n_layers;
            p.n_layers = e.n_layers + L;
            p.upstream = up;
            p.cost = udf->cost_hint > 0 ? udf->cost_hint : head_cost;
        }
    } else if (p.kind == HYDRO_UDF_CNN) {
        if (c.tuple_kind != HYDRO_TUPLE_U8_FRAME) return fail(HYDRO_EINVAL, "CNN UDFs need frame tuples");
        if (p.dims[0] != c.channels) return fail(HYDRO_EINVAL, "CNN dims[0] must equal channels");
        if (!udf->head_weight) return fail(HYDRO_EINVAL, "CNN needs head_weight");
        if (!(p.dims[1] == 16 || p.dims[1] == 32 || p.dims[1] == 64))
            return fail(HYDRO_EUNSUPPORTED, "first conv layer must have 16, 32 or 64 channels");
        if ((c.height * c.width) % 128 != 0) return fail(HYDRO_EUNSUPPORTED, "H*W must be a multiple of 128");
        for (int l = 1; l < L; ++l)
            if (p.dims[l] % 16 != 0 || p.dims[l + 1] % 64 != 0)
                return fail(HYDRO_EUNSUPPORTED, "conv layers after the first need Cin %% 16 == 0, Cout %% 64 == 0");
        if (p.dims[L] > 256) return fail(HYDRO_EUNSUPPORTED, "last conv layer wider than 256");
        for (int l = 0; l < L; ++l) {
            if (!udf->weights[l] || !udf->biases[l]) return fail(HYDRO_EINVAL, "NULL weights");
            p.W.emplace_back(udf->weights[l], udf->weights[l] + (size_t)p.dims[l] * p.dims[l + 1] * 9);
            p.b.emplace_back(udf->biases[l], udf->biases[l] + p.dims[l + 1]);
        }
        p.head_w.assign(udf->head_weight, udf->head_weight + p.dims[L]);
        p.head_b = udf->head_bias;
    } else {
        return fail(HYDRO_EINVAL, "unknown UDF kind");
    }
    p.threshold = threshold;
    if (!p.upstream) p.cost = udf->cost_hint > 0 ? udf->cost_hint : model_cost(p, c);
    *out_pred_id = (int32_t)q->preds.size();
    q->preds.push_back(std::move(p));
    return HYDRO_OK;
}

hydro_status hydro_add_embedding(hydro_query *q, const hydro_udf_desc *udf, int64_t id_capacity,
                                 int32_t *out_emb_id) {
    g_err.clear();
    TRY(check_query(q));
    if (!udf || !out_emb_id) return fail(HYDRO_EINVAL, "NULL argument");
    if (q->finalized) return fail(HYDRO_ESTATE, "embeddings must be added before the first submit");
    if ((int)q->embs.size() >= HYDRO_MAX_PREDICATES) return fail(HYDRO_EINVAL, "too many embeddings");
    const hydro_query_config &c = q->cfg;
    if (c.tuple_kind != HYDRO_TUPLE_F32 || udf->kind != HYDRO_UDF_MLP)
        return fail(HYDRO_EINVAL, "embeddings are MLPs on F32 tuples");
    if (c.precision != HYDRO_PREC_FP32) return fail(HYDRO_EUNSUPPORTED, "embeddings need an FP32 query");
    const int L = udf->n_layers;
    if (L < 1 || L > HYDRO_MAX_LAYERS || !udf->dims || !udf->weights || !udf->biases)
        return fail(HYDRO_EINVAL, "bad layer description");
    if (id_capacity < 1 || id_capacity > (1LL << 31)) return fail(HYDRO_EINVAL, "id_capacity out of range");
    Emb e;
    e.n_layers = L;
    e.dims.assign(udf->dims, udf->dims + L + 1);
    for (int d : e.dims)
        if (d < 1 || d > 8192) return fail(HYDRO_EINVAL, "layer width out of range");
    if (e.dims[0] != c.dim) return fail(HYDRO_EINVAL, "embedding input must be the tuple (dims[0] == dim)");
    if (e.dims[L] % 4 != 0) return fail(HYDRO_EINVAL, "embedding width must be a multiple of 4");
    for (int l = 0; l < L; ++l) {
        if (!udf->weights[l] || !udf->biases[l]) return fail(HYDRO_EINVAL, "NULL weights");
        e.W.emplace_back(udf->weights[l], udf->weights[l] + (size_t)e.dims[l] * e.dims[l + 1]);
        e.b.emplace_back(udf->biases[l], udf->biases[l] + e.dims[l + 1]);
    }
    long long cost = 0;
    for (int l = 0; l < L; ++l) cost += 2LL * e.dims[l] * e.dims[l + 1];
    e.cost = udf->cost_hint > 0 ? udf->cost_hint : cost;
    e.cap = id_capacity;
    q->embs.push_back(std::move(e));
    *out_emb_id = (int32_t)q->embs.size();
    return HYDRO_OK;
}

hydro_status hydro_cache_clear(hydro_query *q, int32_t emb) {
    g_err.clear();
    TRY(check_query(q));
    if (q->finalized) TRY(quiesce(q));
    if (emb < 1 || emb > (int)q->embs.size()) return fail(HYDRO_EINVAL, "unknown embedding id %d", emb);
    CU(cudaSetDevice(q->cfg.device));
    TRY(finalize(q));
    Emb &e = q->embs[emb - 1];
    CU(cudaMemsetAsync(e.tags, 0, sizeof(int) * (size_t)e.cap, q->st));
    return HYDRO_OK;
}

hydro_status hydro_cache_prefill(hydro_query *q, int32_t emb, const void *d_tuples, const int64_t *d_ids,
                                 int64_t n) {
    g_err.clear();
    TRY(check_query(q));
    if (q->finalized) TRY(quiesce(q));
    if (emb < 1 || emb > (int)q->embs.size()) return fail(HYDRO_EINVAL, "unknown embedding id %d", emb);
    if (n < 0 || (n > 0 && (!d_tuples || !d_ids))) return fail(HYDRO_EINVAL, "bad tuples/ids");
    CU(cudaSetDevice(q->cfg.device));
    TRY(finalize(q));
    Pred probe;                    // an embedding-only pass: no head
    probe.upstream = emb;
    const int B = q->cfg.max_batch;
    const size_t tb = (size_t)tuple_bytes(q->cfg);
    for (int64_t s = 0; s < n; s += B) {
        const int m = (int)std::min<int64_t>(B, n - s);
        launch_identity_list(q->alive[0], q->ints + 0, 0, m, q->st);
        TRY(run_grouped(q, probe, q->ints + 0, q->alive[0], (const unsigned char *)d_tuples + (size_t)s * tb,
                        (const long long *)d_ids + s, -1, m, q->ints + 5, nullptr));
        CU(cudaGetLastError());
    }
    CU(cudaStreamSynchronize(q->st));
    unsigned int err = 0;
    CU(cudaMemcpy(&err, q->d_err, sizeof err, cudaMemcpyDeviceToHost));
    if (err) return fail(HYDRO_EDEVICE, "device error word 0x%x", err);
    return HYDRO_OK;
}

hydro_status hydro_set_margins(hydro_query *q, int32_t pred, double margin_lowp, double margin_tf32,
                               double margin_fp32) {
    g_err.clear();
    TRY(check_query(q));
    if (pred < 0 || pred >= (int)q->preds.size()) return fail(HYDRO_EINVAL, "unknown predicate");
    if (q->next_batch > 0) return fail(HYDRO_ESTATE, "margins are fixed after the first submit");
    if (!(margin_lowp >= 0.0) || !(margin_tf32 >= 0.0) || !(margin_fp32 >= 0.0))
        return fail(HYDRO_EINVAL, "margins must be >= 0");
    q->preds[pred].margin_lowp = margin_lowp;
    q->preds[pred].margin_tf32 = margin_tf32;
    q->preds[pred].margin_fp32 = margin_fp32;
    return HYDRO_OK;
}

hydro_status hydro_set_static_order(hydro_query *q, const int32_t *order, int32_t n) {
    g_err.clear();
    TRY(check_query(q));
    if (!order || n != (int)q->preds.size()) return fail(HYDRO_EINVAL, "order must list every predicate");
    std::vector<int> seen(n, 0);
    for (int k = 0; k < n; ++k) {
        if (order[k] < 0 || order[k] >= n || seen[order[k]]) return fail(HYDRO_EINVAL, "not a permutation");
        seen[order[k]] = 1;
    }
    q->static_order.assign(order, order + n);
    return HYDRO_OK;
}

hydro_status hydro_udf_scores(hydro_query *q, int32_t pred, int32_t prec, const void *d_tuples, int64_t n,
                              double *d_scores) {
    g_err.clear();
    TRY(check_query(q));
    if (q->finalized) TRY(quiesce(q));
    if (pred < 0 || pred >= (int)q->preds.size()) return fail(HYDRO_EINVAL, "unknown predicate");
    if (n < 0 || (n > 0 && (!d_tuples || !d_scores))) return fail(HYDRO_EINVAL, "bad tuples/scores");
    if (prec != HYDRO_PREC_FP32 && prec != HYDRO_PREC_FP64 && prec != HYDRO_PREC_BF16 && prec != HYDRO_PREC_TF32X3 &&
        prec != HYDRO_PREC_BF16X3)
        return fail(HYDRO_EINVAL, "unknown precision");
    const bool split = prec == HYDRO_PREC_TF32X3 || prec == HYDRO_PREC_BF16X3;
    if ((prec == HYDRO_PREC_BF16 || split) && !tc_query(q->cfg))
        return fail(HYDRO_EINVAL, "BF16, 3xTF32 and split-BF16 scores need a BF16 or split-BF16 query");
    CU(cudaSetDevice(q->cfg.device));
    TRY(finalize(q));
    const Pred &p = q->preds[pred];
    if (split && !p.tc_all) return fail(HYDRO_EINVAL, "split-form scores need a tensor-core CNN UDF");
    const int B = q->cfg.max_batch;
    const bool cnn = p.kind == HYDRO_UDF_CNN;
    const bool recheck_buf = cnn && tc_query(q->cfg) &&
                             (prec == HYDRO_PREC_FP32 || split);
    int *list = q->alive[0], *count = q->ints + 0;
    // 3xTF32 scores need 8 B a channel: half as many frames fit a 4-byte recheck buffer
    const int rchunk = std::max(1, std::min(q->cap1, q->cap2) / (prec == HYDRO_PREC_TF32X3 && q->ract_esz < 8 ? 2 : 1));
    const int chunk = (prec == HYDRO_PREC_FP64 && cnn) ? q->cap3 : recheck_buf ? rchunk : B;
    const size_t tb = (size_t)tuple_bytes(q->cfg);
    for (int64_t s = 0; s < n; s += chunk) {
        const int m = (int)std::min<int64_t>(chunk, n - s);
        const void *base = (const unsigned char *)d_tuples + (size_t)s * tb;
        launch_identity_list(list, count, 0, m, q->st);
        if (prec == HYDRO_PREC_FP64) {
            TRY(run_udf(q, p, PREC_F64, count, list, base, m, cnn ? q->ract64 : q->act, nullptr, d_scores + s));
        } else {
            void *const *act = recheck_buf ? q->ract32 : q->act;
            const int ip = prec == HYDRO_PREC_BF16     ? PREC_BF16
                           : prec == HYDRO_PREC_TF32X3 ? PREC_TF32X3
                           : prec == HYDRO_PREC_BF16X3 ? PREC_BF16X3
                                                       : PREC_F32;
            TRY(run_udf(q, p, ip, count, list, base, m, act, q->score32, nullptr));
            launch_f32_to_f64(q->score32, d_scores + s, m, q->st);
        }
        CU(cudaGetLastError());
    }
    CU(cudaStreamSynchronize(q->st));
    unsigned int err = 0;
    CU(cudaMemcpy(&err, q->d_err, sizeof err, cudaMemcpyDeviceToHost));
    if (err) return fail(HYDRO_EDEVICE, "device error word 0x%x", err);
    return HYDRO_OK;
}

hydro_status hydro_calibrate(hydro_query *q, const void *d_tuples, int64_t n, hydro_calib_info *info) {
    g_err.clear();
    TRY(check_query(q));
    if (q->finalized) TRY(quiesce(q));
    if (n < 1 || !d_tuples) return fail(HYDRO_EINVAL, "need calibration tuples");
    if (q->next_batch > 0) return fail(HYDRO_ESTATE, "calibrate before the first submit");
    double *d = nullptr;
    CU(cudaSetDevice(q->cfg.device));
    TRY(finalize(q));
    CU(cudaMalloc(&d, sizeof(double) * n * 4));
    std::vector<double> s64(n), s32(n), s16(n), stf(n);
    hydro_status rc = HYDRO_OK;
    const bool bf = tc_query(q->cfg);
    for (int i = 0; i < (int)q->preds.size() && rc == HYDRO_OK; ++i) {
        const bool tf = bf && q->preds[i].tc_all;
        rc = hydro_udf_scores(q, i, HYDRO_PREC_FP64, d_tuples, n, d);
        if (rc == HYDRO_OK) rc = hydro_udf_scores(q, i, HYDRO_PREC_FP32, d_tuples, n, d + n);
        if (rc == HYDRO_OK && bf) rc = hydro_udf_scores(q, i, HYDRO_PREC_BF16, d_tuples, n, d + 2 * n);
        // the first recheck level as configured
        const int lv1 = q->cfg.split_precision == HYDRO_PREC_TF32X3 ? HYDRO_PREC_TF32X3 : HYDRO_PREC_BF16X3;
        if (rc == HYDRO_OK && tf) rc = hydro_udf_scores(q, i, lv1, d_tuples, n, d + 3 * n);
        if (rc != HYDRO_OK) break;
        if (cudaMemcpy(s64.data(), d, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(s32.data(), d + n, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess ||
            (bf && cudaMemcpy(s16.data(), d + 2 * n, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess) ||
            (tf && cudaMemcpy(stf.data(), d + 3 * n, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess)) {
            rc = fail(HYDRO_ECUDA, "copy of calibration scores failed");
            break;
        }
        double e32 = 0, e16 = 0, etf = 0, smax = 0;
        for (int64_t k = 0; k < n; ++k) {
            e32 = std::max(e32, std::fabs(s32[k] - s64[k]));
            if (bf) e16 = std::max(e16, std::fabs(s16[k] - s64[k]));
            if (tf) etf = std::max(etf, std::fabs(stf[k] - s64[k]));
            smax = std::max(smax, std::fabs(s64[k]));
        }
        Pred &p = q->preds[i];
        p.margin_fp32 = std::max(16.0 * e32, 1e-9 * smax);
        if (tf) p.margin_tf32 = std::max(8.0 * etf, 1e-9 * smax);
        if (bf && p.margin_lowp < 4.0 * e16) p.margin_lowp = 4.0 * e16;
        if (info) {
            info[i].max_err_fp32 = e32;
            info[i].max_err_lowp = e16;
            info[i].max_err_tf32 = etf;
            info[i].margin_fp32 = p.margin_fp32;
            info[i].margin_lowp = p.margin_lowp;
            info[i].margin_tf32 = p.margin_tf32;
        }
    }
    cudaFree(d);
    return rc;
}

hydro_status hydro_submit_batch(hydro_query *q, const void *d_tuples, const int64_t *d_ids, int64_t n,
                                int64_t *out_batch_id) {
    g_err.clear();
    TRY(check_query(q));
    (void)d_ids;
    if (!out_batch_id) return fail(HYDRO_EINVAL, "NULL out_batch_id");
    if (n < 0 || n > q->cfg.max_batch) return fail(HYDRO_EINVAL, "n=%lld outside 0..max_batch", (long long)n);
    if (n > 0 && !d_tuples) return fail(HYDRO_EINVAL, "NULL tuples");
    if (q->preds.empty()) return fail(HYDRO_ESTATE, "query has no predicates");
    if (!q->embs.empty() && n > 0 && !d_ids) return fail(HYDRO_EINVAL, "a query with an embedding needs tuple ids");
    const hydro_query_config &c = q->cfg;
    if (c.policy == HYDRO_POLICY_STATIC && !q->static_order.empty() && q->static_order.size() != q->preds.size())
        return fail(HYDRO_ESTATE, "static order does not match the predicates");
    CU(cudaSetDevice(c.device));
    TRY(finalize(q));
    Slot *slot = nullptr;
    int slot_idx = 0;
    for (size_t k = 0; k < q->slots.size(); ++k)
        if (!q->slots[k].busy) {
            slot = &q->slots[k];
            slot_idx = (int)k;
            break;
        }
    if (!slot) return fail(HYDRO_EAGAIN, "all %d in-flight slots are busy; poll first", c.max_in_flight);

    const long long b = q->next_batch;
    const int P = (int)q->preds.size();
    const bool eval_all = c.policy == HYDRO_POLICY_ALL || (adaptive(c.policy) && b < c.warmup_batches);
    int order[kMaxPred];
    for (int i = 0; i < P; ++i) order[i] = i;
    if (!eval_all && c.policy == HYDRO_POLICY_STATIC) {
        if (!q->static_order.empty())
            for (int i = 0; i < P; ++i) order[i] = q->static_order[i];
    }
    // routed batch: its order comes from the statistics of batches <= last
    const long long last = b - 1 - c.route_lag;
    const bool routed = !eval_all && c.policy != HYDRO_POLICY_STATIC && last >= 0;
    // device dispatch: the router and the stages run from the lane's batch graph, no host wait
    const bool dev = routed && device_dispatch(q) && !q->prof.on;
    const long long lo = std::max(0LL, last - c.stats_window + 1);
    const int nwv = (int)std::min<long long>(c.warmup_batches, last + 1);
    RouterCosts costs{};
    for (int i = 0; i < P; ++i) {
        costs.c[i] = q->preds[i].cost;
        costs.group[i] = q->preds[i].upstream - 1;
    }
    for (size_t e = 0; e < q->embs.size(); ++e) costs.cemb[e] = q->embs[e].cost;
    costs.n = n;
    costs.measured = c.cost_source == HYDRO_COST_MEASURED ? 1 : 0;
    const int pol = (c.policy == HYDRO_POLICY_RANK || c.policy == HYDRO_POLICY_LEARNED) ? 0
                    : c.policy == HYDRO_POLICY_COST                                      ? 1
                                                                                         : 2;
    if (routed && !dev) {
        {
            int *dord = q->d_order + slot_idx * kMaxPred;
            int *hord = q->h_order + slot_idx * kMaxPred;
            // every lane's latest batch <= last: with lanes, batch last - 1 may finish after batch last
            for (long long x = std::max(0LL, last - q->n_lanes + 1); x <= last; ++x)
                CU(cudaStreamWaitEvent(q->rst, q->ev_done[x % kEvRing], 0));
            if (!q->embs.empty()) {
                // reuse-aware cost: this batch's ids not cached by batches <= last
                CU(cudaMemsetAsync(q->vmiss, 0, sizeof(int) * kMaxPred, q->rst));
                for (size_t e = 0; e < q->embs.size(); ++e) {
                    launch_probe_visible((const long long *)d_ids, (int)n, q->embs[e].tags, q->embs[e].cap, last,
                                         q->vmiss + e, q->rst);
                    q->launches++;
                }
            }
            launch_router(q->ring, q->ring_len, q->warm, nwv, lo, last, P, pol, costs,
                          q->embs.empty() ? nullptr : q->vmiss, dord, q->rst);
            q->launches++;
            CU(cudaGetLastError());
            CU(cudaMemcpyAsync(hord, dord, sizeof(int) * P, cudaMemcpyDeviceToHost, q->rst));
            CU(cudaEventRecord(q->ev_route, q->rst));
            bool done = false;
            TRY(wait_event(q->ev_route, 600000, &done));
            if (!done) return fail(HYDRO_ETIMEOUT, "router of batch %lld did not finish", b);
            for (int i = 0; i < P; ++i) order[i] = hord[i];
            for (int i = 0; i < P; ++i)
                if (order[i] < 0 || order[i] >= P) return fail(HYDRO_EDEVICE, "router produced a bad order");
        }
    }

    if (q->n_lanes > 1) {
        // this batch's lane; it starts after the caller's work so far (its inputs)
        load_lane(q, (int)(b % q->n_lanes));
        CU(cudaEventRecord(q->ev_user, q->home_st));
        if (q->pipe) {
            // the first position's stream; the lane's scratch is free once the batch that
            // used it before (b - lanes) has left the last position
            q->st = q->pos_st[0];
            if (b >= q->n_lanes) CU(cudaStreamWaitEvent(q->st, q->ev_done[(b - q->n_lanes) % kEvRing], 0));
        }
        CU(cudaStreamWaitEvent(q->st, q->ev_user, 0));
    }
    slot->batch = b;
    slot->n = (int)n;
    slot->busy = true;
    slot->warmup = eval_all && c.policy != HYDRO_POLICY_ALL;
    slot->dev = dev;
    std::memcpy(slot->order, order, sizeof order);
    CU(cudaEventRecord(slot->start, q->st));
    if (dev) {
        // the batch into the lane's buffer, the router on this stream once batch `last` is done,
        // then the lane's graph picks every position's predicate from the router's order
        const size_t tb = (size_t)tuple_bytes(c);
        if (n > 0) CU(cudaMemcpyAsync(q->batch_rows, d_tuples, tb * (size_t)n, cudaMemcpyDeviceToDevice, q->st));
        launch_set_int(q->ln, (int)n, q->st);
        for (long long x = std::max(0LL, last - q->n_lanes + 1); x <= last; ++x)
            CU(cudaStreamWaitEvent(q->st, q->ev_done[x % kEvRing], 0));
        launch_router(q->ring, q->ring_len, q->warm, nwv, lo, last, P, pol, costs, nullptr, q->lord, q->st);
        q->launches += 2;
        hydro_status gs = ensure_batch_graph(q);
        if (gs != HYDRO_OK) {
            slot->busy = false;
            q->dead = true;
            return gs;
        }
        CU(cudaGraphLaunch(q->bgraph[q->cur_lane], q->st));
        q->launches += 3;   // initial list, dispatch and result; the bodies are counted on the device
        launch_commit_rows((const StatRow *)(q->lres + kRowsOff), q->ring + (b % q->ring_len) * kMaxPred, P, q->st);
        q->launches++;
        ResHdr *lh = (ResHdr *)q->lres;
        CU(cudaMemcpyAsync(&lh->err, q->d_err, sizeof(unsigned int), cudaMemcpyDeviceToDevice, q->st));
        const size_t bytes = kBitmapOff + sizeof(unsigned int) * (size_t)((n + 31) / 32);
        CU(cudaMemcpyAsync(slot->hres, q->lres, bytes, cudaMemcpyDeviceToHost, q->st));
        CU(cudaEventRecord(slot->done, q->st));
        CU(cudaEventRecord(q->ev_done[b % kEvRing], q->st));
        cudaError_t le = cudaGetLastError();
        if (le != cudaSuccess) {
            q->dead = true;
            return fail(HYDRO_ECUDA, "kernel launch failed: %s", cudaGetErrorString(le));
        }
        q->next_batch = b + 1;
        *out_batch_id = b;
        return HYDRO_OK;
    }
    int *cnt = q->ints;
    int cur = 0;
    const bool learned = c.policy == HYDRO_POLICY_LEARNED;
    if (learned) {
        hydro_status s = run_batch_learned(q, b, order, eval_all, d_tuples, (int)n, *slot, &cur);
        if (s != HYDRO_OK) {
            slot->busy = false;
            q->dead = true;
            return s;
        }
    } else {
        launch_init_alive(q->alive[0], cnt + 0, (int)n, eval_all ? q->acc : nullptr, q->st);
        q->launches++;
    }
    for (int k = 0; k < P && !learned; ++k) {
        if (q->pipe) {
            // position k: its own stream and SM share, after position k - 1 of this batch
            q->st = q->pos_st[k];
            if (k > 0) CU(cudaStreamWaitEvent(q->st, q->ev_stage[q->cur_lane][k - 1], 0));
            q->sms = q->sms_pos;
        }
        hydro_status s = run_stage(q, order[k], cnt + cur, q->alive[cur], q->alive[1 - cur], cnt + 1 - cur, eval_all,
                                   d_tuples, (const long long *)d_ids, (int)n, b, slot);
        if (q->pipe) {
            q->sms = q->sms_full;
            if (s == HYDRO_OK) CU(cudaEventRecord(q->ev_stage[q->cur_lane][k], q->st));
        }
        if (s != HYDRO_OK) {
            slot->busy = false;
            q->dead = true;
            return s;
        }
        if (!eval_all) cur = 1 - cur;
    }
    if (eval_all && !learned) {
        launch_acc_to_alive(q->acc, (int)n, q->alive[1 - cur], cnt + 1 - cur, q->st);
        q->launches++;
        cur = 1 - cur;
    }
    ResHdr *hdr = (ResHdr *)slot->dres;
    launch_result(cnt + cur, q->alive[cur], (int)n, (unsigned int *)(slot->dres + kBitmapOff), &hdr->n_pass, q->st);
    q->launches++;
    CU(cudaMemcpyAsync(&hdr->err, q->d_err, sizeof(unsigned int), cudaMemcpyDeviceToDevice, q->st));
    const size_t bytes = kBitmapOff + sizeof(unsigned int) * (size_t)((n + 31) / 32);
    CU(cudaMemcpyAsync(slot->hres, slot->dres, bytes, cudaMemcpyDeviceToHost, q->st));
    CU(cudaEventRecord(slot->done, q->st));
    CU(cudaEventRecord(q->ev_done[b % kEvRing], q->st));
    if (learned && c.proxy_refresh > 0 && (b + 1) % c.proxy_refresh == 0 && b + 1 > c.warmup_batches)
        TRY(train_proxy(q));
    cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) {
        q->dead = true;
        return fail(HYDRO_ECUDA, "kernel launch failed: %s", cudaGetErrorString(le));
    }
    q->next_batch = b + 1;
    *out_batch_id = b;
    return HYDRO_OK;
}

hydro_status hydro_poll_result(hydro_query *q, int64_t batch_id, uint32_t *pass_bitmap, int64_t *eval_counts,
                               hydro_batch_info *info, int32_t wait_ms) {
    g_err.clear();
    if (!q) return fail(HYDRO_EINVAL, "NULL query");
    Slot *slot = nullptr;
    for (Slot &s : q->slots)
        if (s.busy && s.batch == batch_id) slot = &s;
    if (!slot) return fail(HYDRO_ENOTFOUND, "batch %lld is not in flight", (long long)batch_id);
    if (!pass_bitmap && slot->n > 0) return fail(HYDRO_EINVAL, "NULL pass_bitmap");
    CU(cudaSetDevice(q->cfg.device));
    bool done = false;
    TRY(wait_event(slot->done, wait_ms, &done));
    if (!done) return fail(HYDRO_EAGAIN, "batch %lld not finished", (long long)batch_id);
    const ResHdr *hdr = (const ResHdr *)slot->hres;
    const StatRow *rows = (const StatRow *)(slot->hres + kRowsOff);
    const int P = (int)q->preds.size();
    if (hdr->err) {
        q->latched_err |= hdr->err;
        slot->busy = false;
        return fail(HYDRO_EDEVICE, "device error word 0x%x in batch %lld", hdr->err, (long long)batch_id);
    }
    if (slot->n > 0)
        std::memcpy(pass_bitmap, slot->hres + kBitmapOff, sizeof(uint32_t) * (size_t)((slot->n + 31) / 32));
    if (q->prof.on && batch_id >= q->prof.base) {
        const size_t k = (size_t)(batch_id - q->prof.base);
        if (q->prof.rows.size() <= k) q->prof.rows.resize(k + 1);
        q->prof.rows[k].assign(rows, rows + P);
    }
    for (int i = 0; i < P; ++i) {
        if (eval_counts) eval_counts[i] = rows[i].evaluated;
        q->tot[i][0] += rows[i].evaluated;
        q->tot[i][1] += rows[i].passed;
        q->tot[i][2] += rows[i].recheck32;
        q->tot[i][3] += rows[i].recheck64;
        q->tot[i][4] += rows[i].recheck_tf32;
        q->tot[i][5] += rows[i].hits;
    }
    if (info) {
        std::memset(info, 0, sizeof *info);
        info->n = slot->n;
        info->n_pass = hdr->n_pass;
        info->n_predicates = P;
        info->warmup = slot->warmup ? 1 : 0;
        for (int i = 0; i < P; ++i) {
            info->order[i] = slot->dev ? hdr->order[i] : slot->order[i];
            info->passed[i] = rows[i].passed;
            info->recheck_tf32[i] = rows[i].recheck_tf32;
            info->cache_hits[i] = rows[i].hits;
            info->recheck_fp32[i] = rows[i].recheck32;
            info->recheck_fp64[i] = rows[i].recheck64;
            info->stage_ns[i] = q->cfg.cost_source == HYDRO_COST_MEASURED ? rows[i].ns : 0;
        }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, slot->start, slot->done) == cudaSuccess) info->device_ms = ms;
        else cudaGetLastError();
    }
    slot->busy = false;
    return HYDRO_OK;
}

hydro_status hydro_debug_trace(hydro_query *q, int64_t batch_id, uint8_t *order, uint8_t *visited) {
    g_err.clear();
    TRY(check_query(q));
    if (q->finalized) TRY(quiesce(q));
    if (q->cfg.policy != HYDRO_POLICY_LEARNED) return fail(HYDRO_EUNSUPPORTED, "trace is kept by the learned router");
    if (batch_id != q->last_learned_batch || batch_id != q->next_batch - 1)
        return fail(HYDRO_ENOTFOUND, "trace is only kept for the most recently submitted batch");
    for (const Slot &s : q->slots)
        if (s.busy && s.batch == batch_id) return fail(HYDRO_ESTATE, "poll the batch first");
    CU(cudaSetDevice(q->cfg.device));
    CU(cudaStreamSynchronize(q->st));
    if (q->last_n > 0) {
        if (order) CU(cudaMemcpy(order, q->order_t, (size_t)q->last_n * kMaxPred, cudaMemcpyDeviceToHost));
        if (visited) CU(cudaMemcpy(visited, q->visited, (size_t)q->last_n, cudaMemcpyDeviceToHost));
    }
    return HYDRO_OK;
}

hydro_status hydro_get_stats(hydro_query *q, hydro_pred_stats *out, int32_t n) {
    g_err.clear();
    if (!q || !out) return fail(HYDRO_EINVAL, "NULL argument");
    if (n < 0 || n > (int)q->preds.size()) return fail(HYDRO_EINVAL, "n out of range");
    for (int i = 0; i < n; ++i) {
        out[i].evaluated = q->tot[i][0];
        out[i].passed = q->tot[i][1];
        out[i].recheck_tf32 = q->tot[i][4];
        out[i].cache_hits = q->tot[i][5];
        out[i].recheck_fp32 = q->tot[i][2];
        out[i].recheck_fp64 = q->tot[i][3];
        out[i].model_cost = q->preds[i].cost;
        out[i].margin_lowp = q->preds[i].margin_lowp;
        out[i].margin_tf32 = q->preds[i].margin_tf32 >= 0 ? q->preds[i].margin_tf32
                                                         : 5e-3 * std::max(1.0, std::fabs(q->preds[i].threshold));
        out[i].margin_fp32 = q->preds[i].margin_fp32 >= 0 ? q->preds[i].margin_fp32
                                                         : 1e-5 * std::max(1.0, std::fabs(q->preds[i].threshold));
    }
    return HYDRO_OK;
}

hydro_status hydro_profile(hydro_query *q, int32_t enable) {
    g_err.clear();
    TRY(check_query(q));
    q->prof.on = enable != 0;
    q->prof.recs.clear();
    q->prof.rows.clear();
    q->prof.base = q->next_batch;
    q->launches = 0;
    if (q->d_launch_ctr) {
        // the recheck graphs' body counter: no batch may be running while it is cleared
        TRY(quiesce(q));
        CU(cudaMemset(q->d_launch_ctr, 0, sizeof(unsigned long long)));
    }
    return HYDRO_OK;
}

hydro_status hydro_profile_read(hydro_query *q, hydro_kernel_profile *out, int32_t max, int32_t *n_out,
                                int64_t *total_launches) {
    g_err.clear();
    TRY(check_query(q));
    if (q->finalized) TRY(quiesce(q));
    if (!n_out || (max > 0 && !out)) return fail(HYDRO_EINVAL, "NULL argument");
    if (q->finalized) CU(cudaStreamSynchronize(q->st));
    double ms[PC_N] = {}, fl[PC_N] = {}, by[PC_N] = {};
    long long nl[PC_N] = {};
    for (const ProfRec &r : q->prof.recs) {
        const long long k = r.batch - q->prof.base;
        if (k < 0 || k >= (long long)q->prof.rows.size() || q->prof.rows[k].empty()) continue;   // not polled
        const StatRow &row = q->prof.rows[k][r.pred];
        const long long items = r.src == SRC_MAIN   ? row.evaluated
                                : r.src == SRC_RTF  ? row.recheck_tf32
                                : r.src == SRC_R32  ? row.recheck32
                                : r.src == SRC_MISS ? row.evaluated - row.hits
                                                    : row.recheck64;
        float t = 0.f;
        if (cudaEventElapsedTime(&t, q->prof.ev[r.ev], q->prof.ev[r.ev + 1]) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        ms[r.cls] += t;
        fl[r.cls] += r.fpi * items;
        by[r.cls] += r.bpi * items + (items > 0 ? r.fixed_bytes : 0.0);
        nl[r.cls] += 1;
    }
    int n = 0;
    for (int c = 0; c < PC_N; ++c) {
        if (!nl[c]) continue;
        if (n < max) {
            std::memset(&out[n], 0, sizeof out[n]);
            std::snprintf(out[n].name, sizeof out[n].name, "%s", kProfNames[c]);
            out[n].launches = nl[c];
            out[n].total_ms = ms[c];
            out[n].flops = fl[c];
            out[n].bytes = by[c];
        }
        ++n;
    }
    *n_out = n < max ? n : max;
    long long body = 0;
    if (q->d_launch_ctr) {
        unsigned long long v = 0;
        CU(cudaMemcpy(&v, q->d_launch_ctr, sizeof v, cudaMemcpyDeviceToHost));
        body = (long long)v;
    }
    if (total_launches) *total_launches = q->launches + body;
    return HYDRO_OK;
}

hydro_status hydro_selftest_bounded_wait(int32_t device, int64_t limit_ns) {
    g_err.clear();
    if (limit_ns < 1000 || limit_ns > 10000000000LL) return fail(HYDRO_EINVAL, "limit_ns must be 1e3..1e10");
    CU(cudaSetDevice(device));
    int *d = nullptr;
    CU(cudaMalloc(&d, sizeof(int)));
    int h = -1;
    cudaError_t e = cudaMemset(d, 0xff, sizeof(int));
    if (e == cudaSuccess) e = wait_selftest((unsigned long long)limit_ns, d, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fail(HYDRO_ECUDA, "self-test: %s", cudaGetErrorString(e));
    if (h == 1) return fail(HYDRO_ETIMEOUT, "the wait ran out after %lld ns, as designed", (long long)limit_ns);
    return fail(HYDRO_EDEVICE, "the wait did not run out (status %d)", h);
}

hydro_status hydro_destroy_query(hydro_query *q) {
    g_err.clear();
    if (!q) return fail(HYDRO_EINVAL, "NULL query");
    hydro_status rc = HYDRO_OK;
    if (q->finalized) {
        cudaSetDevice(q->cfg.device);
        // bounded wait for outstanding work
        for (Slot &s : q->slots) {
            if (!s.busy) continue;
            bool done = false;
            if (wait_event(s.done, 60000, &done) != HYDRO_OK || !done) rc = HYDRO_ETIMEOUT;
        }
        if (rc == HYDRO_OK) {
            cudaStreamSynchronize(q->rst);
            for (int l = 0; l < q->n_lanes; ++l)
                if (q->own_lane_st[l]) cudaStreamSynchronize(q->lane_st[l]);
            if (q->n_lanes > 1) q->st = q->home_st;
            if (q->own_stream) cudaStreamSynchronize(q->st);
        }
        if (q->n_lanes > 1) q->st = q->home_st;
        for (int l = 0; l < kMaxLanes; ++l)
            for (int i = 0; i < kMaxPred; ++i) {
                if (q->tail[l][i]) cudaGraphExecDestroy(q->tail[l][i]);
                if (i == 0 && q->bgraph[l]) cudaGraphExecDestroy(q->bgraph[l]);
                if (q->ev_stage[l][i]) cudaEventDestroy(q->ev_stage[l][i]);
            }
        GreenApi g;
        const bool green = q->gctx[0] && green_api(&g);
        for (int k = 0; k < kMaxPred; ++k)
            if (q->pos_st[k]) {
                cudaStreamSynchronize(q->pos_st[k]);
                if (green)
                    g.stream_destroy((CUstream)q->pos_st[k]);
                else
                    cudaStreamDestroy(q->pos_st[k]);
            }
        for (int k = 0; k < kMaxPred; ++k)
            if (q->gctx[k] && green) g.destroy(q->gctx[k]);
        if (q->cap_st) cudaStreamDestroy(q->cap_st);
        for (int k = 0; k < 3; ++k)
            if (q->cap_help[k]) cudaStreamDestroy(q->cap_help[k]);
        tc_conv_destroy(&q->tc);
        for (cudaEvent_t e : q->prof.ev) cudaEventDestroy(e);
        for (Slot &s : q->slots) {
            if (s.hres) cudaFreeHost(s.hres);
            if (s.start) cudaEventDestroy(s.start);
            if (s.done) cudaEventDestroy(s.done);
        }
        if (q->h_order) cudaFreeHost(q->h_order);
        if (q->h_fallback) cudaFreeHost(q->h_fallback);
        for (void *p : q->allocs) cudaFree(p);
        for (int i = 0; i < kEvRing; ++i)
            if (q->ev_done[i]) cudaEventDestroy(q->ev_done[i]);
        if (q->ev_route) cudaEventDestroy(q->ev_route);
        if (q->ev_user) cudaEventDestroy(q->ev_user);
        for (int l = 0; l < kMaxLanes; ++l)
            if (q->own_lane_st[l] && q->lane_st[l]) cudaStreamDestroy(q->lane_st[l]);
        if (q->rst) cudaStreamDestroy(q->rst);
        if (q->own_stream && q->st) cudaStreamDestroy(q->st);
        cudaGetLastError();
    }
    delete q;
    if (rc != HYDRO_OK) return fail(rc, "outstanding batches did not finish before destroy");
    return HYDRO_OK;
}

}  // extern "C"
