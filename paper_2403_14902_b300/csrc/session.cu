// Multi-query sessions: many queries over one pool of MLP UDFs, one step at a
// time, every step a fixed, device-driven launch sequence (replayed from a
// CUDA graph per in-flight slot).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <random>
#include <cstdarg>
#include <cstddef>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "../../include/hydro.h"
#include "common.cuh"
#include "internal.h"
#include "mq.h"
#include "tc_gemm.h"

using namespace hydro;

namespace {

hydro_status fail(hydro_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return s;
}

#define CU(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(e_ == cudaErrorMemoryAllocation ? HYDRO_ENOMEM : HYDRO_ECUDA, "%s: %s", \
                        #call, cudaGetErrorString(e_));                                       \
    } while (0)

#define TRY(x)                         \
    do {                               \
        hydro_status s_ = (x);         \
        if (s_ != HYDRO_OK) return s_; \
    } while (0)

struct Udf {
    int n_layers = 0;
    std::vector<int> dims;
    std::vector<std::vector<float>> W, b;
    long long cost = 0;
    double margin_lowp = 0.02, margin_x3 = 1e-3, margin_fp32 = 1e-5;
    std::vector<float *> dW, db, dWT;
    std::vector<__nv_bfloat16 *> dW16;
    std::vector<__nv_bfloat16 *> dW3;   // split-BF16 weights [N][3K] = [W_hi | W_lo | W_hi]
    std::vector<int> nt;     // tensor-core tile width per hidden layer (0: widest dividing N)
    bool q8 = false;         // FP8 sessions: first layer in E4M3 at level 0
    unsigned char *dW8 = nullptr;   // E4M3 codes of the first layer [N][K]
    float *dsw = nullptr;           // per output channel scale of dW8
    MlpDev mlp{};
};

struct Query {
    int P = 0;
    int udf[kMqSlots] = {};
    double thr[kMqSlots] = {};
};

// Kernel classes of the session profile.
const char *const kSessProf[] = {"gemm_grouped_bf16_tc", "gather_grouped_bf16", "head_finalize_grouped",
                                 "layer_grouped_f32",    "dot_grouped_f32",     "band_f64",
                                 "route_partition_classify"};
enum { SP_GEMM = 0, SP_GATHER, SP_FINAL, SP_LAYER, SP_DOT, SP_BAND64, SP_CTRL, SP_N };

struct ProfRec {
    int cls;
    cudaEvent_t a, b;
};

struct Slot {
    std::vector<ProfRec> prof;     // this step's timed launches (profiling on)
    long long launches = 0;        // launches outside conditional regions (all, without a graph)
    long long gate_body[kMqGates] = {};   // launches inside each conditional region
    bool conditional = false;
    int *gates = nullptr;          // device copy of the step's condition values
    bool busy = false;
    long long step = -1;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaGraphExec_t exec = nullptr;
    StepHdr *h_hdr = nullptr;      // pinned
    unsigned int *bitmap = nullptr;
    StatRow *rows = nullptr;
    unsigned char *order = nullptr, *evall = nullptr;
    long long *bidx = nullptr, *npass = nullptr;
    int *total = nullptr;
    std::vector<int> counts;
    // load balance of the grouped launches: per launch of the step, the data-aware
    // scheduler's counters and every CTA's {first, last} global-timer stamps
    int *sched = nullptr;
    unsigned long long *rec = nullptr;
    int n_rec = 0;
};

constexpr int kRecLaunches = 128;                // grouped launches per step with counters and records
constexpr int kRecCtas = HYDRO_BALANCE_CTAS;

}  // namespace

struct hydro_session {
    hydro_session_config cfg{};
    std::vector<Udf> udfs;
    std::vector<Query> queries;
    bool finalized = false, dead = false, own_stream = false;
    int sms = 0, wmax = 0, max_hidden = 0, maxP = 0;
    cudaStream_t st = nullptr;
    std::vector<void *> allocs;
    std::vector<void *> host_allocs;
    MqDev d{};
    MqHist h{};
    StepHdr *d_hdr = nullptr;
    float *act32[2] = {};
    __nv_bfloat16 *stage16 = nullptr, *act16[2] = {};
    __nv_bfloat16 *stage3 = nullptr, *act3[2] = {};   // split-BF16 operands (3x the columns)
    unsigned char *stage8 = nullptr;   // FP8 sessions: E4M3 level-0 operand rows [cap][dim]
    float *ascale = nullptr;           // and their scales [cap]
    unsigned q8_mask = 0;              // pool UDFs in the FP8 set
    float *partials = nullptr;
    int pstride = 1;
    void *encode = nullptr;
    float *d_margin[LV_F64] = {};
    GroupedMlps mlps{};
    std::vector<Slot> slots;
    long long next_step = 0;
    std::vector<hydro_tile_choice> tuning;
    // profiling (hydro_session_profile): per class launches and device ms
    bool prof_on = false;
    Slot *prof_slot = nullptr;
    double prof_ms[SP_N] = {};
    long long prof_n[SP_N] = {};
    long long launches = 0;         // kernel launches of polled steps since profiling was (re)started
    long long step_launches = 0;    // launches of the step being enqueued (current region)
    // load balance (hydro_session_balance)
    Slot *cur_slot = nullptr;       // the slot whose step is being enqueued
    int rec_idx = 0;                // its grouped launches so far
    bool bal_on = false;
    hydro_balance_info bal{};
    // graph capture with conditional regions
    bool capturing = false;
    int if_depth = 0;
    cudaStream_t helper[2] = {};
    std::vector<long long> frames;
    unsigned long long handles[kMqGates] = {};   // created on first use (an unused handle fails instantiation)
    cudaGraph_t cap_graph = nullptr;
    hydro_status handle_err = HYDRO_OK;
    // learned routing (one query): proxy D -> H -> P, its training state and ring of outcomes
    int ph = 0;
    float *pW1 = nullptr, *pb1 = nullptr, *pW2 = nullptr, *pb2 = nullptr;
    float *pg = nullptr, *pm = nullptr, *pv = nullptr;
    float *pH = nullptr, *pZ = nullptr, *pdZ = nullptr, *pdH = nullptr, *pinv = nullptr, *ppart = nullptr;
    int *p_ready = nullptr, *p_count = nullptr, *p_rows = nullptr;
    // tensor-core proxy forward (BF16 sessions, hidden width a multiple of 64): BF16 copy of
    // the first layer's FP32 master weights, refreshed after every training, and its output
    bool proxy_tc = false;
    __nv_bfloat16 *pW1_16 = nullptr, *pH16 = nullptr;
    int *p_hrows = nullptr;               // device: H (rows of pW1 for the conversion)
    int *h_one = nullptr;                 // pinned 1
    float *ringX = nullptr;
    unsigned char *ringL = nullptr, *ringM = nullptr;
    std::vector<int> ring_n;
    long long learned_batches = 0, learned_steps = 0;
    long long train_off = 0;              // start of the next training window (proxy_rows)
    // Training runs on its own stream, overlapping the next step.  Steps read an inference
    // copy of the parameters (iW1 | ib1 | iW2 | ib2), refreshed from the FP32 masters on the
    // step stream at the second submit after the step that launched the training (waiting for
    // it): the weights a step uses depend on the submission order only.
    cudaStream_t train_st = nullptr;
    cudaEvent_t ev_ring = nullptr, ev_trained = nullptr;
    bool train_pending = false;
    long long train_step = -1;            // step after which the pending training was launched
    float *iparams = nullptr, *iW1 = nullptr, *ib1 = nullptr, *iW2 = nullptr, *ib2 = nullptr;
    size_t nparam = 0;
    float *tH = nullptr, *tZ = nullptr;   // training activations and logits
    int adam_t = 0;
    long long last_step_total = -1;       // stacked tuples of the most recent step (debug trace)
};

namespace {

template <typename T>
hydro_status dalloc(hydro_session *s, T **p, size_t bytes) {
    void *v = nullptr;
    CU(cudaMalloc(&v, bytes < 16 ? 16 : bytes));
    s->allocs.push_back(v);
    *p = (T *)v;
    return HYDRO_OK;
}

template <typename T>
hydro_status upload(hydro_session *s, T **dst, const T *src, size_t count) {
    TRY(dalloc(s, dst, count * sizeof(T)));
    CU(cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice));
    return HYDRO_OK;
}

hydro_status check(hydro_session *s) {
    if (!s) return fail(HYDRO_EINVAL, "NULL session");
    if (s->dead) return fail(HYDRO_ESTATE, "session is in a failed state");
    return HYDRO_OK;
}

// BF16 and FP8 sessions run the tensor-core levels
bool bf16(const hydro_session *s) { return s->cfg.precision == HYDRO_PREC_BF16 || s->cfg.precision == HYDRO_PREC_FP8; }
bool fp8(const hydro_session *s) { return s->cfg.precision == HYDRO_PREC_FP8; }

// Bracket the launches of one class with events (profiling steps only).
int prof_begin(hydro_session *s, int cls) {
    if (!s->prof_slot) return -1;
    ProfRec r{cls, nullptr, nullptr};
    if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) return -1;
    cudaEventRecord(r.a, s->st);
    s->prof_slot->prof.push_back(r);
    return (int)s->prof_slot->prof.size() - 1;
}
void prof_end(hydro_session *s, int i) {
    if (i >= 0 && s->prof_slot) cudaEventRecord(s->prof_slot->prof[i].b, s->st);
}

// Device address of one level's per-group list lengths.
int *rc_n(const MqDev &d, int level) {
    return reinterpret_cast<int *>(reinterpret_cast<char *>(d.rc) + offsetof(RoundCounters, n)) + level * kMqPool;
}

// Rows of all lists of a level as one stacked operand: the layers of one
// depth for every group in one launch (BF16 on the tensor cores; split3: the
// split-BF16 form, operands [hi | hi | lo] against [W_hi | W_lo | W_hi]).
// heads_out: return the heads and leave the head partials for a fused
// classify (no finalize launch); else finalize into score.
// q8: level 0 of an FP8 session (the FP8 set's first layers in E4M3).
hydro_status eval_tc(hydro_session *s, const int *counts, const int *lists, float *score, bool split3,
                     int min_rows = 0, TcHeads *heads_out = nullptr, bool q8 = false) {
    const MqDev &d = s->d;
    const int x = split3 ? 3 : 1;
    q8 = q8 && !split3 && s->q8_mask;
    __nv_bfloat16 *stage = split3 ? s->stage3 : s->stage16;
    __nv_bfloat16 *const *act = split3 ? s->act3 : s->act16;
    int pe = prof_begin(s, SP_GATHER);
    if (q8)
        launch_gather_grouped_mixed(d.G, counts, lists, d.cap, reinterpret_cast<const float *const *>(s->d_hdr),
                                    d.dim, d.dim, s->q8_mask, stage, s->stage8, s->ascale, d.cap, s->sms, s->st);
    else if (split3)
        launch_gather_grouped_bf16x3(d.G, counts, lists, d.cap, reinterpret_cast<const float *const *>(s->d_hdr),
                                     d.dim, d.dim, stage, d.cap, s->sms, s->st, min_rows);
    else
        launch_gather_grouped_bf16(d.G, counts, lists, d.cap, reinterpret_cast<const float *const *>(s->d_hdr), d.dim,
                                   d.dim, stage, d.cap, s->sms, s->st);
    prof_end(s, pe);
    s->step_launches++;
    TcHeads heads{};
    for (int dd = 0; dd < s->max_hidden; ++dd) {
        TcGemmGroup gr[kMaxGroups];
        for (int g = 0; g < d.G; ++g) {
            const Udf &u = s->udfs[g];
            const bool has = dd + 1 < u.n_layers;
            const bool head = dd + 2 == u.n_layers;
            gr[g] = TcGemmGroup{counts + g,
                                dd == 0 ? stage : act[(dd - 1) % 2],
                                x * (dd == 0 ? d.dim : s->wmax),
                                d.cap,
                                has ? (split3 ? u.dW3[dd] : u.dW16[dd]) : nullptr,
                                has ? u.db[dd] : nullptr,
                                head ? u.dW[u.n_layers - 1] : nullptr,
                                has ? x * u.dims[dd] : 0,
                                has ? u.dims[dd + 1] : 0,
                                has ? u.nt[dd] : 0};
            if (q8 && dd == 0 && u.q8) {
                gr[g].W = nullptr;
                gr[g].X8 = s->stage8;
                gr[g].W8 = u.dW8;
                gr[g].ascale = s->ascale;
                gr[g].wscale = u.dsw;
            }
            if (head) {
                heads.b[g] = u.b[u.n_layers - 1][0];
                heads.tiles[g] = tc_gemm_head_parts(u.dims[dd + 1], u.nt[dd]);
            }
        }
        // a step's launches get their own scheduler counters and balance records
        TcSched ts;
        const TcSched *tsp = nullptr;
        if (s->cur_slot && s->rec_idx < kRecLaunches && s->sms <= kRecCtas) {
            ts.data_aware = s->cfg.tile_sched;
            ts.counters = s->cur_slot->sched + 2 * s->rec_idx;
            ts.rec = s->cur_slot->rec + (size_t)s->rec_idx * kRecCtas * 2;
            tsp = &ts;
            ++s->rec_idx;
        }
        pe = prof_begin(s, SP_GEMM);
        hydro_status rs = tc_gemm_grouped_run(s->encode, gr, d.G, act[dd % 2], x * s->wmax, s->partials, s->pstride,
                                              s->sms, s->st, d.err, split3, min_rows, tsp);
        prof_end(s, pe);
        if (rs != HYDRO_OK) return fail(rs, "grouped tensor-core GEMM: %s", tc_gemm_last_error());
        s->step_launches++;
    }
    if (heads_out) {
        *heads_out = heads;
        return HYDRO_OK;
    }
    pe = prof_begin(s, SP_FINAL);
    launch_head_finalize_grouped(d.G, counts, heads, s->partials, s->pstride, score, d.cap, d.cap, s->sms, s->st,
                                 min_rows);
    prof_end(s, pe);
    s->step_launches++;
    return HYDRO_OK;
}

// The same in FP32 on the CUDA cores (hidden layers per depth, then the
// one-output layer).
void eval_f32(hydro_session *s, const int *counts, const int *lists, float *score) {
    const MqDev &d = s->d;
    for (int dd = 0; dd < s->max_hidden; ++dd) {
        MqLayers L{};
        L.n = d.G;
        L.counts = counts;
        L.rows = dd == 0 ? lists : nullptr;
        L.cap = d.cap;
        L.hdr = s->d_hdr;
        L.ldx = d.dim;
        L.Y = s->act32[dd % 2];
        L.ldy = s->wmax;
        for (int g = 0; g < d.G; ++g) {
            const Udf &u = s->udfs[g];
            if (dd + 1 >= u.n_layers) continue;
            L.l[g] = MqLayer{u.dW[dd], u.db[dd], 0.f, dd == 0 ? nullptr : s->act32[(dd - 1) % 2], s->wmax,
                             u.dims[dd], u.dims[dd + 1]};
        }
        const int pe = prof_begin(s, SP_LAYER);
        mq_launch_layers_f32(L, s->st, s->sms);
        prof_end(s, pe);
        s->step_launches++;
    }
    MqLayers L{};
    L.n = d.G;
    L.counts = counts;
    L.rows = nullptr;
    L.cap = d.cap;
    L.hdr = s->d_hdr;
    L.ldx = d.dim;
    for (int g = 0; g < d.G; ++g) {
        const Udf &u = s->udfs[g];
        const int last = u.n_layers - 1;
        L.l[g] = MqLayer{u.dW[last], nullptr, u.b[last][0], s->act32[(last - 1) % 2], s->wmax, u.dims[last], 1};
    }
    const int pe = prof_begin(s, SP_DOT);
    mq_launch_dots_f32(L, score, d.cap, s->st, s->sms);
    prof_end(s, pe);
    s->step_launches++;
}

// Conditional regions of a captured step.  In graph mode each round is an
// IF node (run while tuples are alive) and inside it the split-BF16, FP32
// and FP64 levels are IF nodes (run when their band is not empty); the
// kernel before each node sets its condition on the device.  Bodies are
// captured on helper streams.  Launch accounting: launches inside a body
// are counted for that body's gate, the rest for every step.
hydro_status open_if(hydro_session *s, Slot &slot, int gate, cudaStream_t *saved) {
    if (!s->capturing) return HYDRO_OK;
    if (!s->handles[gate] || s->handle_err != HYDRO_OK) return fail(HYDRO_ECUDA, "conditional region without handle");
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *ed = nullptr;
    size_t nd = 0;
    CU(cudaStreamGetCaptureInfo(s->st, &cs, nullptr, &g, &deps, &ed, &nd));
    alignas(cudaGraphNodeParams) unsigned char pbuf[sizeof(cudaGraphNodeParams)];
    memset(pbuf, 0, sizeof pbuf);
    cudaGraphNodeParams &p = *reinterpret_cast<cudaGraphNodeParams *>(pbuf);   // zeroed, as the API requires
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = s->handles[gate];
    p.conditional.type = cudaGraphCondTypeIf;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    CU(cudaGraphAddNode(&node, g, deps, ed, nd, &p));
    CU(cudaStreamUpdateCaptureDependencies(s->st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    if (s->if_depth >= 2) return fail(HYDRO_ECUDA, "conditional regions nest at most twice");
    cudaStream_t hs = s->helper[s->if_depth++];
    CU(cudaStreamBeginCaptureToGraph(hs, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                     cudaStreamCaptureModeThreadLocal));
    *saved = s->st;
    s->st = hs;
    s->frames.push_back(s->step_launches);
    s->step_launches = 0;
    (void)slot;
    return HYDRO_OK;
}

hydro_status close_if(hydro_session *s, Slot &slot, int gate, cudaStream_t saved) {
    if (!s->capturing) return HYDRO_OK;
    cudaGraph_t out = nullptr;
    CU(cudaStreamEndCapture(s->st, &out));
    s->st = saved;
    s->if_depth--;
    slot.gate_body[gate] = s->step_launches;
    s->step_launches = s->frames.back();
    s->frames.pop_back();
    return HYDRO_OK;
}

Cond cond_of(hydro_session *s, int gate) {
    Cond c;
    if (s->capturing) {
        if (!s->handles[gate]) {
            cudaGraphConditionalHandle h;
            if (cudaGraphConditionalHandleCreate(&h, s->cap_graph, 0, cudaGraphCondAssignDefault) != cudaSuccess)
                s->handle_err = fail(HYDRO_ECUDA, "conditional handle create failed");
            else
                s->handles[gate] = (unsigned long long)h;
        }
        c.h = s->handles[gate];
        c.flag = s->d.gates + gate;
    }
    return c;
}

// One step's launches, all stream-ordered on s->st (captured into a graph
// when graphs are on).
hydro_status enqueue_step(hydro_session *s, Slot &slot) {
    const MqDev &d = s->d;
    const bool bf = bf16(s);
    auto gate = [](int r, int k) { return 4 * r + k; };   // k: 0 round, 1 split, 2 FP32 band, 3 FP64 band
    CU(cudaMemcpyAsync(s->d_hdr, slot.h_hdr, sizeof(StepHdr), cudaMemcpyHostToDevice, s->st));
    // balance records of this step: launches that do not run (empty rounds) leave zeros
    CU(cudaMemsetAsync(slot.rec, 0, sizeof(unsigned long long) * 2 * kRecCtas * kRecLaunches, s->st));
    s->cur_slot = &slot;
    s->rec_idx = 0;
    s->step_launches = 0;
    s->frames.clear();
    for (int k = 0; k < kMqGates; ++k) slot.gate_body[k] = 0;
    int pe = prof_begin(s, SP_CTRL);
    mq_launch_init(d, s->st, s->sms, cond_of(s, gate(0, 0)));
    mq_launch_router(d, s->h, s->st);
    prof_end(s, pe);
    s->step_launches += 2;
    if (s->cfg.learned) {
        // proxy logits of every tuple (identity rows of the first alive list), then each tuple's order
        const int P = s->queries[0].P;
        MqLayers L1{};
        L1.n = 1;
        L1.counts = &d.rc->alive[0];
        L1.rows = d.alive[0];
        L1.cap = d.cap;
        L1.hdr = s->d_hdr;
        L1.ldx = d.dim;
        L1.Y = s->pH;
        L1.ldy = s->ph;
        L1.l[0] = MqLayer{s->iW1, s->ib1, 0.f, nullptr, 0, d.dim, s->ph, 0};
        MqLayers L2 = L1;
        L2.rows = nullptr;
        L2.Y = s->pZ;
        L2.ldy = P;
        L2.l[0] = MqLayer{s->iW2, s->ib2, 0.f, s->pH, s->ph, s->ph, P, 1};
        if (s->proxy_tc) {
            // BF16 rows -> tensor-core hidden layer (ReLU, stored BF16) -> logits
            pe = prof_begin(s, SP_GATHER);
            launch_gather_grouped_bf16(1, &d.rc->alive[0], d.alive[0], d.cap,
                                       reinterpret_cast<const float *const *>(s->d_hdr), d.dim, d.dim, s->stage16,
                                       d.cap, s->sms, s->st);
            prof_end(s, pe);
            TcGemmGroup g{&d.rc->alive[0], s->stage16, d.dim, d.cap, s->pW1_16, s->ib1, nullptr, d.dim, s->ph, 64};
            pe = prof_begin(s, SP_GEMM);
            hydro_status rs = tc_gemm_grouped_run(s->encode, &g, 1, s->pH16, s->ph, s->partials, s->pstride, s->sms,
                                                  s->st, d.err);
            prof_end(s, pe);
            if (rs != HYDRO_OK) return fail(rs, "proxy layer: %s", tc_gemm_last_error());
            pe = prof_begin(s, SP_CTRL);
            mq_launch_proxy_out(&d.rc->alive[0], s->pH16, s->ph, s->iW2, s->ib2, P, s->pZ, P, d.cap, s->st, s->sms);
        } else {
            pe = prof_begin(s, SP_CTRL);
            mq_launch_layers_f32(L1, s->st, s->sms);
            mq_launch_layers_f32(L2, s->st, s->sms);
        }
        mq_launch_tuple_order(d, s->pZ, P, s->p_ready, s->st, s->sms);
        prof_end(s, pe);
        s->step_launches += s->proxy_tc ? 4 : 3;
    }
    auto classify = [&](int r, int in, int out, Cond next, int next_min, const TcHeads *heads = nullptr) {
        const int p = prof_begin(s, SP_CTRL);
        mq_launch_classify(d, r, in, out, s->st, s->sms, next, next_min, heads, heads ? s->partials : nullptr,
                           s->pstride);
        prof_end(s, p);
        s->step_launches++;
    };
    TcHeads heads{};
    cudaStream_t sv_round = nullptr, sv = nullptr;
    for (int r = 0; r < s->maxP; ++r) {
        TRY(open_if(s, slot, gate(r, 0), &sv_round));
        pe = prof_begin(s, SP_CTRL);
        mq_launch_partition(d, r, s->st, s->sms);
        prof_end(s, pe);
        s->step_launches++;
        if (bf) {
            TRY(eval_tc(s, rc_n(d, LV_MAIN), d.list[LV_MAIN], d.score[LV_MAIN], false, 0, &heads, true));
            classify(r, LV_MAIN, LV_X3, cond_of(s, gate(r, 1)), kMinSplitRows, &heads);
            TRY(open_if(s, slot, gate(r, 1), &sv));
            // level 1: split BF16 (BF16 sessions) or BF16 (the FP8 set of FP8 sessions)
            TRY(eval_tc(s, rc_n(d, LV_X3), d.list[LV_X3], d.score[LV_X3], !fp8(s), kMinSplitRows, &heads));
            TRY(close_if(s, slot, gate(r, 1), sv));
            // decides the split level's entries, or forwards them all when it was skipped
            classify(r, LV_X3, LV_F32, cond_of(s, gate(r, 2)), 1, &heads);
            TRY(open_if(s, slot, gate(r, 2), &sv));
            pe = prof_begin(s, SP_LAYER);
            mq_launch_band32(d, r, s->mlps, s->max_hidden, s->act32[0], s->act32[1], s->wmax, s->st, s->sms,
                             cond_of(s, gate(r, 3)));
            prof_end(s, pe);
            s->step_launches += s->max_hidden + 1;
            TRY(close_if(s, slot, gate(r, 2), sv));
        } else {
            eval_f32(s, rc_n(d, LV_MAIN), d.list[LV_MAIN], d.score[LV_MAIN]);
            classify(r, LV_MAIN, LV_F64, cond_of(s, gate(r, 3)), 1);
        }
        TRY(open_if(s, slot, gate(r, 3), &sv));
        pe = prof_begin(s, SP_BAND64);
        mq_launch_band64(d, r, s->mlps, s->max_hidden, s->st, s->sms);
        prof_end(s, pe);
        s->step_launches += s->max_hidden + 2;
        TRY(close_if(s, slot, gate(r, 3), sv));
        pe = prof_begin(s, SP_CTRL);
        mq_launch_survivors(d, r, s->st, s->sms, r + 1 < s->maxP ? cond_of(s, gate(r + 1, 0)) : Cond());
        prof_end(s, pe);
        s->step_launches++;
        TRY(close_if(s, slot, gate(r, 0), sv_round));
    }
    pe = prof_begin(s, SP_CTRL);
    mq_launch_result(d, slot.bitmap, s->st, s->sms);
    mq_launch_commit(d, s->h, slot.rows, slot.order, slot.evall, slot.bidx, slot.npass, slot.total, slot.gates,
                     s->st);
    prof_end(s, pe);
    s->step_launches += 2;
    slot.launches = s->step_launches;
    slot.conditional = s->capturing;
    slot.n_rec = s->rec_idx;
    s->cur_slot = nullptr;
    CU(cudaGetLastError());
    return HYDRO_OK;
}

hydro_status autotune(hydro_session *s) {
    // time every tile width of every hidden layer on a stacked operand of
    // min(cap, 16384) rows (one group), keep the fastest
    const int rows = std::min(s->d.cap, 16384);
    int *d_rows = nullptr;
    TRY(dalloc(s, &d_rows, sizeof(int)));
    CU(cudaMemcpy(d_rows, &rows, sizeof(int), cudaMemcpyHostToDevice));
    CU(cudaMemset(s->stage16, 0, sizeof(__nv_bfloat16) * (size_t)s->d.cap * s->d.dim));
    CU(cudaMemset(s->act16[0], 0, sizeof(__nv_bfloat16) * (size_t)s->d.cap * s->wmax));
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    // the first pass (the first UDF's layers) only warms up: the first width timed in a
    // process read 30x slower than the same launch later; the second pass is kept
    for (int pass = 0; pass < 2; ++pass)
    for (size_t ui = 0; ui < (pass ? s->udfs.size() : std::min<size_t>(1, s->udfs.size())); ++ui) {
        Udf &u = s->udfs[ui];
        for (int l = 0; l + 1 < u.n_layers; ++l) {
            hydro_tile_choice rec{};
            rec.udf = (int)ui;
            rec.layer = l;
            rec.K = u.dims[l];
            rec.N = u.dims[l + 1];
            double best = 1e30;
            int best_nt = 0;
            for (int k = 0; k < 3; ++k) {
                const int nt = 64 << k;
                if (rec.N % nt) continue;
                TcGemmGroup g{d_rows, l == 0 ? s->stage16 : s->act16[0], l == 0 ? s->d.dim : s->wmax, s->d.cap,
                              u.dW16[l], u.db[l], nullptr, rec.K, rec.N, nt};
                float ms = 0;
                for (int rep = 0; rep < 4; ++rep) {
                    if (rep == 1) CU(cudaEventRecord(e0, s->st));
                    hydro_status rs = tc_gemm_grouped_run(s->encode, &g, 1, s->act16[1], s->wmax, s->partials,
                                                          s->pstride, s->sms, s->st, s->d.err);
                    if (rs != HYDRO_OK) return fail(rs, "autotune: %s", tc_gemm_last_error());
                }
                CU(cudaEventRecord(e1, s->st));
                CU(cudaEventSynchronize(e1));
                CU(cudaEventElapsedTime(&ms, e0, e1));
                rec.us[k] = ms * 1000.0 / 3.0;
                if (rec.us[k] < best) {
                    best = rec.us[k];
                    best_nt = nt;
                }
            }
            if (!pass) continue;
            u.nt[l] = best_nt;
            rec.tile_n = best_nt;
            s->tuning.push_back(rec);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    unsigned int err = 0;
    CU(cudaMemcpy(&err, s->d.err, sizeof err, cudaMemcpyDeviceToHost));
    if (err) return fail(HYDRO_EDEVICE, "device error word 0x%x during autotuning", err);
    return HYDRO_OK;
}

hydro_status finalize(hydro_session *s) {
    if (s->finalized) return HYDRO_OK;
    const hydro_session_config &c = s->cfg;
    if (s->udfs.empty()) return fail(HYDRO_ESTATE, "session has no UDFs");
    if (s->queries.empty()) return fail(HYDRO_ESTATE, "session has no queries");
    CU(cudaSetDevice(c.device));
    CU(cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, c.device));
    if (c.stream) {
        s->st = (cudaStream_t)c.stream;
    } else {
        CU(cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking));
        s->own_stream = true;
    }
    const int NQ = (int)s->queries.size(), G = (int)s->udfs.size(), cap = c.max_step_tuples;
    const int K = c.batches_per_step, Q = NQ * K;   // Q: batches of one step (virtual queries)
    s->wmax = 64;
    s->max_hidden = 0;
    for (const Udf &u : s->udfs) {
        s->max_hidden = std::max(s->max_hidden, u.n_layers - 1);
        for (int l = 1; l < u.n_layers; ++l) s->wmax = std::max(s->wmax, u.dims[l]);
    }
    s->maxP = 0;
    for (const Query &q : s->queries) s->maxP = std::max(s->maxP, q.P);

    // weights
    s->mlps.max_width = std::max(s->wmax, c.dim);
    for (int g = 0; g < G; ++g) {
        Udf &u = s->udfs[g];
        u.dW.assign(u.n_layers, nullptr);
        u.db.assign(u.n_layers, nullptr);
        u.dWT.assign(u.n_layers, nullptr);
        u.dW16.assign(u.n_layers, nullptr);
        u.dW3.assign(u.n_layers, nullptr);
        u.nt.assign(u.n_layers, 0);
        for (int l = 0; l < u.n_layers; ++l) {
            TRY(upload(s, &u.dW[l], u.W[l].data(), u.W[l].size()));
            TRY(upload(s, &u.db[l], u.b[l].data(), u.b[l].size()));
            {
                const int K = u.dims[l], N = u.dims[l + 1];
                std::vector<float> wt((size_t)K * N);
                for (int n = 0; n < N; ++n)
                    for (int k = 0; k < K; ++k) wt[(size_t)k * N + n] = u.W[l][(size_t)n * K + k];
                TRY(upload(s, &u.dWT[l], wt.data(), wt.size()));
            }
            if (bf16(s) && l + 1 < u.n_layers) {
                const int K = u.dims[l], N = u.dims[l + 1];
                std::vector<__nv_bfloat16> w16(u.W[l].size()), w3((size_t)N * 3 * K);
                for (int n = 0; n < N; ++n)
                    for (int k = 0; k < K; ++k) {
                        const float v = u.W[l][(size_t)n * K + k];
                        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
                        const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
                        w16[(size_t)n * K + k] = hi;
                        w3[(size_t)n * 3 * K + k] = hi;
                        w3[(size_t)n * 3 * K + K + k] = lo;
                        w3[(size_t)n * 3 * K + 2 * K + k] = hi;
                    }
                TRY(upload(s, &u.dW16[l], w16.data(), w16.size()));
                TRY(upload(s, &u.dW3[l], w3.data(), w3.size()));
            }
        }
        u.mlp.n_layers = u.n_layers;
        u.mlp.max_width = s->mlps.max_width;
        for (int l = 0; l <= u.n_layers; ++l) u.mlp.dims[l] = u.dims[l];
        for (int l = 0; l < u.n_layers; ++l) {
            u.mlp.W[l] = u.dW[l];
            u.mlp.b[l] = u.db[l];
            u.mlp.WT[l] = u.dWT[l];
        }
        s->mlps.m[g] = u.mlp;
    }
    CU(mq_band_smem_setup(s->mlps.max_width));

    // query tables
    std::vector<unsigned char> np(NQ), udf((size_t)NQ * kMqSlots, 0);
    std::vector<double> thr((size_t)NQ * kMqSlots, 0.0);
    std::vector<long long> cost((size_t)NQ * kMqSlots, 0);
    for (int q = 0; q < NQ; ++q) {
        np[q] = (unsigned char)s->queries[q].P;
        for (int k = 0; k < s->queries[q].P; ++k) {
            udf[(size_t)q * kMqSlots + k] = (unsigned char)s->queries[q].udf[k];
            thr[(size_t)q * kMqSlots + k] = s->queries[q].thr[k];
            cost[(size_t)q * kMqSlots + k] = s->udfs[s->queries[q].udf[k]].cost;
        }
    }
    MqDev &d = s->d;
    d.Q = Q;
    d.K = K;
    d.G = G;
    d.cap = cap;
    d.dim = c.dim;
    unsigned char *np_d, *udf_d;
    double *thr_d;
    long long *cost_d;
    TRY(upload(s, &np_d, np.data(), np.size()));
    TRY(upload(s, &udf_d, udf.data(), udf.size()));
    TRY(upload(s, &thr_d, thr.data(), thr.size()));
    TRY(upload(s, &cost_d, cost.data(), cost.size()));
    d.np = np_d;
    d.udf = udf_d;
    d.thr = thr_d;
    d.cost = cost_d;
    TRY(dalloc(s, &s->d_hdr, sizeof(StepHdr)));
    d.hdr = s->d_hdr;
    TRY(dalloc(s, &d.off, sizeof(int) * (Q + 1)));
    TRY(dalloc(s, &d.qid, sizeof(unsigned short) * (size_t)cap));
    TRY(dalloc(s, &d.order, (size_t)Q * kMqSlots));
    TRY(dalloc(s, &d.evall, (size_t)Q));
    TRY(dalloc(s, &d.bidx, sizeof(long long) * Q));
    TRY(dalloc(s, &d.rows, sizeof(StatRow) * Q * kMqSlots));
    TRY(dalloc(s, &d.npass, sizeof(long long) * Q));
    TRY(dalloc(s, &d.visited, (size_t)cap));
    TRY(dalloc(s, &d.label, (size_t)cap));
    TRY(dalloc(s, &d.ok, (size_t)cap));
    TRY(dalloc(s, &d.alive[0], sizeof(int) * (size_t)cap));
    TRY(dalloc(s, &d.alive[1], sizeof(int) * (size_t)cap));
    for (int lv = 0; lv < LV_N; ++lv) TRY(dalloc(s, &d.list[lv], sizeof(int) * (size_t)G * cap));
    TRY(dalloc(s, &d.rc, sizeof(RoundCounters)));
    CU(cudaMemset(d.rc, 0, sizeof(RoundCounters)));
    for (int lv = 0; lv < LV_F64; ++lv) {
        TRY(dalloc(s, &d.score[lv], sizeof(float) * (size_t)G * cap));
        TRY(dalloc(s, &s->d_margin[lv], sizeof(float) * kMqPool));
        d.margin[lv] = s->d_margin[lv];
    }
    d.cap64 = std::min(cap, 8192);
    d.ld64 = s->mlps.max_width;
    for (int k = 0; k < 2; ++k) TRY(dalloc(s, &d.act64[k], sizeof(double) * (size_t)d.cap64 * d.ld64));
    TRY(dalloc(s, &d.err, sizeof(unsigned int)));
    CU(cudaMemset(d.err, 0, sizeof(unsigned int)));
    TRY(dalloc(s, &d.gates, sizeof(int) * kMqGates));
    CU(cudaMemset(d.gates, 0, sizeof(int) * kMqGates));
    for (int k = 0; k < 2; ++k) CU(cudaStreamCreateWithFlags(&s->helper[k], cudaStreamNonBlocking));
    for (int k = 0; k < 2; ++k) TRY(dalloc(s, &s->act32[k], sizeof(float) * (size_t)cap * s->wmax));
    if (bf16(s)) {
        for (const Udf &u : s->udfs)
            for (int l = 0; l + 1 < u.n_layers; ++l)
                if (!tc_gemm_supported(u.dims[l], u.dims[l + 1]))
                    return fail(HYDRO_EUNSUPPORTED, "BF16 sessions need layer widths that are multiples of 64");
        TRY(dalloc(s, &s->stage16, sizeof(__nv_bfloat16) * (size_t)cap * c.dim));
        for (int k = 0; k < 2; ++k) TRY(dalloc(s, &s->act16[k], sizeof(__nv_bfloat16) * (size_t)cap * s->wmax));
        TRY(dalloc(s, &s->stage3, sizeof(__nv_bfloat16) * (size_t)cap * 3 * c.dim));
        for (int k = 0; k < 2; ++k) TRY(dalloc(s, &s->act3[k], sizeof(__nv_bfloat16) * (size_t)cap * 3 * s->wmax));
        if (fp8(s)) {
            // the FP8 set: first layers wide enough, quantised per output channel on the device
            const int wmin = c.fp8_min_width > 0 ? c.fp8_min_width : 1024;
            for (int g = 0; g < G; ++g) {
                Udf &u = s->udfs[g];
                u.q8 = u.n_layers >= 2 && u.dims[1] >= wmin && tc_gemm_fp8_supported(u.dims[0], u.dims[1]);
                if (!u.q8) continue;
                s->q8_mask |= 1u << g;
                TRY(dalloc(s, &u.dW8, (size_t)u.dims[1] * u.dims[0]));
                TRY(dalloc(s, &u.dsw, sizeof(float) * u.dims[1]));
                launch_quant_rows_e4m3(u.dW[0], u.dims[1], u.dims[0], u.dW8, u.dsw, s->sms, s->st);
            }
            TRY(dalloc(s, &s->stage8, (size_t)cap * c.dim));
            TRY(dalloc(s, &s->ascale, sizeof(float) * (size_t)cap));
            CU(cudaMemsetAsync(s->ascale, 0, sizeof(float) * (size_t)cap, s->st));
            CU(cudaStreamSynchronize(s->st));
            CU(cudaGetLastError());
            // level-0 bands of the UDFs outside the FP8 set (already BF16) skip the BF16 level
            d.lv1_skip = ((1u << G) - 1u) & ~s->q8_mask;
        }
        s->pstride = 2 * (s->wmax / 64);
        TRY(dalloc(s, &s->partials, sizeof(float) * (size_t)cap * s->pstride));
        hydro_status rs = tc_gemm_init(&s->encode);
        if (rs != HYDRO_OK) return fail(rs, "tensor-core GEMM init: %s", tc_gemm_last_error());
    }

    if (c.learned) {
        const int P = s->queries[0].P, D = c.dim;
        const int H = s->ph = c.proxy_hidden > 0 ? c.proxy_hidden : 64;
        const size_t nparam = (size_t)H * D + H + (size_t)P * H + P;
        std::vector<float> init(nparam, 0.f);
        std::mt19937 gen((unsigned)c.proxy_seed);
        std::uniform_real_distribution<float> u1(-std::sqrt(6.f / D), std::sqrt(6.f / D));
        std::uniform_real_distribution<float> u2(-1.f / std::sqrt((float)H), 1.f / std::sqrt((float)H));
        for (size_t k = 0; k < (size_t)H * D; ++k) init[k] = u1(gen);
        for (size_t k = 0; k < (size_t)P * H; ++k) init[(size_t)H * D + H + k] = u2(gen);
        float *params = nullptr;
        TRY(upload(s, &params, init.data(), nparam));
        s->pW1 = params;
        s->pb1 = s->pW1 + (size_t)H * D;
        s->pW2 = s->pb1 + H;
        s->pb2 = s->pW2 + (size_t)P * H;
        s->nparam = nparam;
        TRY(upload(s, &s->iparams, init.data(), nparam));
        s->iW1 = s->iparams;
        s->ib1 = s->iW1 + (size_t)H * D;
        s->iW2 = s->ib1 + H;
        s->ib2 = s->iW2 + (size_t)P * H;
        TRY(dalloc(s, &s->tH, sizeof(float) * (size_t)cap * H));
        TRY(dalloc(s, &s->tZ, sizeof(float) * (size_t)cap * kMqSlots));
        CU(cudaStreamCreateWithFlags(&s->train_st, cudaStreamNonBlocking));
        CU(cudaEventCreateWithFlags(&s->ev_ring, cudaEventDisableTiming));
        CU(cudaEventCreateWithFlags(&s->ev_trained, cudaEventDisableTiming));
        TRY(dalloc(s, &s->pg, sizeof(float) * nparam));
        TRY(dalloc(s, &s->pm, sizeof(float) * nparam));
        TRY(dalloc(s, &s->pv, sizeof(float) * nparam));
        CU(cudaMemset(s->pm, 0, sizeof(float) * nparam));
        CU(cudaMemset(s->pv, 0, sizeof(float) * nparam));
        TRY(dalloc(s, &s->pH, sizeof(float) * (size_t)cap * H));
        TRY(dalloc(s, &s->pZ, sizeof(float) * (size_t)cap * kMqSlots));
        TRY(dalloc(s, &s->pdZ, sizeof(float) * (size_t)cap * kMqSlots));
        TRY(dalloc(s, &s->pdH, sizeof(float) * (size_t)cap * H));
        TRY(dalloc(s, &s->ppart, sizeof(float) * proxy_grad_part_floats(cap, D, H, P)));
        TRY(dalloc(s, &s->pinv, sizeof(float)));
        TRY(dalloc(s, &s->p_ready, sizeof(int)));
        CU(cudaMemset(s->p_ready, 0, sizeof(int)));
        TRY(dalloc(s, &s->p_count, sizeof(int)));
        TRY(dalloc(s, &s->p_rows, sizeof(int) * (size_t)cap));
        void *hp = nullptr;
        CU(cudaMallocHost(&hp, sizeof(int)));
        s->host_allocs.push_back(hp);
        s->h_one = (int *)hp;
        *s->h_one = 1;
        // steps holding proxy_refresh batches, plus the one the next step writes while a
        // training still reads the others
        const int R = (std::max(1, c.proxy_refresh) + K - 1) / K + 1;
        TRY(dalloc(s, &s->ringX, sizeof(float) * (size_t)R * cap * D));
        TRY(dalloc(s, &s->ringL, (size_t)R * cap));
        TRY(dalloc(s, &s->ringM, (size_t)R * cap));
        s->ring_n.assign(R, 0);
        TRY(dalloc(s, &d.order_t, (size_t)cap * kMqSlots));
        s->proxy_tc = bf16(s) && H % 64 == 0 && tc_gemm_supported(D, H);
        if (s->proxy_tc) {
            TRY(dalloc(s, &s->pW1_16, sizeof(__nv_bfloat16) * (size_t)H * D));
            TRY(dalloc(s, &s->pH16, sizeof(__nv_bfloat16) * (size_t)cap * H));
            TRY(upload(s, &s->p_hrows, &H, 1));
            launch_gather_bf16(s->p_hrows, nullptr, s->iW1, D, D, s->pW1_16, H, s->sms, s->st);
            CU(cudaGetLastError());
        }
    }

    // statistics history
    MqHist &h = s->h;
    h.R = c.stats_window + c.route_lag + 2;
    h.lag = c.route_lag;
    h.static_order = c.policy == HYDRO_POLICY_STATIC ? 1 : 0;
    h.warmup = c.warmup_batches;
    h.window = c.stats_window;
    TRY(dalloc(s, &h.ring, sizeof(StatRow) * (size_t)NQ * h.R * kMqSlots));
    TRY(dalloc(s, &h.warm, sizeof(StatRow) * (size_t)NQ * std::max(1, h.warmup) * kMqSlots));
    TRY(dalloc(s, &h.bdone, sizeof(long long) * NQ));
    CU(cudaMemset(h.ring, 0, sizeof(StatRow) * (size_t)NQ * h.R * kMqSlots));
    CU(cudaMemset(h.warm, 0, sizeof(StatRow) * (size_t)NQ * std::max(1, h.warmup) * kMqSlots));
    CU(cudaMemset(h.bdone, 0, sizeof(long long) * NQ));

    // in-flight slots
    s->slots.resize(c.max_in_flight);
    for (Slot &sl : s->slots) {
        CU(cudaEventCreate(&sl.ev0));
        CU(cudaEventCreate(&sl.ev1));
        void *hp = nullptr;
        CU(cudaMallocHost(&hp, sizeof(StepHdr)));
        s->host_allocs.push_back(hp);
        sl.h_hdr = (StepHdr *)hp;
        memset(sl.h_hdr, 0, sizeof(StepHdr));
        TRY(dalloc(s, &sl.bitmap, sizeof(unsigned int) * ((size_t)cap / 32 + 1)));
        TRY(dalloc(s, &sl.rows, sizeof(StatRow) * (size_t)Q * kMqSlots));
        TRY(dalloc(s, &sl.order, (size_t)Q * kMqSlots));
        TRY(dalloc(s, &sl.evall, (size_t)Q));
        TRY(dalloc(s, &sl.bidx, sizeof(long long) * Q));
        TRY(dalloc(s, &sl.npass, sizeof(long long) * Q));
        TRY(dalloc(s, &sl.total, sizeof(int)));
        TRY(dalloc(s, &sl.gates, sizeof(int) * kMqGates));
        TRY(dalloc(s, &sl.sched, sizeof(int) * 2 * kRecLaunches));
        CU(cudaMemset(sl.sched, 0, sizeof(int) * 2 * kRecLaunches));
        TRY(dalloc(s, &sl.rec, sizeof(unsigned long long) * 2 * kRecCtas * kRecLaunches));
        CU(cudaMemset(sl.rec, 0, sizeof(unsigned long long) * 2 * kRecCtas * kRecLaunches));
    }
    s->finalized = true;
    return HYDRO_OK;
}

hydro_status upload_margins(hydro_session *s) {
    // level 0 of a FP32 session decides at FP32 accuracy: its margin is margin_fp32
    float m[LV_F64][kMqPool] = {};
    for (size_t g = 0; g < s->udfs.size(); ++g) {
        const Udf &u = s->udfs[g];
        m[LV_MAIN][g] = (float)(bf16(s) ? u.margin_lowp : u.margin_fp32);
        m[LV_X3][g] = (float)u.margin_x3;
        m[LV_F32][g] = (float)u.margin_fp32;
    }
    for (int lv = 0; lv < LV_F64; ++lv)
        CU(cudaMemcpy(s->d_margin[lv], m[lv], sizeof m[lv], cudaMemcpyHostToDevice));
    return HYDRO_OK;
}

// Learned sessions: refresh the steps' inference copy of the proxy from the
// FP32 masters once the pending training has finished (the step stream
// waits for it), and mark the proxy ready.
hydro_status proxy_swap(hydro_session *s) {
    if (!s->train_pending) return HYDRO_OK;
    CU(cudaStreamWaitEvent(s->st, s->ev_trained, 0));
    CU(cudaMemcpyAsync(s->iparams, s->pW1, sizeof(float) * s->nparam, cudaMemcpyDeviceToDevice, s->st));
    if (s->proxy_tc) {
        launch_gather_bf16(s->p_hrows, nullptr, s->iW1, s->cfg.dim, s->cfg.dim, s->pW1_16, s->ph, s->sms, s->st);
        s->launches++;
    }
    CU(cudaMemcpyAsync(s->p_ready, s->h_one, sizeof(int), cudaMemcpyHostToDevice, s->st));
    s->train_pending = false;
    return HYDRO_OK;
}

// Learned sessions, after a step: keep its tuples and outcomes in the
// training ring; every proxy_refresh batches retrain the proxy on the ring's
// steps holding the last proxy_refresh batches (masked BCE on the slots each
// tuple was evaluated on, Adam), on the training stream, after the ring copy.
// The steps see the result from the second step after this one on
// (proxy_swap at that submit), so training overlaps the next step.
hydro_status learned_after_step(hydro_session *s, const Slot &slot) {
    int n = 0, nb = 0;   // the step's tuples and batches (one query)
    for (int k = 0; k < s->cfg.batches_per_step; ++k) {
        n += slot.counts[k];
        nb += slot.counts[k] > 0;
    }
    if (n <= 0) return HYDRO_OK;
    const hydro_session_config &c = s->cfg;
    const int D = c.dim, H = s->ph, P = s->queries[0].P, cap = s->d.cap;
    const int RR = (int)s->ring_n.size();   // ring entries
    const int R = RR - 1;                   // entries one training reads
    const int rs = (int)(s->learned_steps % RR);
    CU(cudaMemcpyAsync(s->ringX + (size_t)rs * cap * D, slot.h_hdr->X, sizeof(float) * (size_t)n * D,
                       cudaMemcpyDeviceToDevice, s->st));
    CU(cudaMemcpyAsync(s->ringL + (size_t)rs * cap, s->d.label, n, cudaMemcpyDeviceToDevice, s->st));
    CU(cudaMemcpyAsync(s->ringM + (size_t)rs * cap, s->d.visited, n, cudaMemcpyDeviceToDevice, s->st));
    s->ring_n[rs] = n;
    s->learned_steps++;
    const long long before = s->learned_batches;
    s->learned_batches += nb;
    const int refresh = std::max(1, c.proxy_refresh);
    if (before / refresh == s->learned_batches / refresh) return HYDRO_OK;
    // a training still pending (launched after the previous step) takes effect now,
    // before the next one changes the masters
    TRY(proxy_swap(s));
    CU(cudaEventRecord(s->ev_ring, s->st));
    CU(cudaStreamWaitEvent(s->train_st, s->ev_ring, 0));
    const cudaStream_t ts = s->train_st;
    const size_t nW1 = (size_t)H * D;
    for (int e = 0; e < std::max(1, c.proxy_epochs); ++e)
        for (int j = 0; j < R; ++j) {
            const long long stp = s->learned_steps - R + j;   // oldest first
            if (stp < 0) continue;
            const int k = (int)(stp % RR);
            const int Mall = s->ring_n[k];
            if (Mall <= 0) continue;
            const int M = c.proxy_rows > 0 ? std::min(Mall, c.proxy_rows) : Mall;
            const int off = M < Mall ? (int)(s->train_off % (Mall - M + 1)) : 0;
            s->train_off += M;
            const float *Xs = s->ringX + ((size_t)k * cap + off) * D;
            launch_identity_list(s->p_rows, s->p_count, 0, M, ts);
            launch_mlp_layer_f32(s->p_count, nullptr, Xs, D, s->pW1, s->pb1, s->tH, D, H, 1, M, s->sms, ts);
            launch_mlp_layer_f32(s->p_count, nullptr, s->tH, H, s->pW2, s->pb2, s->tZ, H, P, 0, M, s->sms, ts);
            ProxyTrain pt{};
            pt.M = M;
            pt.P = P;
            pt.H = H;
            pt.D = D;
            pt.sms = s->sms;
            pt.t = ++s->adam_t;
            pt.lr = c.proxy_lr;
            pt.X = Xs;
            pt.Hact = s->tH;
            pt.Z = s->tZ;
            pt.dZ = s->pdZ;
            pt.dH = s->pdH;
            pt.inv_pairs = s->pinv;
            pt.part = s->ppart;
            pt.label = s->ringL + (size_t)k * cap + off;
            pt.mask = s->ringM + (size_t)k * cap + off;
            pt.W1 = s->pW1;
            pt.b1 = s->pb1;
            pt.W2 = s->pW2;
            pt.b2 = s->pb2;
            pt.gW1 = s->pg;
            pt.gb1 = s->pg + nW1;
            pt.gW2 = pt.gb1 + H;
            pt.gb2 = pt.gW2 + (size_t)P * H;
            pt.mW1 = s->pm;
            pt.mb1 = s->pm + nW1;
            pt.mW2 = pt.mb1 + H;
            pt.mb2 = pt.mW2 + (size_t)P * H;
            pt.vW1 = s->pv;
            pt.vb1 = s->pv + nW1;
            pt.vW2 = pt.vb1 + H;
            pt.vb2 = pt.vW2 + (size_t)P * H;
            launch_proxy_train_step(pt, ts);
            s->launches += 16;
        }
    CU(cudaEventRecord(s->ev_trained, ts));
    s->train_pending = true;
    s->train_step = s->next_step;
    CU(cudaGetLastError());
    return HYDRO_OK;
}

hydro_status wait_ev(cudaEvent_t ev, long long wait_ms, bool *done) {
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

__global__ void k_single_queue(RoundCounters *rc, int g, int n, int *queues, int cap) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < LV_N * kMqPool) (&rc->n[0][0])[i] = i == g ? n : 0;   // level 0, group g
    for (int m = i; m < n; m += gridDim.x * blockDim.x) queues[(size_t)g * cap + m] = m;
}

__global__ void k_score_to_f64(const float *src, double *dst, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (double)src[i];
}

}  // namespace

// ================================================================ C ABI

extern "C" {

void hydro_session_default_config(hydro_session_config *cfg) {
    if (!cfg) return;
    memset(cfg, 0, sizeof *cfg);
    cfg->precision = HYDRO_PREC_FP32;
    cfg->warmup_batches = 1;
    cfg->stats_window = 8;
    cfg->use_graphs = 1;
    cfg->autotune = 1;
    cfg->max_in_flight = 2;
    cfg->proxy_hidden = 64;
    cfg->proxy_refresh = 16;
    cfg->proxy_epochs = 1;
    cfg->proxy_lr = 1e-3f;
    cfg->proxy_seed = 1;
    cfg->batches_per_step = 1;
    cfg->route_lag = 0;
}

hydro_status hydro_session_create(const hydro_session_config *cfg, hydro_session **out) {
    set_last_error("");
    if (!cfg || !out) return fail(HYDRO_EINVAL, "NULL argument");
    *out = nullptr;
    if (cfg->dim < 64 || cfg->dim % 64) return fail(HYDRO_EINVAL, "dim must be a positive multiple of 64");
    if (cfg->max_step_tuples < 1 || cfg->max_step_tuples > (1 << 22))
        return fail(HYDRO_EINVAL, "max_step_tuples outside 1..4194304");
    if (cfg->precision != HYDRO_PREC_FP32 && cfg->precision != HYDRO_PREC_BF16 && cfg->precision != HYDRO_PREC_FP8)
        return fail(HYDRO_EINVAL, "precision must be FP32, BF16 or FP8");
    if (cfg->precision == HYDRO_PREC_FP8 && (cfg->dim % 128 || cfg->fp8_min_width < 0))
        return fail(HYDRO_EINVAL, "FP8 sessions need dim a multiple of 128 and fp8_min_width >= 0");
    if (cfg->warmup_batches < 0 || cfg->stats_window < 1) return fail(HYDRO_EINVAL, "bad warmup/window");
    if (cfg->policy != HYDRO_POLICY_RANK && cfg->policy != HYDRO_POLICY_STATIC)
        return fail(HYDRO_EINVAL, "session policy must be RANK or STATIC");
    if (cfg->learned && cfg->policy != HYDRO_POLICY_RANK)
        return fail(HYDRO_EINVAL, "learned sessions fall back to rank routing (policy RANK)");
    if (cfg->max_in_flight < 1 || cfg->max_in_flight > 8) return fail(HYDRO_EINVAL, "max_in_flight outside 1..8");
    if (cfg->tile_sched != 0 && cfg->tile_sched != 1) return fail(HYDRO_EINVAL, "tile_sched must be 0 or 1");
    if (cfg->batches_per_step < 1 || cfg->batches_per_step > 32 || cfg->route_lag < cfg->batches_per_step - 1 ||
        cfg->route_lag > 64)
        return fail(HYDRO_EINVAL, "batches_per_step 1..32 with route_lag >= batches_per_step - 1 (<= 64)");
    if (cfg->learned && (cfg->proxy_hidden < 0 || cfg->proxy_hidden > 1024 || cfg->proxy_refresh < 1 ||
                         cfg->proxy_refresh > 256 || cfg->proxy_epochs < 0 || !(cfg->proxy_lr > 0.f) ||
                         cfg->proxy_rows < 0))
        return fail(HYDRO_EINVAL, "bad proxy settings");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev)
        return fail(HYDRO_EINVAL, "no CUDA device %d", cfg->device);
    hydro_session *s = new hydro_session();
    s->cfg = *cfg;
    *out = s;
    return HYDRO_OK;
}

hydro_status hydro_session_add_udf(hydro_session *s, const hydro_udf_desc *udf, int32_t *out_udf) {
    set_last_error("");
    TRY(check(s));
    if (s->finalized) return fail(HYDRO_ESTATE, "UDFs must be added before the first submit");
    if (!udf || udf->kind != HYDRO_UDF_MLP || udf->upstream) return fail(HYDRO_EINVAL, "pool UDFs are plain MLPs");
    if ((int)s->udfs.size() >= HYDRO_MAX_POOL) return fail(HYDRO_EINVAL, "pool is full (%d)", HYDRO_MAX_POOL);
    const int L = udf->n_layers;
    if (L < 2 || L > HYDRO_MAX_LAYERS || !udf->dims || !udf->weights || !udf->biases)
        return fail(HYDRO_EINVAL, "a pool MLP has 2..%d layers with weights and biases", HYDRO_MAX_LAYERS);
    if (udf->dims[0] != s->cfg.dim || udf->dims[L] != 1) return fail(HYDRO_EINVAL, "dims[0] must be dim, last 1");
    Udf u;
    u.n_layers = L;
    u.dims.assign(udf->dims, udf->dims + L + 1);
    long long flops = 0;
    for (int l = 0; l < L; ++l) {
        if (u.dims[l + 1] < 1 || u.dims[l + 1] > 65536) return fail(HYDRO_EINVAL, "bad width");
        if (!udf->weights[l] || !udf->biases[l]) return fail(HYDRO_EINVAL, "NULL weights of layer %d", l);
        u.W.emplace_back(udf->weights[l], udf->weights[l] + (size_t)u.dims[l] * u.dims[l + 1]);
        u.b.emplace_back(udf->biases[l], udf->biases[l] + u.dims[l + 1]);
        flops += 2LL * u.dims[l] * u.dims[l + 1];
    }
    u.cost = udf->cost_hint > 0 ? udf->cost_hint : flops;
    s->udfs.push_back(std::move(u));
    if (out_udf) *out_udf = (int32_t)s->udfs.size() - 1;
    return HYDRO_OK;
}

hydro_status hydro_session_add_query(hydro_session *s, int32_t n_preds, const int32_t *udfs, const double *thresholds,
                                     int32_t *out_query) {
    set_last_error("");
    TRY(check(s));
    if (s->finalized) return fail(HYDRO_ESTATE, "queries must be added before the first submit");
    if (((int)s->queries.size() + 1) * s->cfg.batches_per_step > HYDRO_MAX_QUERIES)
        return fail(HYDRO_EINVAL, "too many queries (queries x batches_per_step <= %d)", HYDRO_MAX_QUERIES);
    if (s->cfg.learned && !s->queries.empty()) return fail(HYDRO_EINVAL, "learned sessions have one query");
    if (n_preds < 1 || n_preds > HYDRO_MAX_PREDICATES || !udfs || !thresholds)
        return fail(HYDRO_EINVAL, "a query has 1..%d predicates", HYDRO_MAX_PREDICATES);
    Query q;
    q.P = n_preds;
    unsigned seen = 0;
    for (int k = 0; k < n_preds; ++k) {
        if (udfs[k] < 0 || udfs[k] >= (int)s->udfs.size()) return fail(HYDRO_EINVAL, "unknown pool UDF %d", udfs[k]);
        if (seen & (1u << udfs[k])) return fail(HYDRO_EINVAL, "pool UDF %d used twice in one query", udfs[k]);
        seen |= 1u << udfs[k];
        q.udf[k] = udfs[k];
        q.thr[k] = thresholds[k];
    }
    s->queries.push_back(q);
    if (out_query) *out_query = (int32_t)s->queries.size() - 1;
    return HYDRO_OK;
}

hydro_status hydro_session_set_margins(hydro_session *s, int32_t udf, double margin_lowp, double margin_split,
                                       double margin_fp32) {
    set_last_error("");
    TRY(check(s));
    if (udf < 0 || udf >= (int)s->udfs.size()) return fail(HYDRO_EINVAL, "unknown pool UDF");
    if (!(margin_lowp >= 0) || !(margin_split >= 0) || !(margin_fp32 >= 0))
        return fail(HYDRO_EINVAL, "margins must be >= 0");
    if (s->next_step > 0) return fail(HYDRO_ESTATE, "margins are fixed after the first submit");
    s->udfs[udf].margin_lowp = margin_lowp;
    s->udfs[udf].margin_x3 = margin_split;
    s->udfs[udf].margin_fp32 = margin_fp32;
    return HYDRO_OK;
}

hydro_status hydro_session_udf_scores(hydro_session *s, int32_t udf, int32_t prec, const void *d_tuples, int64_t n,
                                      double *d_scores) {
    set_last_error("");
    TRY(check(s));
    if (udf < 0 || udf >= (int)s->udfs.size()) return fail(HYDRO_EINVAL, "unknown pool UDF");
    if (n < 0 || (n > 0 && (!d_tuples || !d_scores))) return fail(HYDRO_EINVAL, "bad tuples/scores");
    if ((uintptr_t)d_tuples % 16) return fail(HYDRO_EINVAL, "tuples must be 16-byte aligned");
    if (prec != HYDRO_PREC_FP64 && prec != HYDRO_PREC_FP32 && prec != HYDRO_PREC_BF16 && prec != HYDRO_PREC_BF16X3 &&
        prec != HYDRO_PREC_FP8)
        return fail(HYDRO_EINVAL, "precision must be FP64, FP32, BF16, BF16X3 or FP8");
    if ((prec == HYDRO_PREC_BF16 || prec == HYDRO_PREC_BF16X3) && !bf16(s))
        return fail(HYDRO_EINVAL, "BF16 and split-BF16 scores need a BF16 or FP8 session");
    if (prec == HYDRO_PREC_FP8 && !fp8(s)) return fail(HYDRO_EINVAL, "FP8 scores need an FP8 session");
    CU(cudaSetDevice(s->cfg.device));
    TRY(finalize(s));
    for (Slot &sl : s->slots)
        if (sl.busy) return fail(HYDRO_ESTATE, "poll every step before scoring");
    const float *X = (const float *)d_tuples;
    if (prec == HYDRO_PREC_FP64) {
        if (n > 0) mq_launch_scores_f64(s->udfs[udf].mlp, s->mlps.max_width, X, s->cfg.dim, (int)n, d_scores, s->st, s->sms);
    } else {
        float *score_g = s->d.score[LV_MAIN] + (size_t)udf * s->d.cap;
        for (int64_t o = 0; o < n; o += s->d.cap) {
            const int m = (int)std::min<int64_t>(s->d.cap, n - o);
            StepHdr hh{};
            hh.X = X + (size_t)o * s->cfg.dim;
            CU(cudaMemcpyAsync(s->d_hdr, &hh, sizeof(void *), cudaMemcpyHostToDevice, s->st));
            k_single_queue<<<std::max(1, std::min((m + 255) / 256, s->sms * 4)), 256, 0, s->st>>>(
                s->d.rc, udf, m, s->d.list[LV_MAIN], s->d.cap);
            if (prec == HYDRO_PREC_BF16 || prec == HYDRO_PREC_BF16X3 || prec == HYDRO_PREC_FP8) {
                TRY(eval_tc(s, rc_n(s->d, LV_MAIN), s->d.list[LV_MAIN], s->d.score[LV_MAIN],
                            prec == HYDRO_PREC_BF16X3, 0, nullptr, prec == HYDRO_PREC_FP8));
            } else {
                eval_f32(s, rc_n(s->d, LV_MAIN), s->d.list[LV_MAIN], s->d.score[LV_MAIN]);
            }
            k_score_to_f64<<<(m + 255) / 256, 256, 0, s->st>>>(score_g, d_scores + o, m);
            CU(cudaStreamSynchronize(s->st));
        }
    }
    CU(cudaStreamSynchronize(s->st));
    unsigned int err = 0;
    CU(cudaMemcpy(&err, s->d.err, sizeof err, cudaMemcpyDeviceToHost));
    if (err) return fail(HYDRO_EDEVICE, "device error word 0x%x", err);
    return HYDRO_OK;
}

hydro_status hydro_session_calibrate(hydro_session *s, const void *d_tuples, int64_t n, hydro_calib_info *info) {
    set_last_error("");
    TRY(check(s));
    if (n < 1 || !d_tuples) return fail(HYDRO_EINVAL, "need calibration tuples");
    if (s->next_step > 0) return fail(HYDRO_ESTATE, "calibrate before the first submit");
    CU(cudaSetDevice(s->cfg.device));
    TRY(finalize(s));
    double *d = nullptr;
    CU(cudaMalloc(&d, sizeof(double) * n * 5));
    std::vector<double> s64(n), s32(n), s16(n), s3(n), s8(n);
    hydro_status rc = HYDRO_OK;
    const bool bf = bf16(s), f8 = fp8(s);
    for (int g = 0; g < (int)s->udfs.size() && rc == HYDRO_OK; ++g) {
        rc = hydro_session_udf_scores(s, g, HYDRO_PREC_FP64, d_tuples, n, d);
        if (rc == HYDRO_OK) rc = hydro_session_udf_scores(s, g, HYDRO_PREC_FP32, d_tuples, n, d + n);
        if (rc == HYDRO_OK && bf) rc = hydro_session_udf_scores(s, g, HYDRO_PREC_BF16, d_tuples, n, d + 2 * n);
        if (rc == HYDRO_OK && bf) rc = hydro_session_udf_scores(s, g, HYDRO_PREC_BF16X3, d_tuples, n, d + 3 * n);
        if (rc == HYDRO_OK && f8) rc = hydro_session_udf_scores(s, g, HYDRO_PREC_FP8, d_tuples, n, d + 4 * n);
        if (rc != HYDRO_OK) break;
        if (cudaMemcpy(s64.data(), d, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(s32.data(), d + n, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess ||
            (bf && cudaMemcpy(s16.data(), d + 2 * n, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess) ||
            (bf && cudaMemcpy(s3.data(), d + 3 * n, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess) ||
            (f8 && cudaMemcpy(s8.data(), d + 4 * n, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess)) {
            rc = fail(HYDRO_ECUDA, "copy of calibration scores failed");
            break;
        }
        double e32 = 0, e16 = 0, e3 = 0, e8 = 0, smax = 0;
        for (int64_t k = 0; k < n; ++k) {
            e32 = std::max(e32, std::fabs(s32[k] - s64[k]));
            if (bf) e16 = std::max(e16, std::fabs(s16[k] - s64[k]));
            if (bf) e3 = std::max(e3, std::fabs(s3[k] - s64[k]));
            if (f8) e8 = std::max(e8, std::fabs(s8[k] - s64[k]));
            smax = std::max(smax, std::fabs(s64[k]));
        }
        Udf &u = s->udfs[g];
        u.margin_fp32 = std::max(16.0 * e32, 1e-9 * smax);
        // level 0 (lowp) and level 1 (split BF16; BF16 in FP8 sessions)
        const double e0 = f8 ? e8 : e16, e1 = f8 ? e16 : e3;
        if (bf) u.margin_x3 = std::max((f8 ? 4.0 : 8.0) * e1, 1e-9 * smax);
        if (bf && u.margin_lowp < 4.0 * e0) u.margin_lowp = 4.0 * e0;
        if (info) {
            info[g] = hydro_calib_info{};
            info[g].max_err_fp32 = e32;
            info[g].max_err_lowp = e0;
            info[g].max_err_tf32 = e1;
            info[g].margin_fp32 = u.margin_fp32;
            info[g].margin_lowp = u.margin_lowp;
            info[g].margin_tf32 = u.margin_x3;
        }
    }
    cudaFree(d);
    return rc;
}

hydro_status hydro_session_submit(hydro_session *s, const void *d_tuples, const int32_t *counts, int64_t *out_step) {
    set_last_error("");
    TRY(check(s));
    if (!counts || !out_step) return fail(HYDRO_EINVAL, "NULL counts or out_step");
    CU(cudaSetDevice(s->cfg.device));
    TRY(finalize(s));
    const int K = s->cfg.batches_per_step, Q = (int)s->queries.size() * K;
    long long total = 0;
    for (int q = 0; q < Q; ++q) {
        if (counts[q] < 0) return fail(HYDRO_EINVAL, "count of entry %d is negative", q);
        if (q % K && counts[q] > 0 && counts[q - 1] == 0)
            return fail(HYDRO_EINVAL, "query %d: a non-empty batch after an empty one", q / K);
        total += counts[q];
    }
    if (total > s->cfg.max_step_tuples) return fail(HYDRO_EINVAL, "step of %lld tuples > max_step_tuples", total);
    if (total > 0 && !d_tuples) return fail(HYDRO_EINVAL, "NULL tuples");
    if ((uintptr_t)d_tuples % 16) return fail(HYDRO_EINVAL, "tuples must be 16-byte aligned");
    Slot *slot = nullptr;
    for (Slot &sl : s->slots)
        if (!sl.busy) {
            slot = &sl;
            break;
        }
    if (!slot) return fail(HYDRO_EAGAIN, "all %d in-flight slots are busy; poll first", s->cfg.max_in_flight);
    if (s->next_step == 0) {
        TRY(upload_margins(s));
        if (s->cfg.autotune && bf16(s)) TRY(autotune(s));
    }
    if (s->cfg.learned && s->train_pending && s->next_step >= s->train_step + 2) TRY(proxy_swap(s));
    slot->h_hdr->X = (const float *)d_tuples;
    for (int q = 0; q < Q; ++q) slot->h_hdr->counts[q] = counts[q];
    slot->counts.assign(counts, counts + Q);
    for (ProfRec &r : slot->prof) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    slot->prof.clear();
    if (s->cfg.use_graphs && !s->prof_on) {
        if (!slot->exec) {
            cudaGraph_t graph = nullptr;
            CU(cudaGraphCreate(&graph, 0));
            for (int k = 0; k < kMqGates; ++k) s->handles[k] = 0;
            s->cap_graph = graph;
            s->handle_err = HYDRO_OK;
            cudaError_t be = cudaStreamBeginCaptureToGraph(s->st, graph, nullptr, nullptr, 0,
                                                           cudaStreamCaptureModeThreadLocal);
            if (be != cudaSuccess) {
                cudaGraphDestroy(graph);
                return fail(HYDRO_ECUDA, "capture: %s", cudaGetErrorString(be));
            }
            s->capturing = true;
            s->if_depth = 0;
            const cudaStream_t main_st = s->st;
            hydro_status rs = enqueue_step(s, *slot);
            s->cur_slot = nullptr;
            s->capturing = false;
            // a failure inside a region leaves helper captures open: close them
            while (s->if_depth > 0) {
                cudaGraph_t g2 = nullptr;
                cudaStreamEndCapture(s->helper[--s->if_depth], &g2);
            }
            s->st = main_st;
            cudaGraph_t out = nullptr;
            cudaError_t ce = cudaStreamEndCapture(s->st, &out);
            if (rs != HYDRO_OK) {
                cudaGraphDestroy(graph);
                return rs;
            }
            if (ce != cudaSuccess) {
                cudaGraphDestroy(graph);
                return fail(HYDRO_ECUDA, "graph capture: %s", cudaGetErrorString(ce));
            }
            ce = cudaGraphInstantiate(&slot->exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ce != cudaSuccess) return fail(HYDRO_ECUDA, "graph instantiate: %s", cudaGetErrorString(ce));
        }
        CU(cudaEventRecord(slot->ev0, s->st));
        CU(cudaGraphLaunch(slot->exec, s->st));
    } else {
        CU(cudaEventRecord(slot->ev0, s->st));
        s->prof_slot = s->prof_on ? slot : nullptr;
        hydro_status rs = enqueue_step(s, *slot);
        s->prof_slot = nullptr;
        s->cur_slot = nullptr;
        TRY(rs);
    }
    CU(cudaEventRecord(slot->ev1, s->st));
    if (s->cfg.learned) TRY(learned_after_step(s, *slot));
    s->last_step_total = total;
    slot->busy = true;
    slot->step = s->next_step;
    *out_step = s->next_step++;
    return HYDRO_OK;
}

hydro_status hydro_session_poll(hydro_session *s, int64_t step, uint32_t *pass_bitmap, hydro_step_query *per_query,
                                double *device_ms, int32_t wait_ms) {
    set_last_error("");
    TRY(check(s));
    Slot *slot = nullptr;
    for (Slot &sl : s->slots)
        if (sl.busy && sl.step == step) slot = &sl;
    if (!slot) return fail(HYDRO_ENOTFOUND, "step %lld is not in flight", (long long)step);
    CU(cudaSetDevice(s->cfg.device));
    bool done = false;
    TRY(wait_ev(slot->ev1, wait_ms, &done));
    if (!done) return fail(HYDRO_EAGAIN, "step %lld not finished", (long long)step);
    slot->busy = false;
    if (s->cfg.learned && s->train_pending) {
        // nothing else in flight: later work on the step stream follows the training
        bool idle = true;
        for (const Slot &sl : s->slots) idle = idle && !sl.busy;
        if (idle) CU(cudaStreamWaitEvent(s->st, s->ev_trained, 0));
    }
    s->launches += slot->launches;
    if (slot->conditional) {
        int g[kMqGates];
        CU(cudaMemcpy(g, slot->gates, sizeof g, cudaMemcpyDeviceToHost));
        for (int k = 0; k < kMqGates; ++k) s->launches += g[k] ? slot->gate_body[k] : 0;
    }
    for (ProfRec &r : slot->prof) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            s->prof_ms[r.cls] += ms;
            s->prof_n[r.cls]++;
        }
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    slot->prof.clear();
    if (s->bal_on && slot->n_rec > 0) {
        // per grouped launch: CTAs with work have a start stamp; busy = last - first
        std::vector<unsigned long long> rec((size_t)slot->n_rec * kRecCtas * 2);
        CU(cudaMemcpy(rec.data(), slot->rec, sizeof(unsigned long long) * rec.size(), cudaMemcpyDeviceToHost));
        hydro_balance_info &B = s->bal;
        for (int k = 0; k < slot->n_rec; ++k) {
            const unsigned long long *r = rec.data() + (size_t)k * kRecCtas * 2;
            unsigned long long t0 = ~0ull, t1 = 0;
            double sum = 0, mx = 0;
            int n = 0;
            for (int c = 0; c < kRecCtas; ++c) {
                if (!r[2 * c] || r[2 * c + 1] < r[2 * c]) continue;
                const double busy = (double)(r[2 * c + 1] - r[2 * c]) * 1e-6;
                t0 = std::min(t0, r[2 * c]);
                t1 = std::max(t1, r[2 * c + 1]);
                sum += busy;
                mx = std::max(mx, busy);
                B.cta_busy_ms[c] += busy;
                ++n;
            }
            if (!n) continue;
            B.launches++;
            B.ctas = std::max(B.ctas, n);
            B.makespan_ms += (double)(t1 - t0) * 1e-6;
            B.busy_mean_ms += sum / n;
            B.busy_max_ms += mx;
        }
    }
    unsigned int err = 0;
    CU(cudaMemcpy(&err, s->d.err, sizeof err, cudaMemcpyDeviceToHost));
    if (err) {
        s->dead = true;
        return fail(HYDRO_EDEVICE, "device error word 0x%x", err);
    }
    const int Q = (int)s->queries.size() * s->cfg.batches_per_step;
    int total = 0;
    CU(cudaMemcpy(&total, slot->total, sizeof(int), cudaMemcpyDeviceToHost));
    if (pass_bitmap && total > 0)
        CU(cudaMemcpy(pass_bitmap, slot->bitmap, sizeof(uint32_t) * ((size_t)(total + 31) / 32),
                      cudaMemcpyDeviceToHost));
    if (per_query) {
        std::vector<StatRow> rows((size_t)Q * kMqSlots);
        std::vector<unsigned char> order((size_t)Q * kMqSlots), evall(Q);
        std::vector<long long> bidx(Q), npass(Q);
        CU(cudaMemcpy(rows.data(), slot->rows, sizeof(StatRow) * rows.size(), cudaMemcpyDeviceToHost));
        CU(cudaMemcpy(order.data(), slot->order, order.size(), cudaMemcpyDeviceToHost));
        CU(cudaMemcpy(evall.data(), slot->evall, evall.size(), cudaMemcpyDeviceToHost));
        CU(cudaMemcpy(bidx.data(), slot->bidx, sizeof(long long) * Q, cudaMemcpyDeviceToHost));
        CU(cudaMemcpy(npass.data(), slot->npass, sizeof(long long) * Q, cudaMemcpyDeviceToHost));
        for (int q = 0; q < Q; ++q) {
            hydro_step_query &o = per_query[q];
            o = hydro_step_query{};
            o.n = slot->counts[q];
            o.n_pass = npass[q];
            o.batch = bidx[q];
            o.warmup = evall[q];
            for (int k = 0; k < HYDRO_MAX_PREDICATES; ++k) {
                const bool used = k < s->queries[q / s->cfg.batches_per_step].P;
                o.order[k] = used ? order[(size_t)q * kMqSlots + k] : -1;
                const StatRow &r = rows[(size_t)q * kMqSlots + k];
                o.evaluated[k] = r.evaluated;
                o.passed[k] = r.passed;
                o.recheck_split[k] = r.recheck_tf32;
                o.recheck_fp32[k] = r.recheck32;
                o.recheck_fp64[k] = r.recheck64;
            }
        }
    }
    if (device_ms) {
        float ms = 0;
        CU(cudaEventElapsedTime(&ms, slot->ev0, slot->ev1));
        *device_ms = ms;
    }
    return HYDRO_OK;
}

hydro_status hydro_session_debug_trace(hydro_session *s, int64_t step, uint8_t *order, uint8_t *visited) {
    set_last_error("");
    TRY(check(s));
    if (!order || !visited) return fail(HYDRO_EINVAL, "NULL output");
    if (step != s->next_step - 1 || s->last_step_total < 0) return fail(HYDRO_ESTATE, "only the last step has a trace");
    for (Slot &sl : s->slots)
        if (sl.busy) return fail(HYDRO_ESTATE, "poll the step first");
    const size_t n = (size_t)s->last_step_total;
    CU(cudaMemcpy(visited, s->d.visited, n, cudaMemcpyDeviceToHost));
    if (s->d.order_t) {
        CU(cudaMemcpy(order, s->d.order_t, n * kMqSlots, cudaMemcpyDeviceToHost));
    } else {
        std::vector<unsigned short> qid(n);
        std::vector<unsigned char> ord((size_t)s->d.Q * kMqSlots);
        CU(cudaMemcpy(qid.data(), s->d.qid, sizeof(unsigned short) * n, cudaMemcpyDeviceToHost));
        CU(cudaMemcpy(ord.data(), s->d.order, ord.size(), cudaMemcpyDeviceToHost));
        for (size_t e = 0; e < n; ++e) memcpy(order + e * kMqSlots, ord.data() + (size_t)qid[e] * kMqSlots, kMqSlots);
    }
    return HYDRO_OK;
}

hydro_status hydro_session_tuning(hydro_session *s, hydro_tile_choice *out, int32_t max, int32_t *n_out) {
    set_last_error("");
    TRY(check(s));
    if (!n_out || (max > 0 && !out)) return fail(HYDRO_EINVAL, "NULL output");
    const int n = std::min<int>(max, (int)s->tuning.size());
    for (int i = 0; i < n; ++i) out[i] = s->tuning[i];
    *n_out = n;
    return HYDRO_OK;
}

hydro_status hydro_session_profile(hydro_session *s, int32_t enable) {
    set_last_error("");
    TRY(check(s));
    for (Slot &sl : s->slots)
        if (sl.busy) return fail(HYDRO_ESTATE, "poll every step before switching profiling");
    s->prof_on = enable != 0;
    for (int k = 0; k < SP_N; ++k) {
        s->prof_ms[k] = 0;
        s->prof_n[k] = 0;
    }
    s->launches = 0;
    return HYDRO_OK;
}

hydro_status hydro_session_balance(hydro_session *s, int32_t enable, hydro_balance_info *out) {
    set_last_error("");
    TRY(check(s));
    if (enable == 0 || enable == 1) {
        for (Slot &sl : s->slots)
            if (sl.busy) return fail(HYDRO_ESTATE, "poll every step before switching the balance record");
        s->bal_on = enable == 1;
        if (enable == 1) s->bal = hydro_balance_info{};
    }
    if (out) *out = s->bal;
    return HYDRO_OK;
}

hydro_status hydro_session_profile_read(hydro_session *s, hydro_kernel_profile *out, int32_t max, int32_t *n_out,
                                        int64_t *total_launches) {
    set_last_error("");
    TRY(check(s));
    if (!n_out || (max > 0 && !out)) return fail(HYDRO_EINVAL, "NULL output");
    int n = 0;
    for (int k = 0; k < SP_N && n < max; ++k) {
        if (!s->prof_n[k]) continue;
        hydro_kernel_profile &o = out[n++];
        memset(&o, 0, sizeof o);
        snprintf(o.name, sizeof o.name, "%s", kSessProf[k]);
        o.launches = s->prof_n[k];
        o.total_ms = s->prof_ms[k];
    }
    *n_out = n;
    if (total_launches) *total_launches = s->launches;
    return HYDRO_OK;
}

hydro_status hydro_session_destroy(hydro_session *s) {
    set_last_error("");
    if (!s) return fail(HYDRO_EINVAL, "NULL session");
    cudaSetDevice(s->cfg.device);
    for (Slot &sl : s->slots) {
        if (sl.busy && sl.ev1) {
            bool done = false;
            wait_ev(sl.ev1, 60000, &done);
        }
        if (sl.exec) cudaGraphExecDestroy(sl.exec);
        for (ProfRec &r : sl.prof) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        if (sl.ev0) cudaEventDestroy(sl.ev0);
        if (sl.ev1) cudaEventDestroy(sl.ev1);
    }
    if (s->st) cudaStreamSynchronize(s->st);
    if (s->train_st) {
        cudaStreamSynchronize(s->train_st);
        cudaStreamDestroy(s->train_st);
    }
    if (s->ev_ring) cudaEventDestroy(s->ev_ring);
    if (s->ev_trained) cudaEventDestroy(s->ev_trained);
    for (int k = 0; k < 2; ++k)
        if (s->helper[k]) cudaStreamDestroy(s->helper[k]);
    for (void *p : s->allocs) cudaFree(p);
    for (void *p : s->host_allocs) cudaFreeHost(p);
    if (s->own_stream && s->st) cudaStreamDestroy(s->st);
    delete s;
    return HYDRO_OK;
}

}  // extern "C"
