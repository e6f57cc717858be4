/*
 * hydro.h - C ABI of the adaptive ML-predicate engine (B300, sm_103a).
 *
 * A query is a conjunction of UDF predicates  UDF_i(tuple) > threshold_i
 * (Hydro, Sec. 1 Listing 1 and Sec. 4.1 Listing 2).  Tuples arrive in routing
 * batches (Sec. 3.3 "Batch Evaluation"); every batch visits the predicates in
 * an order chosen from statistics the engine collects while it runs (Sec. 3.2
 * "Data Flow and Routing", Sec. 4.1 "Cost-Driven Routing Policy"): the rank
 * cost / (1 - selectivity), lowest first.  Tuples that fail a predicate are
 * dropped at once (Sec. 3.3 "Eager Materialization"), so later predicates run
 * only on survivors.  The answer is the same for every order: bit j of a
 * batch's result is 1 iff tuple j passes every predicate.
 *
 * Conventions
 *  - Every call returns a hydro_status and never aborts.  On failure,
 *    hydro_last_error() gives a message (thread-local, valid until the next
 *    call on the same thread).
 *  - Pointers named d_* are CUDA device pointers on the query's device; all
 *    others are host pointers.  Host arrays passed in are copied before the
 *    call returns (the caller keeps ownership); device arrays passed to
 *    hydro_submit_batch are BORROWED until that batch has been polled OK.
 *  - Device errors detected by kernels are latched in a per-query error word
 *    and reported as HYDRO_EDEVICE by the next poll.
 *  - A query is not thread-safe: one host thread at a time per query.
 */
#ifndef HYDRO_H
#define HYDRO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define HYDRO_API __attribute__((visibility("default")))
#else
#define HYDRO_API
#endif

#define HYDRO_MAX_PREDICATES 8
#define HYDRO_MAX_LAYERS 16

typedef struct hydro_query hydro_query;

typedef enum hydro_status {
    HYDRO_OK = 0,
    HYDRO_EINVAL = 1,       /* an argument is out of range or NULL */
    HYDRO_ENOMEM = 2,       /* a host or device allocation failed */
    HYDRO_ECUDA = 3,        /* a CUDA runtime/driver call failed */
    HYDRO_EAGAIN = 4,       /* not finished within the wait, or no free in-flight slot */
    HYDRO_ETIMEOUT = 5,     /* a bounded internal wait ran out */
    HYDRO_ESTATE = 6,       /* the call is not valid in the query's current state */
    HYDRO_EDEVICE = 7,      /* a kernel reported an error through the error word */
    HYDRO_ENOTFOUND = 8,    /* unknown or already-polled batch id */
    HYDRO_EUNSUPPORTED = 9  /* valid request the library does not implement */
} hydro_status;

/* Tuple layouts. */
enum {
    HYDRO_TUPLE_F32 = 0,        /* row-major fp32 [n][dim] feature vectors */
    HYDRO_TUPLE_U8_FRAME = 1    /* uint8 frames [n][channels][height][width] (CHW) */
};

/* Routing policies (Sec. 4.2 "System Variants"). */
enum {
    HYDRO_POLICY_RANK = 0,        /* cost/(1-s), lowest first: score-driven */
    HYDRO_POLICY_STATIC = 1,      /* fixed order (declared, or hydro_set_static_order) */
    HYDRO_POLICY_ALL = 2,         /* every predicate on every tuple, no short-circuit */
    HYDRO_POLICY_COST = 3,        /* cost only, lowest first: cost-driven */
    HYDRO_POLICY_SELECTIVITY = 4, /* selectivity only, lowest first: selectivity-driven */
    HYDRO_POLICY_LEARNED = 5      /* per-tuple order from a learned proxy of the pass
                                     probabilities (content-based routing, Sec. 2.2), trained
                                     online on the evaluated outcomes; rank routing until the
                                     first refresh.  FP32 MLP predicates only */
};

/* Working precision of UDF inference. */
enum {
    HYDRO_PREC_FP32 = 0,   /* FP32 everywhere; FP32 scores within margin_fp32 of the
                              threshold are re-evaluated in FP64 */
    HYDRO_PREC_BF16 = 1,   /* BF16 operands, FP32 accumulation on the tensor cores (the
                              first CNN layer takes FP16 operands: pixels exact as 1024 + b,
                              weights W/255 in FP16, bias folded in; frames 8..512 wide);
                              scores within margin_lowp are re-evaluated more accurately:
                              CNN UDFs first on the tensor cores in split BF16 or 3xTF32
                              (split_precision; scores within margin_tf32 go on), then in FP32
                              on CUDA cores (within margin_fp32 go on to FP64); MLP UDFs in
                              FP32 then FP64 */
    HYDRO_PREC_FP64 = 2,   /* FP64 (only for hydro_udf_scores) */
    HYDRO_PREC_TF32X3 = 3, /* 3xTF32 on the tensor cores (hi*hi + hi*lo + lo*hi): a first BF16
                              recheck level of CNN UDFs (split_precision; hydro_udf_scores on
                              BF16 CNN queries) */
    HYDRO_PREC_BF16X3 = 4, /* split BF16 on the tensor cores: x = hi + lo with hi = bf16(x),
                              lo = bf16(x - hi), products hi*hi + hi*lo + lo*hi in one BF16 GEMM
                              over [hi | hi | lo] x [W_hi | W_lo | W_hi] (about 16 significant bits);
                              the first recheck level of BF16 sessions
                              (hydro_session_udf_scores) and, by default, of BF16 CNN queries
                              ([hi | lo] BF16 planes of the activations and weights).  As the
                              working precision of a frame (CNN) query it gives FP32-class
                              scores on the tensor cores: scores within margin_tf32 go to FP32
                              on CUDA cores, and those within margin_fp32 on to FP64 */
    HYDRO_PREC_FP8 = 5     /* sessions only: the first layer of every pool UDF in the FP8 set
                              (first hidden width >= fp8_min_width) runs with E4M3 operands on
                              the tensor cores (kind::f8f6f4, FP32 accumulation): weights scaled
                              per output channel (max |w| / 448), each tuple row scaled by its
                              own max |x| / 448; its other layers and the other UDFs run in
                              BF16.  Scores within margin_lowp go to a BF16 level (FP8 set) or
                              straight to FP32 (the others), then FP32 -> FP64 as in BF16
                              sessions */
};

/* Where the router's per-tuple cost comes from. */
enum {
    HYDRO_COST_MODEL = 0,    /* flops per tuple of the UDF (or cost_hint): deterministic */
    HYDRO_COST_MEASURED = 1  /* device time per evaluated tuple (Sec. 4.2 profiles time per tuple):
                                each stage's duration is taken on the device (global timer from
                                the stage's first launch to the end of its compaction); c_i = the
                                window's stage time / tuples evaluated.  Rank and cost policies
                                with warmup_batches >= 1; orders then depend on timing, so counts
                                are checked against each batch's reported order only */
};

/* UDF kinds. */
enum {
    HYDRO_UDF_MLP = 0,   /* linear layers, ReLU between them, last layer has 1 output */
    HYDRO_UDF_CNN = 1    /* conv3x3 (stride 1, zero pad 1) + bias + ReLU layers on the
                            frame scaled by 1/255, global average pool, linear head */
};

typedef struct hydro_query_config {
    int32_t tuple_kind;      /* HYDRO_TUPLE_* */
    int32_t dim;             /* F32: features per tuple (row stride = dim floats) */
    int32_t channels;        /* U8_FRAME: frame channels (3) */
    int32_t height;          /* U8_FRAME: frame height (64) */
    int32_t width;           /* U8_FRAME: frame width (64) */
    int32_t max_batch;       /* largest n a submit may pass, 1..65536 */
    int32_t policy;          /* HYDRO_POLICY_* */
    int32_t precision;       /* HYDRO_PREC_FP32, HYDRO_PREC_BF16, or (U8_FRAME tuples, CNN
                                UDFs whose layers after the first run on the tensor cores)
                                HYDRO_PREC_BF16X3 */
    int32_t cost_source;     /* HYDRO_COST_* */
    int32_t warmup_batches;  /* adaptive policies: the first batches evaluate every
                                predicate on every tuple (Sec. 4.1 "Warmup Phase") */
    int32_t stats_window;    /* W >= 1: router uses the last W visible batches */
    int32_t route_lag;       /* 0..7: batch b is routed on batches <= b-1-lag */
    int32_t max_in_flight;   /* submitted but not yet polled batches, 1..64 */
    int32_t device;          /* CUDA device ordinal */
    void *stream;            /* cudaStream_t the batches run on; NULL = library stream */
    int32_t proxy_hidden;    /* LEARNED: proxy MLP hidden width (default 64) */
    int32_t proxy_refresh;   /* LEARNED: retrain after every this many batches (default 16) */
    int32_t proxy_epochs;    /* LEARNED: passes over the last proxy_refresh batches per retrain (2) */
    float proxy_lr;          /* LEARNED: Adam learning rate (1e-3) */
    int32_t proxy_seed;      /* LEARNED: seed of the proxy's initial weights */
    int32_t lanes;           /* 1 (default) .. 8, <= route_lag + 1: batch b runs on stream lane
                                b % lanes, each lane with its own scratch, so that up to `lanes`
                                consecutive batches run at once (batch b's order waits only for
                                batch b - 1 - route_lag).  The batches then run on library streams
                                that wait for the caller's stream at each submit.  With
                                embeddings each lane probes the shared cache into its own miss
                                list (the cache is indexed by tuple id).  Not with the LEARNED
                                policy */
    int32_t split_precision; /* BF16 queries with tensor-core CNN UDFs: the first recheck level,
                                HYDRO_PREC_BF16X3 (default; 0 also selects it: split BF16 [hi | lo]
                                operands, three BF16 passes) or HYDRO_PREC_TF32X3 (3xTF32).  On the
                                CNN workload split BF16 runs at twice the MMA rate with half the
                                operand bytes and misses FP64 by less than 3xTF32 does */
    int32_t recheck_graphs;  /* 1 (hydro_default_config): a stage's recheck levels replay from a
                                CUDA graph captured once per stream lane and predicate, each
                                level an IF node that runs only when its band is not empty (the
                                band's tuples are first copied to a per-lane staging buffer, so
                                the graph never sees the batch's own tuple pointer); 0: every
                                level's kernels are launched for every stage, empty or not */
    int32_t pipeline;        /* 1: predicates as concurrent workers on separate resources (Sec. 4.1
                                "Example comparison"): position k of every batch's order runs on a
                                stream of its own with 1/P of the SMs (every kernel's grid sized to
                                that share), so that batches flow through the positions like a
                                pipeline; batch b's position k waits for its position k - 1 only.
                                Needs lanes >= 2 (each batch in the pipeline keeps its own
                                scratch) and a query without embeddings or the LEARNED policy.
                                With the COST policy (cheapest predicate first) this is the
                                paper's cost-driven routing for concurrent predicates.
                                2: the same with hardware SM partitions: the SMs are split into
                                P equal partitions (multiples of 8 SMs; CUDA green contexts) and
                                position k's stream runs only on partition k (recheck levels are
                                then launched directly, not from graphs).  0: off */
} hydro_query_config;

typedef struct hydro_udf_desc {
    int32_t kind;                 /* HYDRO_UDF_* */
    int32_t n_layers;             /* MLP: linear layers; CNN: conv layers (1..HYDRO_MAX_LAYERS) */
    const int32_t *dims;          /* n_layers+1 widths.  MLP: dims[0] = dim, dims[n_layers] = 1.
                                     CNN: channel chain, dims[0] = channels */
    const float *const *weights;  /* per layer, fp32.  MLP: [dims[l+1]][dims[l]] row-major.
                                     CNN: [dims[l+1]][dims[l]][3][3] */
    const float *const *biases;   /* per layer, fp32 [dims[l+1]] */
    const float *head_weight;     /* CNN: [dims[n_layers]] fp32; MLP: NULL */
    double head_bias;             /* CNN: head bias; MLP: ignored */
    int64_t cost_hint;            /* > 0 replaces the model cost (flops per tuple) */
    int32_t upstream;             /* 0: the UDF reads the tuple.  >= 1: an embedding id from
                                     hydro_add_embedding; the UDF (a "head") reads that shared
                                     upstream UDF's output, which is cached per tuple id and
                                     reused by every predicate on it (dims[0] = its width) */
} hydro_udf_desc;

/* Per-batch result detail. */
typedef struct hydro_batch_info {
    int64_t n;                                  /* tuples in the batch */
    int64_t n_pass;                             /* tuples in the result */
    int32_t n_predicates;
    int32_t warmup;                             /* 1: every predicate saw every tuple */
    int32_t order[HYDRO_MAX_PREDICATES];        /* predicate ids in evaluation order */
    int64_t passed[HYDRO_MAX_PREDICATES];       /* of the tuples predicate i evaluated, how many passed */
    int64_t recheck_tf32[HYDRO_MAX_PREDICATES]; /* re-evaluated by 3xTF32 (low-precision band, CNN) */
    int64_t recheck_fp32[HYDRO_MAX_PREDICATES]; /* re-evaluated in FP32 on CUDA cores */
    int64_t recheck_fp64[HYDRO_MAX_PREDICATES]; /* re-evaluated in FP64 (FP32 band) */
    int64_t cache_hits[HYDRO_MAX_PREDICATES];   /* evaluated tuples whose upstream output was cached */
    double device_ms;                           /* GPU time from the batch's first to last kernel */
    int64_t stage_ns[HYDRO_MAX_PREDICATES];     /* HYDRO_COST_MEASURED: device ns of predicate i's stage
                                                   in this batch (0 if it did not run), else 0 */
} hydro_batch_info;

/* Cumulative per-predicate statistics (Sec. 3.3 "Metadata for Data Routing"). */
typedef struct hydro_pred_stats {
    int64_t evaluated;       /* tuples the UDF ran on at working precision */
    int64_t passed;
    int64_t recheck_tf32;
    int64_t recheck_fp32;
    int64_t recheck_fp64;
    int64_t cache_hits;
    int64_t model_cost;      /* flops per tuple used by HYDRO_COST_MODEL (a head's own cost for
                                predicates on an embedding) */
    double margin_lowp;      /* current margins */
    double margin_tf32;
    double margin_fp32;
} hydro_pred_stats;

/* Calibration report of one predicate (hydro_calibrate). */
typedef struct hydro_calib_info {
    double max_err_fp32;     /* max |s_fp32 - s_fp64| over the calibration tuples */
    double max_err_lowp;     /* max |s_bf16 - s_fp64| (BF16 queries), else 0 */
    double max_err_tf32;     /* max |s_3xtf32 - s_fp64| (BF16 CNN queries), else 0 */
    double margin_fp32;      /* margins set */
    double margin_lowp;      /* (raised if the error needed it) */
    double margin_tf32;
} hydro_calib_info;

/* One kernel class in a profile (hydro_profile_read). */
typedef struct hydro_kernel_profile {
    char name[48];           /* kernel class, e.g. "conv3x3_bf16_tc" */
    int64_t launches;        /* launches recorded */
    double total_ms;         /* sum of per-launch device durations (CUDA events) */
    double flops;            /* algorithmic flops of those launches (2 x MACs) */
    double bytes;            /* algorithmic HBM bytes: activations in + out, weights once */
} hydro_kernel_profile;

/* Fill *cfg with defaults: F32 tuples, RANK policy, FP32, MODEL cost, one
 * warmup batch, window 8, lag 1, 4 batches in flight, device 0, NULL stream.
 * dim/channels/height/width/max_batch are left 0 and must be set. */
HYDRO_API void hydro_default_config(hydro_query_config *cfg);

/* Create a query on cfg->device.  *out receives an opaque handle owned by
 * the library (free with hydro_destroy_query).  No device memory is taken
 * until the first submit or calibrate. */
HYDRO_API hydro_status hydro_create_query(const hydro_query_config *cfg, hydro_query **out);

/* Add predicate  UDF(tuple) > threshold  (strict).  The UDF's weights are
 * copied.  Only valid before the first submit/calibrate (else HYDRO_ESTATE).
 * *out_pred_id receives the predicate id (0, 1, ... in call order), which is
 * also its position in the declared order.  Default margins: margin_lowp =
 * 0.02, margin_fp32 = 1e-5 * max(1, |threshold|). */
HYDRO_API hydro_status hydro_add_predicate(hydro_query *q, const hydro_udf_desc *udf, double threshold,
                                 int32_t *out_pred_id);

/* Declare a shared upstream UDF (an MLP on the tuple whose layers are all
 * followed by ReLU; output width dims[n_layers], a multiple of 4) whose
 * outputs are cached per tuple id and reused across predicates and batches:
 * EvaDB's materialized UDF results (Sec. 2.1) feeding reuse-aware routing
 * (Sec. 4.3).  Predicates on it pass its id as hydro_udf_desc.upstream; their
 * estimated cost for a batch becomes head cost + (1 - hit rate) x this UDF's
 * cost (the reuse-aware estimate of Sec. 4.3 "Reuse-aware Routing").  Tuple
 * ids must lie in [0, id_capacity); the cache holds id_capacity x width
 * floats.  F32 tuples, FP32 queries; before the first submit.  *out_emb_id
 * receives 1, 2, ... */
HYDRO_API hydro_status hydro_add_embedding(hydro_query *q, const hydro_udf_desc *udf, int64_t id_capacity,
                                           int32_t *out_emb_id);

/* Compute and cache embedding emb for n device tuples with device ids (as an
 * earlier exploratory query would have); these entries count as cached for
 * every later batch.  Stream-ordered after the batches already submitted;
 * synchronous (returns when the cache holds them). */
HYDRO_API hydro_status hydro_cache_prefill(hydro_query *q, int32_t emb, const void *d_tuples, const int64_t *d_ids,
                                           int64_t n);

/* Forget every cached output of embedding emb (asynchronous on the query's
 * stream, ordered after the batches already submitted). */
HYDRO_API hydro_status hydro_cache_clear(hydro_query *q, int32_t emb);

/* Set the recheck margins of predicate pred (absolute score units, >= 0).
 * A score s at a precision decides the test only if |s - t| > that level's
 * margin; otherwise the tuple is re-evaluated at the next level
 * (BF16 -> 3xTF32 (CNN) -> FP32 -> FP64).  Valid before the first submit.
 * Defaults: margin_lowp 0.02, margin_tf32 5e-3*max(1,|t|), margin_fp32
 * 1e-5*max(1,|t|). */
HYDRO_API hydro_status hydro_set_margins(hydro_query *q, int32_t pred, double margin_lowp, double margin_tf32,
                                         double margin_fp32);

/* Order for HYDRO_POLICY_STATIC: a permutation of 0..P-1 (n must equal P). */
HYDRO_API hydro_status hydro_set_static_order(hydro_query *q, const int32_t *order, int32_t n);

/* Calibrate the margins on n device tuples: runs every UDF in FP64, FP32 and
 * (BF16 queries) BF16 and 3xTF32 on the GPU and sets margin_fp32 = 16 * max
 * FP32 error and margin_tf32 = 8 * max 3xTF32 error (each at least
 * 1e-9 * max |score|), and raises margin_lowp to 4 * max BF16 error if that
 * is larger.  info[P] (nullable) receives the report.  Valid before the
 * first submit; synchronous. */
HYDRO_API hydro_status hydro_calibrate(hydro_query *q, const void *d_tuples, int64_t n, hydro_calib_info *info);

/* Scores of predicate pred's UDF on n device tuples at precision prec
 * (HYDRO_PREC_FP64/FP32/BF16/TF32X3) into d_scores (device, n doubles).
 * Synchronous; for tests, calibration and error reports. */
HYDRO_API hydro_status hydro_udf_scores(hydro_query *q, int32_t pred, int32_t prec, const void *d_tuples,
                              int64_t n, double *d_scores);

/* Submit a batch of n tuples (0 <= n <= max_batch).  d_tuples: device, layout
 * of cfg->tuple_kind; d_ids: device int64 tuple ids (required when the query
 * has an embedding, else may be NULL).  Stream-ordered
 * and asynchronous; it may wait for the batch submitted route_lag+1 earlier
 * to be routed (bounded).  *out_batch_id receives 0, 1, 2, ... */
HYDRO_API hydro_status hydro_submit_batch(hydro_query *q, const void *d_tuples, const int64_t *d_ids, int64_t n,
                                int64_t *out_batch_id);

/* Result of batch batch_id.  pass_bitmap: host, ceil(n/32) words, bit j of
 * word j/32 (LSB first) = tuple j passed every predicate.  eval_counts: host
 * [P], tuples each predicate evaluated at working precision (nullable).
 * info nullable.  wait_ms: 0 = do not wait, < 0 = wait without limit, else
 * wait up to wait_ms.  HYDRO_EAGAIN if not finished in time. */
HYDRO_API hydro_status hydro_poll_result(hydro_query *q, int64_t batch_id, uint32_t *pass_bitmap,
                               int64_t *eval_counts, hydro_batch_info *info, int32_t wait_ms);

/* Per-tuple trace of the most recently submitted batch (polled, no later
 * submit): order[n * 8] receives each tuple's predicate order (first P
 * bytes used) and visited[n] the bit set of predicates it was evaluated on.
 * For per-batch policies every tuple shows the batch's order.  Synchronous. */
HYDRO_API hydro_status hydro_debug_trace(hydro_query *q, int64_t batch_id, uint8_t *order, uint8_t *visited);

/* Cumulative statistics of the first n predicates into out[n] (host). */
HYDRO_API hydro_status hydro_get_stats(hydro_query *q, hydro_pred_stats *out, int32_t n);

/* Start (enable = 1, clearing earlier records) or stop (enable = 0)
 * per-launch timing of the UDF layer kernels: each recorded launch is
 * bracketed by CUDA events on the query's stream.  Also resets the launch
 * counter read by hydro_profile_read (waits for the query's batches to
 * finish first).  With recheck_graphs the recheck levels replay from graphs
 * and are not timed; their kernels are counted on the device. */
HYDRO_API hydro_status hydro_profile(hydro_query *q, int32_t enable);

/* Per kernel class totals since the last hydro_profile(q, 1), for batches
 * polled since then.  out[max] receives up to max classes, *n_out how many;
 * *total_launches (nullable) every kernel this query launched since then,
 * counting inside recheck graphs the gates and the bodies that ran.
 * Synchronises the query's stream. */
HYDRO_API hydro_status hydro_profile_read(hydro_query *q, hydro_kernel_profile *out, int32_t max, int32_t *n_out,
                                          int64_t *total_launches);

/* Allocation-free FP32 MLP scores.  The paper has no counterpart: this
 * entry point is for callers that cannot allocate device memory once they
 * are running: code inside a framework that owns the device memory pool and
 * forbids allocations from outside it, a latency-bound service that cannot
 * take the device-wide synchronisation and unbounded time of a cudaMalloc,
 * or a process that reserved nearly all device memory up front.  It
 * computes the same scores as hydro_udf_scores(FP32) on an MLP UDF, with
 * the caller's device buffers:
 *   d_x        device fp32 [n][dims[0]] tuples
 *   dims       host, n_layers+1 widths, dims[n_layers] == 1
 *   d_weights  host array of n_layers DEVICE pointers, layer l [dims[l+1]][dims[l]]
 *   d_biases   host array of n_layers DEVICE pointers, layer l [dims[l+1]]
 *   d_scores   device double [n] (output)
 *   stream     cudaStream_t (NULL = legacy default stream)
 * The activations between layers live in one static device array of the
 * library (two buffers of 1,048,576 floats, 8 MiB), which every GPU that
 * loads the library holds until the process exits; n times the widest
 * hidden layer must not exceed 1,048,576 (else HYDRO_EINVAL).  It calls no
 * allocator.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current, so make that
 * first call before any stream capture.  The address is kept for the life
 * of the process: do not cudaDeviceReset a device this entry point is used on.  All calls share the array and keep
 * the last call's contents: calls whose kernels overlap on the GPU (other
 * streams, other threads) race on it and must be serialised by the caller.
 * Asynchronous on `stream`; errors are returned as status codes. */
HYDRO_API hydro_status hydro_mlp_scores_noalloc(const float *d_x, int64_t n, int32_t n_layers, const int32_t *dims,
                                                const float *const *d_weights, const float *const *d_biases,
                                                double *d_scores, void *stream);

/* Failure-detection self-test of the kernels' bounded waits: a kernel waits
 * on an mbarrier that nothing completes, with a limit of limit_ns (1e3 ..
 * 1e10); the wait must run out, the kernel return and the context stay
 * usable.  Returns HYDRO_ETIMEOUT when that happened (the expected outcome).
 * No counterpart in the paper (its deadlock avoidance is a queue-capacity
 * rule, Sec. 3.3 "Deadlock Prevention"); every spin in this library's
 * kernels is bounded the same way. */
HYDRO_API hydro_status hydro_selftest_bounded_wait(int32_t device, int64_t limit_ns);

/* ------------------------------------------------------------ sessions
 *
 * Many concurrent queries over one shared pool of MLP UDFs.  The paper's
 * Laminar operator (Sec. 5.1 "Batch-agnostic Parallelization", Sec. 5.3
 * "Data-Aware Load Balancing") runs several predicate workers at once because
 * one worker on small routing batches leaves the GPU mostly idle (Sec. 5.2
 * "GPU Utilization Study": about 20 %).  A session does the same work
 * inside the GPU: in a step, every query contributes its next chunk of
 * tuples; in round r every surviving tuple goes to the pool UDF of the r-th
 * predicate of its query's current order; all queries' work on one UDF forms
 * one group, and all groups of a layer depth run in ONE persistent grouped
 * launch whose tile scheduler balances the uneven group sizes.  A step's
 * launches are stream-ordered and device-driven (counts, orders and lists
 * live on the GPU), so they replay from a captured CUDA graph.
 *
 * Each query is routed exactly as a single query would be with route_lag 0
 * (Sec. 4.1): its k-th step with tuples is its batch k, ordered by rank
 * cost/(1-s) over its own window of earlier batches (ties to the lower slot),
 * its first warmup_batches batches evaluating every predicate on every tuple.
 * Its pass set, orders and counts therefore equal those of that query run
 * alone over the same chunks.
 */
#define HYDRO_MAX_QUERIES 512
#define HYDRO_MAX_POOL 8

typedef struct hydro_session hydro_session;

typedef struct hydro_session_config {
    int32_t dim;              /* features per fp32 tuple row; a multiple of 64 */
    int32_t max_step_tuples;  /* largest sum of counts one step may pass, 1..4194304 */
    int32_t precision;        /* HYDRO_PREC_FP32, HYDRO_PREC_BF16 (tensor cores, pool UDFs
                                 whose widths are multiples of 64) or HYDRO_PREC_FP8 (as BF16,
                                 dim a multiple of 128) */
    int32_t warmup_batches;   /* per query, as in hydro_query_config */
    int32_t stats_window;     /* per query, W >= 1 */
    int32_t use_graphs;       /* 1: each in-flight slot replays its step from a CUDA graph
                                 captured at its first use; 0: launch kernel by kernel */
    int32_t autotune;         /* 1: at the first submit, time every tensor-core tile width
                                 (64/128/256 columns) of every pool layer and keep the fastest */
    int32_t max_in_flight;    /* submitted, unpolled steps, 1..8 */
    int32_t device;           /* CUDA device ordinal */
    void *stream;             /* cudaStream_t the steps run on; NULL = library stream */
    int32_t learned;          /* 1: per-tuple orders from a learned proxy of the pass probabilities
                                 (content-based routing, Sec. 2.2), as HYDRO_POLICY_LEARNED does for
                                 one query: a proxy MLP dim -> proxy_hidden -> P predicts each slot's
                                 pass probability p, each tuple visits its slots by c (1 + e^z),
                                 z = logit(p); trained online (Adam, masked BCE) on the outcomes of
                                 the last proxy_refresh batches every proxy_refresh batches, on a
                                 stream of its own: a training launched after step j takes effect
                                 from step j + 2 on (it overlaps step j + 1); rank orders until
                                 the first training.  Sessions with one query only */
    int32_t proxy_hidden;     /* learned: proxy hidden width (default 64) */
    int32_t proxy_refresh;    /* learned: train after every this many steps (default 16) */
    int32_t proxy_epochs;     /* learned: passes over the stored steps per training (default 1) */
    float proxy_lr;           /* learned: Adam learning rate (default 1e-3) */
    int32_t proxy_seed;       /* learned: seed of the proxy's initial weights */
    int32_t batches_per_step; /* K, 1..32 (n_queries x K <= 512): routing batches of each query one
                                 step may hold; with K > 1
                                 counts (submit) and the per-query results (poll) have n_queries x K
                                 entries, entry q K + k being query q's k-th batch of the step */
    int32_t route_lag;        /* a query's batch b is routed on its batches <= b - 1 - route_lag
                                 (Sec. 4.1 with a lag, as hydro_query_config.route_lag); must be
                                 >= K - 1 so that every batch of a step sees only earlier steps */
    int32_t fp8_min_width;    /* HYDRO_PREC_FP8: pool UDFs whose first hidden layer has at least
                                 this many outputs form the FP8 set (0: 1024) */
    int32_t proxy_rows;       /* learned: rows of one stored step that one Adam step trains on
                                 (0: all of them); a contiguous window that moves on by
                                 proxy_rows at every Adam step, so that the stored rows are
                                 used in turn */
    int32_t policy;           /* HYDRO_POLICY_RANK (default: per-batch rank order) or
                                 HYDRO_POLICY_STATIC (every batch in the query's declared slot
                                 order, no warmup batches) */
    int32_t tile_sched;       /* tile scheduling of the grouped tensor-core launches:
                                 0 = static round robin over the tiles in UDF order;
                                 1 = data-aware (Sec. 5.3 "Data-Aware Load Balancing" on one GPU):
                                 tiles numbered by estimated work (K x tile width), heaviest
                                 first, each CTA claiming its next tile when it is ready for one */
} hydro_session_config;

/* Load balance of a session's grouped tensor-core launches (Sec. 5.3 and
 * 5.4: per-worker load), measured on the device: each CTA (one per SM)
 * stamps the global timer when it starts and when its last tile is done. */
#define HYDRO_BALANCE_CTAS 160
typedef struct hydro_balance_info {
    int64_t launches;         /* grouped launches measured (with at least one tile) */
    int32_t ctas;             /* most CTAs with work in one launch */
    int32_t reserved;
    double makespan_ms;       /* sum over launches: last CTA end - first CTA start */
    double busy_mean_ms;      /* sum over launches: mean busy time of the CTAs with work */
    double busy_max_ms;       /* sum over launches: the longest CTA busy time */
    double cta_busy_ms[HYDRO_BALANCE_CTAS];   /* per CTA index: busy time summed over the launches */
} hydro_balance_info;

/* Per query result of one step (hydro_session_poll). */
typedef struct hydro_step_query {
    int64_t n;                                   /* the query's tuples in the step */
    int64_t n_pass;                              /* of them, in the result */
    int64_t batch;                               /* the query's batch number (-1: no tuples) */
    int32_t warmup;                              /* 1: every predicate saw every tuple */
    int32_t order[HYDRO_MAX_PREDICATES];         /* slots in evaluation order (first n_preds) */
    int64_t evaluated[HYDRO_MAX_PREDICATES];     /* per slot: tuples evaluated at working precision */
    int64_t passed[HYDRO_MAX_PREDICATES];        /* per slot: of those, passed */
    int64_t recheck_split[HYDRO_MAX_PREDICATES]; /* per slot: re-evaluated at level 1 (split BF16 in BF16
                                                    sessions, BF16 in FP8 sessions) */
    int64_t recheck_fp32[HYDRO_MAX_PREDICATES];  /* per slot: re-evaluated in FP32 (BF16 sessions) */
    int64_t recheck_fp64[HYDRO_MAX_PREDICATES];  /* per slot: re-evaluated in FP64 */
} hydro_step_query;

/* Autotuner record of one pool layer (hydro_session_tuning). */
typedef struct hydro_tile_choice {
    int32_t udf, layer;       /* pool UDF and hidden layer */
    int32_t K, N;             /* layer shape */
    int32_t tile_n;           /* chosen tensor-core tile width (columns) */
    double us[3];             /* measured microseconds for tile widths 64, 128, 256 (0: not tried) */
} hydro_tile_choice;

/* Defaults: FP32, warmup 1, window 8, graphs on, autotune on, 2 in flight,
 * device 0, NULL stream, not learned (proxy 64 hidden, refresh 16, 1 epoch,
 * lr 1e-3, seed 1), one batch per step, route lag 0; dim and
 * max_step_tuples must be set. */
HYDRO_API void hydro_session_default_config(hydro_session_config *cfg);

HYDRO_API hydro_status hydro_session_create(const hydro_session_config *cfg, hydro_session **out);

/* Add pool UDF *out_udf = 0, 1, ... (an MLP, dims[0] = dim, dims[n_layers] = 1,
 * at most HYDRO_MAX_POOL).  Weights copied.  Before the first submit.
 * Default margins: margin_lowp 0.02, margin_fp32 1e-5. */
HYDRO_API hydro_status hydro_session_add_udf(hydro_session *s, const hydro_udf_desc *udf, int32_t *out_udf);

/* Add query *out_query = 0, 1, ...: the conjunction over slots k < n_preds
 * (1..HYDRO_MAX_PREDICATES) of  pool UDF udfs[k] (distinct) > thresholds[k].
 * Before the first submit. */
HYDRO_API hydro_status hydro_session_add_query(hydro_session *s, int32_t n_preds, const int32_t *udfs,
                                               const double *thresholds, int32_t *out_query);

/* Margins of pool UDF udf (absolute score units, >= 0): a score within its
 * level's margin of a threshold is re-evaluated at the next level (BF16
 * sessions: BF16 -> split BF16 -> FP32 -> FP64; FP8 sessions: FP8 -> BF16 ->
 * FP32 -> FP64 for the FP8 set, BF16 -> FP32 -> FP64 for the others, so
 * margin_split is the BF16 level's margin there; FP32 sessions: FP32 ->
 * FP64).  Defaults: margin_lowp 0.02, margin_split 1e-3, margin_fp32 1e-5.
 * Before the first submit. */
HYDRO_API hydro_status hydro_session_set_margins(hydro_session *s, int32_t udf, double margin_lowp,
                                                 double margin_split, double margin_fp32);

/* Calibrate every pool UDF's margins on n device tuples, with the rule of
 * hydro_calibrate (margin_fp32 = 16 x max FP32 error, margin_split = 8 x max
 * split-BF16 error, each at least 1e-9 x max |score|; margin_lowp raised to
 * 4 x max BF16 error).  FP8 sessions: margin_lowp raised to 4 x the max
 * error of the level-0 scores (HYDRO_PREC_FP8), margin_split = 4 x max BF16
 * error (at least 1e-9 x max |score|).  info[n_udfs] nullable (max_err_tf32
 * / margin_tf32 report level 1: split BF16, or BF16 in FP8 sessions).
 * Synchronous. */
HYDRO_API hydro_status hydro_session_calibrate(hydro_session *s, const void *d_tuples, int64_t n,
                                               hydro_calib_info *info);

/* Scores of pool UDF udf on n device tuples at HYDRO_PREC_FP64/FP32/BF16/
 * BF16X3, or FP8 (an FP8 session's level-0 scores: FP8 first layer for the
 * FP8 set, BF16 for the others) into d_scores (device, n doubles).
 * Synchronous. */
HYDRO_API hydro_status hydro_session_udf_scores(hydro_session *s, int32_t udf, int32_t prec, const void *d_tuples,
                                                int64_t n, double *d_scores);

/* Submit one step.  d_tuples: device fp32 rows, 16-byte aligned, counts[0]
 * rows of query 0, then counts[1] rows of query 1, ... (BORROWED until the
 * step is polled).  With K = batches_per_step > 1, counts has n_queries x K
 * entries (query q's batches k = 0..K-1 at q K + k, stacked in that order; a
 * query's non-empty batches come first).
 * counts: host, each >= 0, sum <= max_step_tuples.  A query with
 * count 0 sits the step out (its batch number does not advance).
 * Asynchronous; *out_step receives 0, 1, 2, ... */
HYDRO_API hydro_status hydro_session_submit(hydro_session *s, const void *d_tuples, const int32_t *counts,
                                            int64_t *out_step);

/* Result of a step.  pass_bitmap: host, ceil(total/32) words, bit j = the
 * j-th stacked tuple passed every predicate of its query.  per_query: host
 * [n_queries x K] (nullable), one entry per (query, batch of the step).  device_ms (nullable): GPU time of the step.
 * wait_ms as in hydro_poll_result; HYDRO_EAGAIN if not finished. */
HYDRO_API hydro_status hydro_session_poll(hydro_session *s, int64_t step, uint32_t *pass_bitmap,
                                          hydro_step_query *per_query, double *device_ms, int32_t wait_ms);

/* Per-tuple trace of step `step` (polled, and the last step submitted):
 * order[total * 8] receives each stacked tuple's slot order (first n_preds
 * bytes of its query used) and visited[total] the bit set of slots it was
 * evaluated on.  Synchronous. */
HYDRO_API hydro_status hydro_session_debug_trace(hydro_session *s, int64_t step, uint8_t *order, uint8_t *visited);

/* Autotuner records (after the first submit): out[max], *n_out written. */
HYDRO_API hydro_status hydro_session_tuning(hydro_session *s, hydro_tile_choice *out, int32_t max, int32_t *n_out);

/* Start (enable = 1, clearing earlier records) or stop per-class timing of a
 * session's kernels: while on, steps launch kernel by kernel (no graph)
 * with CUDA events around each launch class; also resets the launch counter.
 * No step may be in flight. */
HYDRO_API hydro_status hydro_session_profile(hydro_session *s, int32_t enable);

/* Per kernel class launches and device ms of the steps polled since the
 * last hydro_session_profile(s, 1) (flops and bytes are left 0: they depend
 * on the per-query counts the caller reads from the polls); *total_launches
 * (nullable) = kernel launches of all steps polled since then, graph
 * replays included. */
/* Start (enable = 1, clearing the totals) or stop (enable = 0) collecting the
 * load balance of the grouped launches of the steps polled from now on (a
 * device-to-host copy of the step's records at each poll); any other value
 * only reads.  out (nullable) receives the totals so far.  No step may be in
 * flight when collection starts or stops. */
HYDRO_API hydro_status hydro_session_balance(hydro_session *s, int32_t enable, hydro_balance_info *out);

HYDRO_API hydro_status hydro_session_profile_read(hydro_session *s, hydro_kernel_profile *out, int32_t max,
                                                  int32_t *n_out, int64_t *total_launches);

/* Wait for outstanding steps (bounded), free every resource of s. */
HYDRO_API hydro_status hydro_session_destroy(hydro_session *s);

/* Wait for outstanding work (bounded), free every resource of q. */
HYDRO_API hydro_status hydro_destroy_query(hydro_query *q);

/* Message of the last failed call on this thread ("" if none). */
HYDRO_API const char *hydro_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HYDRO_H */
