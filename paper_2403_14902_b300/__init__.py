"""Python binding of the adaptive ML-predicate engine (``include/hydro.h``).

Argument marshalling only: every step of the batch path (UDF inference,
threshold tests and rechecks, compaction, statistics, routing, the result
bitmap) runs in the CUDA kernels of ``libhydro.so``.  PyTorch supplies device
memory and streams.  Importing this module loads the library and fails loudly
if it has not been built (``python -m paper_2403_14902_b300.build``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhydro.so")

MAX_PREDICATES = 8
MAX_LAYERS = 16

STATUS = {0: "HYDRO_OK", 1: "HYDRO_EINVAL", 2: "HYDRO_ENOMEM", 3: "HYDRO_ECUDA", 4: "HYDRO_EAGAIN",
          5: "HYDRO_ETIMEOUT", 6: "HYDRO_ESTATE", 7: "HYDRO_EDEVICE", 8: "HYDRO_ENOTFOUND",
          9: "HYDRO_EUNSUPPORTED"}
OK, EINVAL, ENOMEM, ECUDA, EAGAIN, ETIMEOUT, ESTATE, EDEVICE, ENOTFOUND, EUNSUPPORTED = range(10)

TUPLE_F32, TUPLE_U8_FRAME = 0, 1
POLICIES = {"rank": 0, "static": 1, "all": 2, "cost": 3, "selectivity": 4, "learned": 5}
PRECISIONS = {"fp32": 0, "bf16": 1, "fp64": 2, "tf32x3": 3, "bf16x3": 4, "fp8": 5}
COSTS = {"model": 0, "measured": 1}
UDF_MLP, UDF_CNN = 0, 1

EXPORTED = ["hydro_default_config", "hydro_create_query", "hydro_add_predicate", "hydro_add_embedding",
            "hydro_cache_prefill", "hydro_cache_clear", "hydro_set_margins",
            "hydro_set_static_order", "hydro_calibrate", "hydro_udf_scores", "hydro_submit_batch",
            "hydro_poll_result", "hydro_debug_trace", "hydro_get_stats", "hydro_profile", "hydro_profile_read",
            "hydro_mlp_scores_noalloc", "hydro_selftest_bounded_wait",
            "hydro_session_default_config", "hydro_session_create", "hydro_session_add_udf",
            "hydro_session_add_query", "hydro_session_set_margins", "hydro_session_calibrate",
            "hydro_session_udf_scores", "hydro_session_submit", "hydro_session_poll", "hydro_session_tuning",
            "hydro_session_profile", "hydro_session_profile_read", "hydro_session_debug_trace", "hydro_session_balance",
            "hydro_session_destroy", "hydro_destroy_query", "hydro_last_error"]
MAX_QUERIES = 512
MAX_POOL = 8


class QueryConfig(ctypes.Structure):
    _fields_ = [("tuple_kind", ctypes.c_int32), ("dim", ctypes.c_int32), ("channels", ctypes.c_int32),
                ("height", ctypes.c_int32), ("width", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("policy", ctypes.c_int32), ("precision", ctypes.c_int32), ("cost_source", ctypes.c_int32),
                ("warmup_batches", ctypes.c_int32), ("stats_window", ctypes.c_int32),
                ("route_lag", ctypes.c_int32), ("max_in_flight", ctypes.c_int32), ("device", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("proxy_hidden", ctypes.c_int32), ("proxy_refresh", ctypes.c_int32),
                ("proxy_epochs", ctypes.c_int32), ("proxy_lr", ctypes.c_float), ("proxy_seed", ctypes.c_int32),
                ("lanes", ctypes.c_int32), ("split_precision", ctypes.c_int32), ("recheck_graphs", ctypes.c_int32),
                ("pipeline", ctypes.c_int32)]


class UdfDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n_layers", ctypes.c_int32),
                ("dims", ctypes.POINTER(ctypes.c_int32)),
                ("weights", ctypes.POINTER(ctypes.POINTER(ctypes.c_float))),
                ("biases", ctypes.POINTER(ctypes.POINTER(ctypes.c_float))),
                ("head_weight", ctypes.POINTER(ctypes.c_float)), ("head_bias", ctypes.c_double),
                ("cost_hint", ctypes.c_int64), ("upstream", ctypes.c_int32)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_pass", ctypes.c_int64), ("n_predicates", ctypes.c_int32),
                ("warmup", ctypes.c_int32), ("order", ctypes.c_int32 * MAX_PREDICATES),
                ("passed", ctypes.c_int64 * MAX_PREDICATES), ("recheck_tf32", ctypes.c_int64 * MAX_PREDICATES),
                ("recheck_fp32", ctypes.c_int64 * MAX_PREDICATES),
                ("recheck_fp64", ctypes.c_int64 * MAX_PREDICATES), ("cache_hits", ctypes.c_int64 * MAX_PREDICATES),
                ("device_ms", ctypes.c_double), ("stage_ns", ctypes.c_int64 * MAX_PREDICATES)]


class PredStats(ctypes.Structure):
    _fields_ = [("evaluated", ctypes.c_int64), ("passed", ctypes.c_int64), ("recheck_tf32", ctypes.c_int64),
                ("recheck_fp32", ctypes.c_int64), ("recheck_fp64", ctypes.c_int64), ("cache_hits", ctypes.c_int64),
                ("model_cost", ctypes.c_int64),
                ("margin_lowp", ctypes.c_double), ("margin_tf32", ctypes.c_double), ("margin_fp32", ctypes.c_double)]


class CalibInfo(ctypes.Structure):
    _fields_ = [("max_err_fp32", ctypes.c_double), ("max_err_lowp", ctypes.c_double),
                ("max_err_tf32", ctypes.c_double), ("margin_fp32", ctypes.c_double),
                ("margin_lowp", ctypes.c_double), ("margin_tf32", ctypes.c_double)]


class SessionConfig(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("max_step_tuples", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("warmup_batches", ctypes.c_int32), ("stats_window", ctypes.c_int32), ("use_graphs", ctypes.c_int32),
                ("autotune", ctypes.c_int32), ("max_in_flight", ctypes.c_int32), ("device", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("learned", ctypes.c_int32), ("proxy_hidden", ctypes.c_int32),
                ("proxy_refresh", ctypes.c_int32), ("proxy_epochs", ctypes.c_int32), ("proxy_lr", ctypes.c_float),
                ("proxy_seed", ctypes.c_int32), ("batches_per_step", ctypes.c_int32), ("route_lag", ctypes.c_int32),
                ("fp8_min_width", ctypes.c_int32), ("proxy_rows", ctypes.c_int32), ("policy", ctypes.c_int32),
                ("tile_sched", ctypes.c_int32)]


BALANCE_CTAS = 160


class BalanceInfo(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("ctas", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("makespan_ms", ctypes.c_double), ("busy_mean_ms", ctypes.c_double), ("busy_max_ms", ctypes.c_double),
                ("cta_busy_ms", ctypes.c_double * BALANCE_CTAS)]


class StepQuery(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_pass", ctypes.c_int64), ("batch", ctypes.c_int64),
                ("warmup", ctypes.c_int32), ("order", ctypes.c_int32 * MAX_PREDICATES),
                ("evaluated", ctypes.c_int64 * MAX_PREDICATES), ("passed", ctypes.c_int64 * MAX_PREDICATES),
                ("recheck_split", ctypes.c_int64 * MAX_PREDICATES), ("recheck_fp32", ctypes.c_int64 * MAX_PREDICATES),
                ("recheck_fp64", ctypes.c_int64 * MAX_PREDICATES)]


class TileChoice(ctypes.Structure):
    _fields_ = [("udf", ctypes.c_int32), ("layer", ctypes.c_int32), ("K", ctypes.c_int32), ("N", ctypes.c_int32),
                ("tile_n", ctypes.c_int32), ("us", ctypes.c_double * 3)]


class KernelProfile(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double),
                ("flops", ctypes.c_double), ("bytes", ctypes.c_double)]


_lib = None


def load():
    """Load ``libhydro.so`` (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run python -m paper_2403_14902_b300.build")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    vp, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    L.hydro_default_config.argtypes = [P(QueryConfig)]
    L.hydro_default_config.restype = None
    L.hydro_create_query.argtypes = [P(QueryConfig), P(vp)]
    L.hydro_add_predicate.argtypes = [vp, P(UdfDesc), f64, P(i32)]
    L.hydro_set_margins.argtypes = [vp, i32, f64, f64, f64]
    L.hydro_add_embedding.argtypes = [vp, P(UdfDesc), i64, P(i32)]
    L.hydro_cache_prefill.argtypes = [vp, i32, vp, vp, i64]
    L.hydro_cache_clear.argtypes = [vp, i32]
    L.hydro_set_static_order.argtypes = [vp, P(i32), i32]
    L.hydro_calibrate.argtypes = [vp, vp, i64, P(CalibInfo)]
    L.hydro_udf_scores.argtypes = [vp, i32, i32, vp, i64, vp]
    L.hydro_submit_batch.argtypes = [vp, vp, vp, i64, P(i64)]
    L.hydro_poll_result.argtypes = [vp, i64, P(ctypes.c_uint32), P(i64), P(BatchInfo), i32]
    L.hydro_get_stats.argtypes = [vp, P(PredStats), i32]
    L.hydro_debug_trace.argtypes = [vp, i64, P(ctypes.c_uint8), P(ctypes.c_uint8)]
    L.hydro_profile.argtypes = [vp, i32]
    L.hydro_profile_read.argtypes = [vp, P(KernelProfile), i32, P(i32), P(i64)]
    L.hydro_mlp_scores_noalloc.argtypes = [vp, i64, i32, P(i32), P(vp), P(vp), vp, vp]
    L.hydro_selftest_bounded_wait.argtypes = [i32, i64]
    L.hydro_destroy_query.argtypes = [vp]
    L.hydro_session_default_config.argtypes = [P(SessionConfig)]
    L.hydro_session_create.argtypes = [P(SessionConfig), P(vp)]
    L.hydro_session_add_udf.argtypes = [vp, P(UdfDesc), P(i32)]
    L.hydro_session_add_query.argtypes = [vp, i32, P(i32), P(f64), P(i32)]
    L.hydro_session_set_margins.argtypes = [vp, i32, f64, f64, f64]
    L.hydro_session_calibrate.argtypes = [vp, vp, i64, P(CalibInfo)]
    L.hydro_session_udf_scores.argtypes = [vp, i32, i32, vp, i64, vp]
    L.hydro_session_submit.argtypes = [vp, vp, P(i32), P(i64)]
    L.hydro_session_poll.argtypes = [vp, i64, P(ctypes.c_uint32), P(StepQuery), P(f64), i32]
    L.hydro_session_tuning.argtypes = [vp, P(TileChoice), i32, P(i32)]
    L.hydro_session_destroy.argtypes = [vp]
    L.hydro_session_profile.argtypes = [vp, i32]
    L.hydro_session_balance.argtypes = [vp, i32, P(BalanceInfo)]
    L.hydro_session_debug_trace.argtypes = [vp, i64, P(ctypes.c_uint8), P(ctypes.c_uint8)]
    L.hydro_session_profile_read.argtypes = [vp, P(KernelProfile), i32, P(i32), P(i64)]
    L.hydro_last_error.argtypes = []
    L.hydro_last_error.restype = ctypes.c_char_p
    for name in EXPORTED[1:-1]:
        getattr(L, name).restype = ctypes.c_int
    L.hydro_session_default_config.restype = None
    _lib = L
    return L


class HydroError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = load().hydro_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


def _check(rc: int, where: str):
    if rc != OK:
        raise HydroError(rc, where)


def _ptr(t) -> int:
    """Device (or host) address of a torch tensor / numpy array, or 0."""
    if t is None:
        return 0
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    return t.ctypes.data


class Query:
    """One query: a conjunction of UDF predicates over a tuple stream.

    ``kind`` is ``"vec"`` (fp32 rows of ``dim`` features) or ``"frame"``
    (uint8 ``frame = (C, H, W)``)."""

    def __init__(self, kind: str, *, dim: int = 0, frame=(3, 64, 64), max_batch: int, policy: str = "rank",
                 precision: str = "fp32", warmup: int = 1, window: int = 8, lag: int = 1,
                 max_in_flight: int = 4, device: int = 0, stream=None, proxy_hidden: int = 64,
                 proxy_refresh: int = 16, proxy_epochs: int = 2, proxy_lr: float = 1e-3, proxy_seed: int = 1,
                 lanes: int = 1, cost: str = "model", split: str = "bf16x3", recheck_graphs: bool = True,
                 pipeline: bool = False):
        L = load()
        cfg = QueryConfig()
        L.hydro_default_config(ctypes.byref(cfg))
        cfg.tuple_kind = TUPLE_F32 if kind == "vec" else TUPLE_U8_FRAME
        cfg.dim = dim
        cfg.channels, cfg.height, cfg.width = frame
        cfg.max_batch = max_batch
        cfg.policy = POLICIES[policy]
        cfg.precision = PRECISIONS[precision]
        cfg.warmup_batches = warmup
        cfg.stats_window = window
        cfg.route_lag = lag
        cfg.max_in_flight = max_in_flight
        cfg.device = device
        cfg.stream = stream.cuda_stream if stream is not None else None
        cfg.proxy_hidden = proxy_hidden
        cfg.proxy_refresh = proxy_refresh
        cfg.proxy_epochs = proxy_epochs
        cfg.proxy_lr = proxy_lr
        cfg.proxy_seed = proxy_seed
        cfg.lanes = lanes
        cfg.cost_source = COSTS[cost]
        cfg.split_precision = PRECISIONS[split]
        cfg.recheck_graphs = 1 if recheck_graphs else 0
        cfg.pipeline = {False: 0, True: 1, "shares": 1, "partitions": 2}[pipeline]
        self.kind = kind
        self.policy = policy
        self.cfg = cfg
        self._h = ctypes.c_void_p()
        _check(L.hydro_create_query(ctypes.byref(cfg), ctypes.byref(self._h)), "hydro_create_query")
        self.n_pred = 0
        self._n_of = {}

    # -- predicates
    def _desc(self, kind, dims, Ws, bs, head_w=None, head_b=0.0, cost_hint=0, upstream=0):
        FP = ctypes.POINTER(ctypes.c_float)
        Ws = [np.ascontiguousarray(w, np.float32) for w in Ws]
        bs = [np.ascontiguousarray(b, np.float32) for b in bs]
        keep = [Ws, bs]
        d = (ctypes.c_int32 * len(dims))(*dims)
        wp = (FP * len(Ws))(*[w.ctypes.data_as(FP) for w in Ws])
        bp = (FP * len(bs))(*[b.ctypes.data_as(FP) for b in bs])
        desc = UdfDesc()
        desc.kind = kind
        desc.n_layers = len(Ws)
        desc.dims = d
        desc.weights = wp
        desc.biases = bp
        if head_w is not None:
            head_w = np.ascontiguousarray(head_w, np.float32)
            keep.append(head_w)
            desc.head_weight = head_w.ctypes.data_as(FP)
        desc.head_bias = float(head_b)
        desc.cost_hint = int(cost_hint)
        desc.upstream = int(upstream)
        return desc, (keep, d, wp, bp)

    def add_embedding(self, layers, id_capacity: int, cost_hint: int = 0) -> int:
        """Shared upstream MLP (all layers ReLU) whose outputs are cached per tuple id."""
        dims = [layers[0][0].shape[1]] + [W.shape[0] for W, _ in layers]
        desc, keep = self._desc(UDF_MLP, dims, [W for W, _ in layers], [b for _, b in layers], cost_hint=cost_hint)
        eid = ctypes.c_int32()
        _check(load().hydro_add_embedding(self._h, ctypes.byref(desc), int(id_capacity), ctypes.byref(eid)),
               "hydro_add_embedding")
        return eid.value

    def cache_prefill(self, emb: int, tuples, ids):
        _check(load().hydro_cache_prefill(self._h, int(emb), _ptr(tuples), _ptr(ids), int(tuples.shape[0])),
               "hydro_cache_prefill")

    def cache_clear(self, emb: int):
        _check(load().hydro_cache_clear(self._h, int(emb)), "hydro_cache_clear")

    def _add(self, kind, dims, Ws, bs, threshold, head_w=None, head_b=0.0, cost_hint=0, upstream=0):
        desc, keep = self._desc(kind, dims, Ws, bs, head_w, head_b, cost_hint, upstream)
        pid = ctypes.c_int32()
        _check(load().hydro_add_predicate(self._h, ctypes.byref(desc), float(threshold), ctypes.byref(pid)),
               "hydro_add_predicate")
        self.n_pred += 1
        return pid.value

    def add_mlp(self, layers, threshold: float, cost_hint: int = 0, upstream: int = 0) -> int:
        """``layers``: [(W [out, in] fp32, b [out] fp32)], last layer 1 output;
        with ``upstream`` (an embedding id) the layers are the head on it."""
        dims = [layers[0][0].shape[1]] + [W.shape[0] for W, _ in layers]
        return self._add(UDF_MLP, dims, [W for W, _ in layers], [b for _, b in layers], threshold,
                         cost_hint=cost_hint, upstream=upstream)

    def add_cnn(self, udf, threshold: float, cost_hint: int = 0) -> int:
        """``udf = (convs, (head_w, head_b))`` with convs [(W [Cout, Cin, 3, 3], b)]."""
        convs, (hw, hb) = udf
        dims = [convs[0][0].shape[1]] + [W.shape[0] for W, _ in convs]
        return self._add(UDF_CNN, dims, [W for W, _ in convs], [b for _, b in convs], threshold, hw, hb,
                         cost_hint)

    def set_margins(self, pred: int, lowp: float, tf32: float, fp32: float):
        _check(load().hydro_set_margins(self._h, pred, float(lowp), float(tf32), float(fp32)), "hydro_set_margins")

    def set_static_order(self, order):
        arr = (ctypes.c_int32 * len(order))(*order)
        _check(load().hydro_set_static_order(self._h, arr, len(order)), "hydro_set_static_order")

    def calibrate(self, tuples) -> list:
        info = (CalibInfo * MAX_PREDICATES)()
        _check(load().hydro_calibrate(self._h, _ptr(tuples), int(tuples.shape[0]), info), "hydro_calibrate")
        return [{f: getattr(info[i], f) for f, _ in CalibInfo._fields_} for i in range(self.n_pred)]

    def udf_scores(self, pred: int, precision: str, tuples, out):
        """Scores of one predicate's UDF on device tuples into ``out`` (device float64 [n])."""
        _check(load().hydro_udf_scores(self._h, pred, PRECISIONS[precision], _ptr(tuples), int(tuples.shape[0]),
                                       _ptr(out)), "hydro_udf_scores")
        return out

    # -- batches
    def submit(self, tuples, ids=None, n: int | None = None) -> int:
        n = int(tuples.shape[0]) if n is None else n
        bid = ctypes.c_int64()
        _check(load().hydro_submit_batch(self._h, _ptr(tuples), _ptr(ids), n, ctypes.byref(bid)),
               "hydro_submit_batch")
        self._n_of[bid.value] = n
        return bid.value

    def poll(self, batch_id: int, wait_ms: int = -1):
        """(bitmap uint32 [ceil(n/32)], eval counts int64 [P], info dict) or
        raises HydroError (HYDRO_EAGAIN if not done within wait_ms)."""
        n = self._n_of.get(batch_id, 0)
        bitmap = np.zeros(max(1, (n + 31) // 32), np.uint32)
        counts = np.zeros(MAX_PREDICATES, np.int64)
        info = BatchInfo()
        _check(load().hydro_poll_result(self._h, batch_id,
                                        bitmap.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                        counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                        ctypes.byref(info), int(wait_ms)), "hydro_poll_result")
        self._n_of.pop(batch_id, None)
        P = self.n_pred
        d = dict(n=info.n, n_pass=info.n_pass, warmup=bool(info.warmup), order=list(info.order[:P]),
                 passed=list(info.passed[:P]), recheck_tf32=list(info.recheck_tf32[:P]),
                 recheck_fp32=list(info.recheck_fp32[:P]), cache_hits=list(info.cache_hits[:P]),
                 recheck_fp64=list(info.recheck_fp64[:P]), device_ms=info.device_ms,
                 stage_ns=list(info.stage_ns[:P]))
        return bitmap[:(n + 31) // 32], counts[:P], d

    def debug_trace(self, batch_id: int, n: int):
        """(order uint8 [n, P], visited uint8 [n]) of the most recent batch (learned router)."""
        order = np.zeros((max(n, 1), MAX_PREDICATES), np.uint8)
        visited = np.zeros(max(n, 1), np.uint8)
        _check(load().hydro_debug_trace(self._h, batch_id, order.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                        visited.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))), "hydro_debug_trace")
        return order[:n, :self.n_pred], visited[:n]

    def stats(self) -> list:
        out = (PredStats * MAX_PREDICATES)()
        _check(load().hydro_get_stats(self._h, out, self.n_pred), "hydro_get_stats")
        return [{f: getattr(out[i], f) for f, _ in PredStats._fields_} for i in range(self.n_pred)]

    def profile(self, enable: bool = True):
        """Start (clearing) or stop per-launch timing of the UDF layer kernels."""
        _check(load().hydro_profile(self._h, 1 if enable else 0), "hydro_profile")

    def profile_read(self):
        """({kernel class: dict(launches, total_ms, flops, bytes)}, total launches)."""
        out = (KernelProfile * 32)()
        n = ctypes.c_int32()
        tot = ctypes.c_int64()
        _check(load().hydro_profile_read(self._h, out, 32, ctypes.byref(n), ctypes.byref(tot)), "hydro_profile_read")
        d = {}
        for i in range(n.value):
            d[out[i].name.decode()] = dict(launches=out[i].launches, total_ms=out[i].total_ms, flops=out[i].flops,
                                           bytes=out[i].bytes)
        return d, tot.value

    def close(self):
        if self._h:
            h, self._h = self._h, ctypes.c_void_p()
            _check(load().hydro_destroy_query(h), "hydro_destroy_query")

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            if self._h:
                load().hydro_destroy_query(self._h)
        except Exception:
            pass


def mlp_scores_noalloc(x, weights, biases, out, stream=None):
    """FP32 MLP scores with no device allocation (see hydro.h): ``x`` device
    fp32 [n, dim]; ``weights``/``biases`` lists of device fp32 tensors
    ([out, in] / [out]); ``out`` device float64 [n].

    The C entry point takes raw pointers and cannot see shapes, dtypes or
    strides, so every tensor is checked here first (ValueError on a
    mismatch): a wrong shape or dtype would make its kernels read or write
    outside the caller's buffers."""
    import torch

    def _need(ok, what):
        if not ok:
            raise ValueError(f"mlp_scores_noalloc: {what}")

    _need(isinstance(x, torch.Tensor) and x.is_cuda and x.dim() == 2 and x.dtype == torch.float32
          and x.is_contiguous(), "x must be a contiguous 2-D float32 CUDA tensor")
    _need(len(weights) >= 1 and len(weights) == len(biases), "need one bias per weight, at least one layer")
    dev = x.device
    dims = [int(x.shape[1])] + [int(w.shape[0]) for w in weights]
    for l, (W, b) in enumerate(zip(weights, biases)):
        _need(isinstance(W, torch.Tensor) and W.device == dev and W.dtype == torch.float32 and W.is_contiguous()
              and W.dim() == 2 and tuple(W.shape) == (dims[l + 1], dims[l]),
              f"weight {l} must be a contiguous float32 tensor of shape ({dims[l + 1]}, {dims[l]}) on {dev}")
        _need(isinstance(b, torch.Tensor) and b.device == dev and b.dtype == torch.float32 and b.is_contiguous()
              and b.numel() == dims[l + 1], f"bias {l} must be a contiguous float32 tensor of {dims[l + 1]} "
              f"elements on {dev}")
    _need(dims[-1] == 1, "the last layer must have one output")
    _need(isinstance(out, torch.Tensor) and out.device == dev and out.dtype == torch.float64 and out.is_contiguous()
          and out.numel() >= int(x.shape[0]), f"out must be a contiguous float64 tensor of >= {x.shape[0]} "
          f"elements on {dev}")
    d = (ctypes.c_int32 * len(dims))(*dims)
    wp = (ctypes.c_void_p * len(weights))(*[w.data_ptr() for w in weights])
    bp = (ctypes.c_void_p * len(biases))(*[b.data_ptr() for b in biases])
    s = stream.cuda_stream if stream is not None else None
    _check(load().hydro_mlp_scores_noalloc(x.data_ptr(), int(x.shape[0]), len(weights), d, wp, bp, out.data_ptr(), s),
           "hydro_mlp_scores_noalloc")
    return out


def bits_from_words(words: np.ndarray, n: int) -> np.ndarray:
    """Unpack an LSB-first bitmap into n bools."""
    w = np.asarray(words, np.uint32)
    j = np.arange(n)
    return ((w[j >> 5] >> (j & 31).astype(np.uint32)) & 1).astype(bool)





class Session:
    """Many concurrent queries over one pool of MLP UDFs (``hydro_session_*``).

    Each step stacks every query's next chunk of fp32 rows; ``submit`` takes
    the stacked device tensor and the per-query counts, ``poll`` returns the
    pass bitmap words, a per-query report and the step's GPU time."""

    def __init__(self, *, dim: int, max_step_tuples: int, precision: str = "fp32", warmup: int = 1,
                 window: int = 8, graphs: bool = True, autotune: bool = True, max_in_flight: int = 2,
                 device: int = 0, stream=None, learned: bool = False, proxy_hidden: int = 64,
                 proxy_refresh: int = 16, proxy_epochs: int = 1, proxy_lr: float = 1e-3, proxy_seed: int = 1,
                 batches_per_step: int = 1, lag: int = 0, fp8_min_width: int = 0, proxy_rows: int = 0,
                 policy: str = "rank", tile_sched: str | None = None):
        L = load()
        cfg = SessionConfig()
        L.hydro_session_default_config(ctypes.byref(cfg))
        cfg.dim = dim
        cfg.max_step_tuples = max_step_tuples
        cfg.precision = PRECISIONS[precision]
        cfg.warmup_batches = warmup
        cfg.stats_window = window
        cfg.use_graphs = 1 if graphs else 0
        cfg.autotune = 1 if autotune else 0
        cfg.max_in_flight = max_in_flight
        cfg.device = device
        cfg.stream = stream.cuda_stream if stream is not None else None
        cfg.learned = 1 if learned else 0
        cfg.proxy_hidden = proxy_hidden
        cfg.proxy_refresh = proxy_refresh
        cfg.proxy_epochs = proxy_epochs
        cfg.proxy_lr = proxy_lr
        cfg.proxy_seed = proxy_seed
        cfg.batches_per_step = batches_per_step
        cfg.route_lag = lag
        cfg.fp8_min_width = fp8_min_width
        cfg.proxy_rows = proxy_rows
        cfg.policy = POLICIES[policy]
        if tile_sched is not None:
            cfg.tile_sched = {"static": 0, "data_aware": 1}[tile_sched]
        self.tile_sched = {0: "static", 1: "data_aware"}[cfg.tile_sched]
        self.K = batches_per_step
        self._h = ctypes.c_void_p()
        _check(L.hydro_session_create(ctypes.byref(cfg), ctypes.byref(self._h)), "hydro_session_create")
        self.n_udf = 0
        self.queries = []

    def add_udf(self, layers) -> int:
        """Pool MLP from [(W [out, in], b [out]), ...]; returns its id."""
        FP = ctypes.POINTER(ctypes.c_float)
        Ws = [np.ascontiguousarray(w, np.float32) for w, _ in layers]
        bs = [np.ascontiguousarray(b, np.float32) for _, b in layers]
        dims = [Ws[0].shape[1]] + [w.shape[0] for w in Ws]
        d = (ctypes.c_int32 * len(dims))(*dims)
        desc = UdfDesc()
        desc.kind = UDF_MLP
        desc.n_layers = len(Ws)
        desc.dims = d
        desc.weights = (FP * len(Ws))(*[w.ctypes.data_as(FP) for w in Ws])
        desc.biases = (FP * len(bs))(*[b.ctypes.data_as(FP) for b in bs])
        out = ctypes.c_int32()
        _check(load().hydro_session_add_udf(self._h, ctypes.byref(desc), ctypes.byref(out)), "hydro_session_add_udf")
        self.n_udf += 1
        return out.value

    def add_query(self, udfs, thresholds) -> int:
        n = len(udfs)
        u = (ctypes.c_int32 * n)(*udfs)
        t = (ctypes.c_double * n)(*thresholds)
        out = ctypes.c_int32()
        _check(load().hydro_session_add_query(self._h, n, u, t, ctypes.byref(out)), "hydro_session_add_query")
        self.queries.append(list(udfs))
        return out.value

    def set_margins(self, udf: int, lowp: float, split: float, fp32: float):
        _check(load().hydro_session_set_margins(self._h, udf, lowp, split, fp32), "hydro_session_set_margins")

    def calibrate(self, tuples) -> list:
        info = (CalibInfo * MAX_POOL)()
        _check(load().hydro_session_calibrate(self._h, _ptr(tuples), int(tuples.shape[0]), info),
               "hydro_session_calibrate")
        return [{f: getattr(info[i], f) for f, _ in CalibInfo._fields_} for i in range(self.n_udf)]

    def udf_scores(self, udf: int, precision: str, tuples, out):
        _check(load().hydro_session_udf_scores(self._h, udf, PRECISIONS[precision], _ptr(tuples),
                                               int(tuples.shape[0]), _ptr(out)), "hydro_session_udf_scores")

    def submit(self, tuples, counts) -> int:
        """counts: per query (K = 1) or per (query, batch) q*K + k."""
        Q = len(self.queries) * self.K
        c = (ctypes.c_int32 * Q)(*[int(v) for v in counts])
        sid = ctypes.c_int64()
        _check(load().hydro_session_submit(self._h, _ptr(tuples), c, ctypes.byref(sid)), "hydro_session_submit")
        self._last_total = int(sum(int(v) for v in counts))
        return sid.value

    def poll(self, step: int, total: int | None = None, wait_ms: int = -1):
        """(bitmap words uint32, [per (query, batch) dict], device_ms)."""
        Q = len(self.queries) * self.K
        total = self._last_total if total is None else total
        words = np.zeros(max(1, (total + 31) // 32), np.uint32)
        per = (StepQuery * max(Q, 1))()
        ms = ctypes.c_double()
        _check(load().hydro_session_poll(self._h, step, words.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), per,
                                         ctypes.byref(ms), wait_ms), "hydro_session_poll")
        out = []
        for q in range(Q):
            r = per[q]
            P = len(self.queries[q // self.K])
            out.append(dict(n=r.n, n_pass=r.n_pass, batch=r.batch, warmup=bool(r.warmup), order=list(r.order[:P]),
                            evaluated=list(r.evaluated[:P]), passed=list(r.passed[:P]),
                            recheck_split=list(r.recheck_split[:P]), recheck_fp32=list(r.recheck_fp32[:P]), recheck_fp64=list(r.recheck_fp64[:P])))
        return words, out, ms.value

    def profile(self, enable: bool = True):
        _check(load().hydro_session_profile(self._h, 1 if enable else 0), "hydro_session_profile")

    def profile_read(self):
        """({kernel class: dict(launches, total_ms)}, total launches)."""
        out = (KernelProfile * 16)()
        n = ctypes.c_int32()
        tot = ctypes.c_int64()
        _check(load().hydro_session_profile_read(self._h, out, 16, ctypes.byref(n), ctypes.byref(tot)),
               "hydro_session_profile_read")
        return {out[i].name.decode(): dict(launches=out[i].launches, total_ms=out[i].total_ms)
                for i in range(n.value)}, tot.value

    def balance(self, enable: bool | None = None):
        """Load balance of the grouped tensor-core launches of the steps polled
        since ``balance(True)``: launches, summed makespan / mean / max CTA busy
        ms and per-CTA busy ms.  ``enable`` True (re)starts, False stops, None
        only reads."""
        out = BalanceInfo()
        en = -1 if enable is None else (1 if enable else 0)
        _check(load().hydro_session_balance(self._h, en, ctypes.byref(out)), "hydro_session_balance")
        n = max(1, out.ctas)
        return dict(launches=out.launches, ctas=out.ctas, makespan_ms=out.makespan_ms,
                    busy_mean_ms=out.busy_mean_ms, busy_max_ms=out.busy_max_ms,
                    cta_busy_ms=[out.cta_busy_ms[i] for i in range(n)])

    def debug_trace(self, step: int, total: int):
        """(order uint8 [total, 8], visited uint8 [total]) of a polled step."""
        order = np.zeros((max(total, 1), 8), np.uint8)
        visited = np.zeros(max(total, 1), np.uint8)
        _check(load().hydro_session_debug_trace(self._h, step, order.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                                visited.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))),
               "hydro_session_debug_trace")
        return order[:total], visited[:total]

    def tuning(self) -> list:
        out = (TileChoice * 64)()
        n = ctypes.c_int32()
        _check(load().hydro_session_tuning(self._h, out, 64, ctypes.byref(n)), "hydro_session_tuning")
        return [dict(udf=o.udf, layer=o.layer, K=o.K, N=o.N, tile_n=o.tile_n, us=list(o.us)) for o in out[:n.value]]

    def close(self):
        if self._h:
            h, self._h = self._h, ctypes.c_void_p()
            _check(load().hydro_session_destroy(h), "hydro_session_destroy")

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
