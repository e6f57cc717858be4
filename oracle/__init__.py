"""Oracle for the adaptive predicate path: plain, slow, FP64, CPU only.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path (``paper_2403_14902_b300``) and never imports it.

What it computes:

* ``udf_scores``: every UDF on every tuple in FP64 (``oracle.c``: direct
  loops over the layer definitions).
* ``pass_matrix``: ``score > threshold`` per (tuple, predicate); a tuple is in
  the result iff it passes every predicate (the conjunction of Listing 1 /
  Sec. 1).
* ``simulate``: the adaptive Eddy router written out per batch (Sec. 3.2
  "Data Flow and Routing", Sec. 3.3, Sec. 4.1 "Cost-Driven Routing Policy"
  and "Warmup Phase"): which order each batch takes and how many tuples
  each predicate evaluates when failing tuples are dropped at once (Sec. 3.3
  "Eager Materialization").
* ``rank_key`` / ``expected_cost``: the rank cost/(1 - selectivity) of
  Sec. 4.1 (after Hellerstein) and the per-tuple expected cost of an order.

Readings where the paper is silent (each is also listed in the design notes):
selectivity is smoothed as (passed+1)/(evaluated+2) over a window of the last
W visible batches; a batch is routed on statistics of batches that finished
at least ``lag`` batches earlier; the model cost is the UDF's flops per tuple;
ties go to the lower predicate id; the test is strict (score > threshold).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from fractions import Fraction
from itertools import permutations

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` (gcc, -O3, pthreads)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        cmd = ["gcc", "-O3", "-march=x86-64-v3", "-fPIC", "-shared", "-o", _SO, src, "-lpthread", "-lm"]
        subprocess.run(cmd, check=True)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        fp = ctypes.POINTER(ctypes.c_float)
        L.oracle_mlp_scores.argtypes = [fp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(fp),
                                        ctypes.POINTER(fp), ctypes.POINTER(ctypes.c_double), ctypes.c_int]
        L.oracle_mlp_scores.restype = ctypes.c_int
        L.oracle_cnn_scores.argtypes = [ctypes.POINTER(ctypes.c_uint8), ctypes.c_int64, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(fp),
                                        ctypes.POINTER(fp), fp, ctypes.c_double,
                                        ctypes.POINTER(ctypes.c_double), ctypes.c_int]
        L.oracle_cnn_scores.restype = ctypes.c_int
        L.oracle_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def threads() -> int:
    return lib().oracle_threads()


def _fptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


# ------------------------------------------------------------------ scores

def mlp_scores(X: np.ndarray, layers, n_threads: int = 0) -> np.ndarray:
    """FP64 scores of an MLP UDF ``layers = [(W [out,in] fp32, b [out] fp32)]``
    on rows of ``X`` (fp32 [n, in])."""
    X = np.ascontiguousarray(X, np.float32)
    n = X.shape[0]
    dims = [layers[0][0].shape[1]] + [W.shape[0] for W, _ in layers]
    Ws = [np.ascontiguousarray(W, np.float32) for W, _ in layers]
    bs = [np.ascontiguousarray(b, np.float32) for _, b in layers]
    FP = ctypes.POINTER(ctypes.c_float)
    Wp = (FP * len(Ws))(*[_fptr(W) for W in Ws])
    bp = (FP * len(bs))(*[_fptr(b) for b in bs])
    d = np.asarray(dims, np.int32)
    out = np.empty(n, np.float64)
    rc = lib().oracle_mlp_scores(_fptr(X), n, X.shape[1], len(layers),
                                 d.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), Wp, bp,
                                 out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n_threads)
    if rc != 0:
        raise RuntimeError("oracle_mlp_scores failed")
    return out


def cnn_scores(frames: np.ndarray, udf, n_threads: int = 0) -> np.ndarray:
    """FP64 scores of a CNN UDF ``udf = (convs, (head_w, head_b))`` on uint8
    frames [n, C, H, W]."""
    frames = np.ascontiguousarray(frames, np.uint8)
    n, C, H, W = frames.shape
    convs, (hw, hb) = udf
    ch = [convs[0][0].shape[1]] + [Wc.shape[0] for Wc, _ in convs]
    Ws = [np.ascontiguousarray(Wc, np.float32) for Wc, _ in convs]
    bs = [np.ascontiguousarray(b, np.float32) for _, b in convs]
    hw = np.ascontiguousarray(hw, np.float32)
    FP = ctypes.POINTER(ctypes.c_float)
    Wp = (FP * len(Ws))(*[_fptr(x) for x in Ws])
    bp = (FP * len(bs))(*[_fptr(x) for x in bs])
    d = np.asarray(ch, np.int32)
    out = np.empty(n, np.float64)
    rc = lib().oracle_cnn_scores(frames.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), n, C, H, W,
                                 len(convs), d.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                 Wp, bp, _fptr(hw), float(hb),
                                 out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n_threads)
    if rc != 0:
        raise RuntimeError("oracle_cnn_scores failed")
    return out


def udf_scores(kind: str, tuples: np.ndarray, udfs, n_threads: int = 0) -> np.ndarray:
    """[n, P] FP64 scores of every predicate's UDF on every tuple."""
    f = mlp_scores if kind == "vec" else cnn_scores
    if len(udfs) == 0:
        return np.zeros((tuples.shape[0], 0))
    return np.stack([f(tuples, u, n_threads) for u in udfs], axis=1)


# ------------------------------------------------------------- thresholds

def threshold_for_selectivity(calib_scores: np.ndarray, s: float) -> float:
    """Threshold with exactly round(s*n) calibration scores strictly above it:
    the midpoint between the k-th and (k+1)-th largest calibration scores."""
    d = np.sort(np.asarray(calib_scores, np.float64))[::-1]
    n = d.size
    k = int(round(s * n))
    if k <= 0:
        return float(d[0]) + 1.0
    if k >= n:
        return float(d[-1]) - 1.0
    return float((d[k - 1] + d[k]) / 2.0)


def pass_matrix(scores: np.ndarray, thresholds) -> np.ndarray:
    """bool [n, P]: score > threshold (strict)."""
    t = np.asarray(thresholds, np.float64)[None, :]
    return np.asarray(scores, np.float64) > t


def result_bits(pm: np.ndarray) -> np.ndarray:
    """bool [n]: the conjunction over predicates."""
    return pm.all(axis=1) if pm.shape[1] else np.ones(pm.shape[0], bool)


def bitmap_words(bits: np.ndarray) -> np.ndarray:
    """Pack bools LSB-first: tuple j -> word j // 32, bit j % 32 (uint32)."""
    bits = np.asarray(bits, bool)
    n = bits.size
    words = np.zeros((n + 31) // 32, np.uint32)
    for j in np.flatnonzero(bits):
        words[j >> 5] |= np.uint32(1) << np.uint32(j & 31)
    return words


# ------------------------------------------------------------- cost model

def mlp_flops(dims) -> int:
    """2 x multiply-adds per tuple of an MLP with widths ``dims``."""
    return sum(2 * dims[l] * dims[l + 1] for l in range(len(dims) - 1))


def cnn_flops(chans, H: int = 64, W: int = 64) -> int:
    """2 x multiply-adds per frame: 3x3 convs at H x W plus the linear head."""
    conv = sum(2 * H * W * 9 * chans[l] * chans[l + 1] for l in range(len(chans) - 1))
    return conv + 2 * chans[-1]


# ------------------------------------------------------------- rank logic

def smoothed_selectivity(evaluated: int, passed: int) -> Fraction:
    return Fraction(passed + 1, evaluated + 2)


def rank_key(cost, evaluated: int, passed: int) -> Fraction:
    """cost / (1 - s) with s = (passed+1)/(evaluated+2) (Sec. 4.1)."""
    s = smoothed_selectivity(evaluated, passed)
    return Fraction(cost) / (1 - s)


def order_by(keys) -> list:
    """Ascending by key, ties to the lower predicate id."""
    return sorted(range(len(keys)), key=lambda i: (keys[i], i))


def expected_cost(order, costs, sel) -> float:
    """Per-tuple expected cost sum_k c_{pi_k} prod_{j<k} s_{pi_j} of evaluating
    the conjunction in ``order`` when predicates are independent."""
    total, survive = 0.0, 1.0
    for i in order:
        total += costs[i] * survive
        survive *= sel[i]
    return total


def best_order_bruteforce(costs, sel):
    """(order, cost) minimising ``expected_cost`` over all P! orders."""
    best = None
    for p in permutations(range(len(costs))):
        c = expected_cost(p, costs, sel)
        if best is None or c < best[1] - 1e-15 * max(1.0, abs(best[1])):
            best = (list(p), c)
    return best


def static_counts(pm: np.ndarray, order) -> np.ndarray:
    """Evaluation counts of a fixed order with eager dropping: predicate
    order[k] sees the tuples that passed order[0..k-1]."""
    P = pm.shape[1]
    counts = np.zeros(P, np.int64)
    alive = np.ones(pm.shape[0], bool)
    for i in order:
        counts[i] = int(alive.sum())
        alive &= pm[:, i]
    return counts


# ------------------------------------------------------------- simulation

POLICIES = ("rank", "static", "all", "cost", "selectivity")


def simulate(pm: np.ndarray, batch: int, policy: str = "rank", costs=None, static_order=None,
             warmup: int = 1, window: int = 8, lag: int = 1, groups=None, group_costs=None, ids=None,
             prefilled=None):
    """Route a stream through the conjunction batch by batch.

    ``pm`` is the [n, P] pass matrix of the stream in submission order; the
    stream is cut into consecutive batches of ``batch`` tuples.  Returns a
    list of dicts per batch: ``order``, ``counts`` [P] (tuples each predicate
    evaluated), ``passed`` [P] (of those, how many passed), ``warmup`` flag,
    ``bits`` (the batch's result) and ``hits`` [P] (reuse-cache hits).

    Reuse (Sec. 4.3 "Reuse-aware Routing"): ``groups[i]`` names the shared
    upstream UDF of predicate i (or None).  Its output is cached per tuple id
    (``ids`` [n], ``prefilled`` ids cached before the query).  A predicate of
    a group runs the group UDF only on alive tuples whose id is not cached
    yet, then caches them.  The router's cost of such a predicate for batch b
    is ``costs[i] + miss_b / n_b * group_costs[g]`` (the estimated cost of
    the reuse-aware formula, with the hit rate of the batch), where miss_b
    counts the batch's ids not cached by batches finished lag+1 earlier (or
    prefilled); ``costs[i]`` is then the head's own cost.  That surcharge
    applies only while no head of the same group precedes it in the batch's
    order: a later head finds every tuple that reaches it cached by the
    earlier head.  So the order is built position by position, each time the
    remaining predicate with the lowest key given the groups already
    computed (ties to the lower id); without groups this is the ascending
    key order."""
    assert policy in POLICIES
    n, P = pm.shape
    costs = [1] * P if costs is None else list(costs)
    groups = [None] * P if groups is None else list(groups)
    declared = list(range(P))
    gnames = sorted({g for g in groups if g is not None})
    # cache tags per group: 0 absent, -1 prefilled, b+1 computed in batch b
    tag = {}
    if gnames:
        ids = np.arange(n, dtype=np.int64) if ids is None else np.asarray(ids, np.int64)
        cap = int(ids.max()) + 1 if n else 1
        if prefilled is not None and len(prefilled):
            cap = max(cap, int(np.max(prefilled)) + 1)
        for g in gnames:
            tag[g] = np.zeros(cap, np.int64)
            if prefilled is not None:
                tag[g][np.asarray(prefilled, np.int64)] = -1
    stat_e, stat_p = [], []
    out = []
    nb = (n + batch - 1) // batch
    for b in range(nb):
        rows = pm[b * batch:(b + 1) * batch]
        bids = ids[b * batch:(b + 1) * batch] if gnames else None
        nbt = rows.shape[0]
        evaluate_all = policy == "all" or (policy in ("rank", "cost", "selectivity") and b < warmup)
        if evaluate_all:
            order = declared
        elif policy == "static":
            order = list(static_order) if static_order is not None else declared
        else:
            last = b - 1 - lag
            if last < 0:
                order = declared
            else:
                lo = max(0, last - window + 1)
                miss = {}
                for g in gnames:
                    t = tag[g][bids]
                    visible = (t == -1) | ((t > 0) & (t - 1 <= last))
                    miss[g] = int((~visible).sum())
                stats = []
                for i in range(P):
                    E = sum(stat_e[x][i] for x in range(lo, last + 1))
                    Pp = sum(stat_p[x][i] for x in range(lo, last + 1))
                    if E == 0:
                        E = sum(stat_e[x][i] for x in range(min(warmup, last + 1)))
                        Pp = sum(stat_p[x][i] for x in range(min(warmup, last + 1)))
                    stats.append((E, Pp))

                def key(i, computed):
                    # a head pays its group's cost for the batch's misses only while no
                    # head of the group is placed before it: every tuple reaching a
                    # later head was cached by the earlier one
                    c = Fraction(costs[i])
                    g = groups[i]
                    if g is not None and g not in computed and nbt > 0:
                        c += Fraction(miss[g], nbt) * group_costs[g]
                    E, Pp = stats[i]
                    if policy == "rank":
                        return c / (1 - smoothed_selectivity(E, Pp))
                    if policy == "cost":
                        return c
                    return smoothed_selectivity(E, Pp)
                # position by position, the remaining predicate with the lowest key under
                # the groups computed so far (ties to the lower id)
                order, computed, rest = [], set(), list(range(P))
                while rest:
                    pick = min(rest, key=lambda i: (key(i, computed), i))
                    order.append(pick)
                    rest.remove(pick)
                    if groups[pick] is not None:
                        computed.add(groups[pick])
        counts = np.zeros(P, np.int64)
        passed = np.zeros(P, np.int64)
        hits = np.zeros(P, np.int64)
        alive = np.ones(nbt, bool)
        for i in order:
            ev = np.ones(nbt, bool) if evaluate_all else alive
            counts[i] = int(ev.sum())
            passed[i] = int((ev & rows[:, i]).sum())
            g = groups[i]
            if g is not None:
                idx = bids[ev]
                absent = tag[g][idx] == 0
                hits[i] = int((~absent).sum())
                tag[g][idx[absent]] = b + 1
            if not evaluate_all:
                alive &= rows[:, i]
        stat_e.append([int(v) for v in counts])
        stat_p.append([int(v) for v in passed])
        out.append(dict(order=list(order), counts=counts, passed=passed, warmup=evaluate_all,
                        bits=result_bits(rows), hits=hits))
    return out


# ------------------------------------------------------------- concurrent model

def concurrent_makespan(order, costs, sel, n: int, passes=None) -> float:
    """Makespan of a conjunction whose predicates run concurrently, each on its
    own resource (Sec. 4.1 "Example comparison": one predicate on the GPU, the
    other on the CPU): tuples flow through the predicates in ``order``, each
    resource serves its queue first-come first-served, a tuple that fails is
    dropped.  ``passes[k][j]`` says whether tuple j passes the k-th predicate
    of the order (default: tuple j passes predicate i iff
    floor((j+1) s_i) > floor(j s_i), an even spread of round(n s_i) passes)."""
    P = len(order)
    if passes is None:
        passes = [[int((j + 1) * sel[i]) > int(j * sel[i]) for j in range(n)] for i in order]
    ready = [0.0] * n                  # when tuple j is available for the next stage
    alive = [True] * n
    end = 0.0
    for k, i in enumerate(order):
        free = 0.0                     # the resource of predicate i
        for j in sorted(range(n), key=lambda j: (ready[j], j)):
            if not alive[j]:
                continue
            start = max(free, ready[j])
            free = start + costs[i]
            ready[j] = free
            end = max(end, free)
            alive[j] = alive[j] and passes[k][j]
    return end


def fluid_makespan(order, costs, sel, n: int) -> float:
    """Large-n limit of ``concurrent_makespan``: the slowest resource bounds
    the makespan, n * max_k c_{pi_k} * prod_{j<k} s_{pi_j}."""
    surv, worst = float(n), 0.0
    for i in order:
        worst = max(worst, surv * costs[i])
        surv *= sel[i]
    return worst
