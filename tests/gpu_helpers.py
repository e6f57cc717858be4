"""Shared helpers of the GPU parity tests: drive a query through the Python
binding of the C ABI and compare with the oracle."""
import json
import os

import numpy as np

import datagen as D
import oracle as O

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def stored_thresholds(name):
    with open(os.path.join(GOLDEN, f"{name}_thresholds.json")) as f:
        return json.load(f)["thresholds"]


def stored_pass_matrix(name, q=None):
    """The oracle's [n, P] pass matrix of a whole benchmarked stream (bool),
    written by ``tests/golden/make_full_oracle.py``; ``q`` selects one query
    of the many-query workload."""
    z = np.load(os.path.join(GOLDEN, f"{name}_oracle.npz"))
    key, kn, kp = ("pm", "n", "P") if q is None else (f"pm_{q}", f"n_{q}", f"P_{q}")
    n, P = int(z[kn]), int(z[kp])
    return np.unpackbits(z[key], bitorder="little")[:n * P].reshape(n, P).astype(bool)


def prefix_visits(pm, order):
    """Per tuple, the bit set of predicates a per-tuple order evaluates: its
    order up to and including the first failing predicate (all of them if
    the tuple passes).  ``order`` is [n, >=P] uint8."""
    n, P = pm.shape
    want = np.zeros(n, np.uint16)
    alive = np.ones(n, bool)
    rows = np.arange(n)
    for k in range(P):
        i = order[:, k].astype(np.int64)
        want[alive] |= (np.uint16(1) << i[alive].astype(np.uint16))
        alive &= pm[rows, i]
    return want


def oracle_thresholds(w):
    S = O.udf_scores(w.kind, D.calib_tuples(w), D.predicate_weights(w))
    return [O.threshold_for_selectivity(S[:, i], s) for i, s in enumerate(w.selectivity)], S


def model_costs(w):
    if w.kind == "vec":
        return [O.mlp_flops(d) for d in w.udfs]
    C, H, W = w.frame
    return [O.cnn_flops(c, H, W) for c in w.udfs]


def make_query(w, thresholds, *, batch, policy="rank", precision="fp32", warmup=1, window=8, lag=1,
               static_order=None, max_in_flight=4, preds=None, reuse=False, id_capacity=None, cost="model",
               lanes=1, split="bf16x3", recheck_graphs=True):
    """A query over the workload's predicates.  With ``reuse`` the predicates
    listed in ``extra['emb_preds']`` run as heads on one shared, cached
    embedding (query.emb_id)."""
    import paper_2403_14902_b300 as H
    q = H.Query(w.kind, dim=w.dim, frame=w.frame, max_batch=batch, policy=policy, precision=precision,
                warmup=warmup, window=window, lag=lag, max_in_flight=max_in_flight, cost=cost, lanes=lanes,
                split=split, recheck_graphs=recheck_graphs)
    weights = D.predicate_weights(w)
    idx = list(range(len(weights))) if preds is None else list(preds)
    shared = set(w.extra.get("emb_preds", ())) if (reuse and w.extra) else set()
    q.emb_id = q.add_embedding(D.embedding_weights(w), id_capacity or w.n) if shared else 0
    for i in idx:
        if w.kind == "vec" and i in shared:
            q.add_mlp(D.head_weights(w, i), thresholds[i], upstream=q.emb_id)
        elif w.kind == "vec":
            q.add_mlp(weights[i], thresholds[i])
        else:
            q.add_cnn(weights[i], thresholds[i])
    if static_order is not None:
        q.set_static_order(static_order)
    return q


def run_stream(q, X, batch, max_in_flight=4, ids=None):
    """Submit X (device tensor) in consecutive batches (with device int64
    ``ids`` when given); return per-batch (bits bool [n_b], counts int64 [P],
    info dict) in submission order."""
    import paper_2403_14902_b300 as H
    n = X.shape[0]
    out = {}
    pending = []
    sizes = {}
    for b0 in range(0, max(n, 1), batch):
        xb = X[b0:b0 + batch]
        bid = q.submit(xb, None if ids is None else ids[b0:b0 + batch])
        sizes[bid] = xb.shape[0]
        pending.append(bid)
        if len(pending) >= max_in_flight:
            b = pending.pop(0)
            words, counts, info = q.poll(b)
            out[b] = (H.bits_from_words(words, sizes[b]), counts, info)
    for b in pending:
        words, counts, info = q.poll(b)
        out[b] = (H.bits_from_words(words, sizes[b]), counts, info)
    return [out[k] for k in sorted(out)]


def check_against_oracle(res, pm, batch, *, policy, costs, warmup=1, window=8, lag=1, static_order=None,
                         **reuse):
    """Bit-exact result and exact per-batch order/counts (and reuse-cache
    hits when ``reuse`` describes the groups) versus the oracle's router
    simulation."""
    sim = O.simulate(pm, batch, policy=policy, costs=costs, static_order=static_order, warmup=warmup,
                     window=window, lag=lag, **reuse)
    assert len(sim) == len(res)
    for b, ((bits, counts, info), s) in enumerate(zip(res, sim)):
        assert np.array_equal(bits, s["bits"]), f"batch {b}: pass set differs"
        assert info["order"] == s["order"], f"batch {b}: order {info['order']} vs {s['order']}"
        assert counts.tolist() == s["counts"].tolist(), f"batch {b}: counts {counts} vs {s['counts']}"
        assert info["passed"] == s["passed"].tolist(), f"batch {b}: passed"
        assert info["warmup"] == s["warmup"] or policy == "all"
        assert info["n_pass"] == int(s["bits"].sum())
        if reuse:
            assert info["cache_hits"] == s["hits"].tolist(), f"batch {b}: hits {info['cache_hits']} vs {s['hits']}"
    return sim


def score_tolerance_ok(s_gpu, s64, rms, rel=1e-3):
    """|s - s64| <= rel * max(|s64|, rms): relative error with the
    calibration RMS as the scale near zero."""
    bound = rel * np.maximum(np.abs(s64), rms)
    return np.abs(s_gpu - s64) <= bound
