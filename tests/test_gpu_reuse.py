"""GPU parity of reuse-aware routing with a cached shared embedding on the
drifting stream (512-d fp32 tuples; two predicates are heads on one
embedding 512-1024-256 whose outputs are cached per tuple id)."""
import numpy as np
import pytest

import datagen as D
import oracle as O
from gpu_helpers import (check_against_oracle, make_query, oracle_thresholds, run_stream, stored_pass_matrix,
                         stored_thresholds)

pytestmark = pytest.mark.gpu

N = 8 * 4096


def _costs(w):
    emb = w.extra["embedding"]
    heads = {i: w.udfs[i][len(emb) - 1:] for i in w.extra["emb_preds"]}
    costs = [O.mlp_flops(heads[i]) if i in heads else O.mlp_flops(d) for i, d in enumerate(w.udfs)]
    groups = ["E" if i in heads else None for i in range(len(w.udfs))]
    return costs, groups, {"E": O.mlp_flops(emb)}


@pytest.fixture(scope="module")
def drift():
    import torch
    w = D.workload("drift5", n=N, extra=dict(D.WORKLOADS["drift5"].extra, segment_len=4096))
    th, _ = oracle_thresholds(w)
    X = D.stream_tuples(w)
    S = O.udf_scores("vec", X, D.predicate_weights(w))
    ids = np.arange(N, dtype=np.int64)
    return dict(w=w, th=th, X=X, pm=O.pass_matrix(S, th), Xd=torch.from_numpy(X).cuda(),
                ids=torch.from_numpy(ids).cuda())


@pytest.mark.parametrize("policy", ["rank", "static", "all", "cost"])
@pytest.mark.parametrize("prefill", [False, True])
def test_reuse_parity(drift, policy, prefill):
    w = drift["w"]
    costs, groups, gcost = _costs(w)
    q = make_query(w, drift["th"], batch=4096, policy=policy, reuse=True, id_capacity=N)
    pre = np.arange(2 * 4096, 4 * 4096) if prefill else np.zeros(0, np.int64)
    if prefill:
        q.cache_prefill(q.emb_id, drift["Xd"][pre[0]:pre[-1] + 1], drift["ids"][pre[0]:pre[-1] + 1])
    res = run_stream(q, drift["Xd"], 4096, ids=drift["ids"])
    check_against_oracle(res, drift["pm"], 4096, policy=policy, costs=costs, groups=groups, group_costs=gcost,
                         ids=np.arange(N), prefilled=pre)
    q.close()


@pytest.mark.parametrize("policy", ["rank", "cost"])
def test_reuse_parity_two_lanes(drift, policy):
    """Two stream lanes (route lag 1) with the cached embedding and part of
    the stream prefilled: each lane probes the cache into its own miss list;
    every batch's order, counts and cache hits and the pass set are the
    oracle's."""
    w = drift["w"]
    costs, groups, gcost = _costs(w)
    q = make_query(w, drift["th"], batch=4096, policy=policy, reuse=True, id_capacity=N, lanes=2, lag=1)
    pre = np.arange(2 * 4096, 4 * 4096)
    q.cache_prefill(q.emb_id, drift["Xd"][pre[0]:pre[-1] + 1], drift["ids"][pre[0]:pre[-1] + 1])
    res = run_stream(q, drift["Xd"], 4096, ids=drift["ids"])
    check_against_oracle(res, drift["pm"], 4096, policy=policy, costs=costs, groups=groups, group_costs=gcost,
                         ids=np.arange(N), prefilled=pre, lag=1)
    q.close()


def test_reuse_changes_order_not_result(drift):
    # prefilling the embedding for part of the stream makes its heads cheap
    # there; the router must pick a different order for those batches while
    # the pass set stays the same
    w = drift["w"]
    costs, groups, gcost = _costs(w)
    pre = np.arange(2 * 4096, 6 * 4096)
    a = O.simulate(drift["pm"], 4096, policy="rank", costs=costs, groups=groups, group_costs=gcost,
                   ids=np.arange(N), prefilled=np.zeros(0, np.int64))
    b = O.simulate(drift["pm"], 4096, policy="rank", costs=costs, groups=groups, group_costs=gcost,
                   ids=np.arange(N), prefilled=pre)
    assert any(x["order"] != y["order"] for x, y in zip(a, b))
    q = make_query(w, drift["th"], batch=4096, policy="rank", reuse=True, id_capacity=N)
    q.cache_prefill(q.emb_id, drift["Xd"][pre[0]:pre[-1] + 1], drift["ids"][pre[0]:pre[-1] + 1])
    res = run_stream(q, drift["Xd"], 4096, ids=drift["ids"])
    assert [r[2]["order"] for r in res] == [x["order"] for x in b]
    assert all(np.array_equal(r[0], x["bits"]) for r, x in zip(res, a))
    q.close()


def test_full_drift_stream_exact():
    """1,048,576 tuples in batches of 4,096 with the cached embedding, in the
    bench's configuration (route lag 3, four stream lanes): every tuple's
    result, and every batch's order,
    evaluation counts, pass counts and cache hits, equal the oracle's (its
    stored FP64 pass matrix of the whole stream and its router and cache
    simulation)."""
    import torch
    w = D.workload("drift5")
    th = stored_thresholds("drift5")
    pm = stored_pass_matrix("drift5")
    X = D.stream_tuples(w)
    Xd = torch.from_numpy(X).cuda()
    ids = torch.arange(w.n, dtype=torch.int64, device="cuda")
    q = make_query(w, th, batch=w.batch, policy="rank", reuse=True, max_in_flight=8, lag=3, lanes=4)
    res = run_stream(q, Xd, w.batch, max_in_flight=8, ids=ids)
    costs, groups, gcost = _costs(w)
    sim = check_against_oracle(res, pm, w.batch, policy="rank", costs=costs, groups=groups, group_costs=gcost,
                               ids=np.arange(w.n), lag=3)
    assert len({tuple(x["order"]) for x in sim}) > 1, "the drifting stream should make the router change its order"
    q.close()
