"""GPU parity of the pipeline mode: every position of a batch's order runs on
a stream of its own with a share of the SMs, so that predicates work as
concurrent workers on separate resources (Sec. 4.1 "Cost-Driven Routing
Policy", "Example comparison").  The pass set, orders and counts must equal
the oracle's simulation of the same routing rule whatever runs concurrently."""
import pytest

import datagen as D
import oracle as O
from gpu_helpers import check_against_oracle, model_costs, run_stream, stored_thresholds

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def uc1():
    import json
    import os

    import torch
    w = D.workload("uc1", n=16 * 512)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "uc1_thresholds.json")) as f:
        G = json.load(f)
    X = D.stream_tuples(w)
    S = O.udf_scores("vec", X, D.predicate_weights(w))
    return dict(w=w, G=G, X=X, S=S, Xd=torch.from_numpy(X).cuda())


def _query(uc1, sa, sb, *, policy, lanes, lag, precision="fp32", pipeline=True):
    import paper_2403_14902_b300 as H
    w = uc1["w"]
    q = H.Query("vec", dim=w.dim, max_batch=512, policy=policy, precision=precision, lanes=lanes, lag=lag,
                max_in_flight=8, pipeline=pipeline)
    L = D.predicate_weights(w)
    th = [uc1["G"]["A"][f"{sa:.1f}"], uc1["G"]["B"][f"{sb:.1f}"]]
    q.add_mlp(L[0], th[0])
    q.add_mlp(L[1], th[1])
    return q, O.pass_matrix(uc1["S"], th)


@pytest.mark.parametrize("policy", ["cost", "rank", "selectivity", "static", "all"])
@pytest.mark.parametrize("lanes,lag,pipeline", [(2, 1, "shares"), (4, 3, "shares"), (2, 1, "partitions"),
                                                (4, 3, "partitions")])
def test_pipeline_two_predicates_exact(uc1, policy, lanes, lag, pipeline):
    """The two synthetic-cost predicates (the worked example's selectivities
    0.6 / 0.1) pipelined over two SM shares (grid sizes) or two hardware SM
    partitions: orders, counts and pass sets equal the oracle's simulation
    with the route lag."""
    q, pm = _query(uc1, 0.6, 0.1, policy=policy, lanes=lanes, lag=lag, pipeline=pipeline)
    res = run_stream(q, uc1["Xd"], 512, max_in_flight=8)
    check_against_oracle(res, pm, 512, policy=policy, costs=model_costs(uc1["w"]), lag=lag)
    q.close()


def test_pipeline_cost_policy_puts_cheap_first(uc1):
    """Cost-driven routing evaluates the cheaper predicate A first in every
    routed batch; score-driven and selectivity-driven routing put the
    selective expensive B first (2 / (1 - 0.1) < 1 / (1 - 0.6))."""
    want = {"cost": [0, 1], "rank": [1, 0], "selectivity": [1, 0]}
    for policy, order in want.items():
        q, pm = _query(uc1, 0.6, 0.1, policy=policy, lanes=2, lag=1)
        res = run_stream(q, uc1["Xd"], 512, max_in_flight=8)
        routed = [r[2]["order"] for r in res if not r[2]["warmup"]][2:]
        assert routed and all(o == order for o in routed), (policy, routed)
        q.close()


@pytest.mark.parametrize("precision,pipeline", [("bf16", "shares"), ("fp32", "shares"), ("bf16", "partitions")])
def test_pipeline_four_cnn_predicates_exact(precision, pipeline):
    """Four CNN predicates (BF16 with the recheck cascade, or FP32) on four
    positions, four lanes, route lag 3: exact against the oracle."""
    import torch
    w = D.workload("cnn4")
    th = stored_thresholds("cnn4")
    F = D.stream_tuples(w, 72)
    pm = O.pass_matrix(O.udf_scores("frame", F, D.predicate_weights(w)), th)
    import paper_2403_14902_b300 as H
    q = H.Query("frame", frame=w.frame, max_batch=16, policy="rank", precision=precision, lanes=4, lag=3,
                max_in_flight=8, pipeline=pipeline)
    for i, udf in enumerate(D.predicate_weights(w)):
        q.add_cnn(udf, th[i])
    if precision == "bf16":
        q.calibrate(torch.from_numpy(D.calib_tuples(w)[:64]).cuda())
    res = run_stream(q, torch.from_numpy(F).cuda(), 16, max_in_flight=8)
    check_against_oracle(res, pm, 16, policy="rank", costs=model_costs(w), lag=3)
    q.close()


def test_pipeline_needs_lanes():
    import paper_2403_14902_b300 as H
    with pytest.raises(H.HydroError) as e:
        H.Query("vec", dim=512, max_batch=64, pipeline=True, lanes=1, lag=0)
    assert e.value.status == H.EUNSUPPORTED
