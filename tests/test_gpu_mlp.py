"""GPU parity of the FP32 MLP path (4,096 x 256 fp32 Gaussian-mixture tuples,
three MLP UDFs, batches of 256) against the oracle."""
import numpy as np
import pytest

import datagen as D
import oracle as O
from gpu_helpers import (check_against_oracle, make_query, model_costs, oracle_thresholds, run_stream,
                         score_tolerance_ok)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mlp3():
    import torch
    w = D.workload("mlp3")
    th, calib_scores = oracle_thresholds(w)
    X = D.stream_tuples(w)
    S = O.udf_scores("vec", X, D.predicate_weights(w))
    return dict(w=w, th=th, calib_rms=np.sqrt((calib_scores ** 2).mean(axis=0)), X=X, S=S,
                pm=O.pass_matrix(S, th), Xd=torch.from_numpy(X).cuda())


@pytest.mark.parametrize("policy", ["rank", "static", "all", "cost", "selectivity"])
def test_full_stream_parity(mlp3, policy):
    w = mlp3["w"]
    q = make_query(w, mlp3["th"], batch=w.batch, policy=policy)
    res = run_stream(q, mlp3["Xd"], w.batch)
    check_against_oracle(res, mlp3["pm"], w.batch, policy=policy, costs=model_costs(w))
    q.close()


@pytest.mark.parametrize("policy,lag,precision,lanes", [("rank", 0, "fp32", 1), ("rank", 1, "fp32", 1),
                                                        ("cost", 2, "fp32", 1), ("selectivity", 1, "fp32", 1),
                                                        ("rank", 1, "bf16", 1), ("rank", 3, "bf16", 4)])
def test_device_dispatch_matches_host_routing(mlp3, policy, lag, precision, lanes):
    """Routed batches dispatched on the device (the router writes the order,
    the lane's graph picks each position's predicate through SWITCH nodes)
    against the same query routed on the host (recheck graphs off, the host
    reads the order and launches the stages): identical orders, counts and
    pass sets, both equal to the oracle's simulation."""
    w = mlp3["w"]
    got = {}
    for graphs in (True, False):
        q = make_query(w, mlp3["th"], batch=w.batch, policy=policy, lag=lag, window=2, precision=precision,
                       lanes=lanes, max_in_flight=8, recheck_graphs=graphs)
        if precision == "bf16":
            q.calibrate(mlp3["Xd"][:512])
        res = run_stream(q, mlp3["Xd"], w.batch, max_in_flight=8)
        check_against_oracle(res, mlp3["pm"], w.batch, policy=policy, costs=model_costs(w), lag=lag, window=2)
        got[graphs] = [(r[2]["order"], r[1].tolist(), r[0].tolist()) for r in res]
        q.close()
    assert got[True] == got[False]


def test_device_dispatch_on_a_drifting_stream():
    """Eight segments of 4,096 tuples with their own cluster mixtures (six
    MLPs of cost 1:2:...:32): the orders change between batches; device
    dispatch and host routing agree with each other and with the oracle."""
    import torch
    w = D.workload("drift6", n=8 * 4096, extra=dict(D.WORKLOADS["drift6"].extra, segment_len=4096))
    th, _ = oracle_thresholds(w)
    X = D.stream_tuples(w)
    pm = O.pass_matrix(O.udf_scores("vec", X, D.predicate_weights(w)), th)
    Xd = torch.from_numpy(X).cuda()
    got = {}
    for graphs in (True, False):
        q = make_query(w, th, batch=1024, policy="rank", lag=1, window=2, recheck_graphs=graphs, max_in_flight=8)
        res = run_stream(q, Xd, 1024, max_in_flight=8)
        check_against_oracle(res, pm, 1024, policy="rank", costs=model_costs(w), lag=1, window=2)
        got[graphs] = [r[2]["order"] for r in res]
        q.close()
    assert got[True] == got[False]
    assert len({tuple(o) for o in got[True]}) > 1, "the drifting stream should change the order"


def test_static_permuted_order_and_lag0(mlp3):
    w = mlp3["w"]
    q = make_query(w, mlp3["th"], batch=w.batch, policy="static", static_order=[2, 0, 1])
    res = run_stream(q, mlp3["Xd"], w.batch)
    check_against_oracle(res, mlp3["pm"], w.batch, policy="static", costs=model_costs(w), static_order=[2, 0, 1])
    q.close()
    q = make_query(w, mlp3["th"], batch=w.batch, policy="rank", lag=0, window=2, warmup=2)
    res = run_stream(q, mlp3["Xd"], w.batch)
    check_against_oracle(res, mlp3["pm"], w.batch, policy="rank", costs=model_costs(w), lag=0, window=2, warmup=2)
    q.close()


def test_scores_fp32_within_tolerance_and_fp64_exactish(mlp3):
    import torch
    w = mlp3["w"]
    q = make_query(w, mlp3["th"], batch=w.batch)
    n = 1000   # not a multiple of the tile sizes
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    for i in range(len(w.udfs)):
        s64 = mlp3["S"][:n, i]
        q.udf_scores(i, "fp32", mlp3["Xd"][:n], out)
        s32 = out.cpu().numpy()
        assert score_tolerance_ok(s32, s64, mlp3["calib_rms"][i]).all()
        q.udf_scores(i, "fp64", mlp3["Xd"][:n], out)
        assert np.max(np.abs(out.cpu().numpy() - s64)) <= 1e-10 * max(1.0, np.abs(s64).max())
    q.close()


def test_calibrate_sets_margins(mlp3):
    import torch
    w = mlp3["w"]
    q = make_query(w, mlp3["th"], batch=w.batch)
    info = q.calibrate(torch.from_numpy(D.calib_tuples(w)).cuda())
    for d in info:
        assert 0 <= d["max_err_fp32"] < 1e-3
        assert d["margin_fp32"] >= 16 * d["max_err_fp32"]
    res = run_stream(q, mlp3["Xd"], w.batch)
    check_against_oracle(res, mlp3["pm"], w.batch, policy="rank", costs=model_costs(w))
    q.close()


def test_wide_margin_forces_fp64_recheck_and_stays_exact(mlp3):
    # a margin covering most scores sends nearly every tuple to the FP64 recheck
    w = mlp3["w"]
    q = make_query(w, mlp3["th"], batch=w.batch)
    for i in range(3):
        q.set_margins(i, 0.02, 5e-3, 2.0)
    res = run_stream(q, mlp3["Xd"], w.batch)
    check_against_oracle(res, mlp3["pm"], w.batch, policy="rank", costs=model_costs(w))
    assert sum(sum(r[2]["recheck_fp64"]) for r in res) > 1000
    q.close()


def test_edge_batches(mlp3):
    # empty, single tuple, ragged sizes (not multiples of 32 or of the tiles)
    import torch
    w = mlp3["w"]
    X = mlp3["Xd"]
    pm = mlp3["pm"]
    for n in [0, 1, 31, 33, 255, 256]:
        q = make_query(w, mlp3["th"], batch=256, policy="static")
        bid = q.submit(X[:n], n=n)
        words, counts, info = q.poll(bid)
        import paper_2403_14902_b300 as H
        bits = H.bits_from_words(words, n)
        assert np.array_equal(bits, O.result_bits(pm[:n]))
        assert counts.tolist() == O.static_counts(pm[:n], [0, 1, 2]).tolist()
        q.close()


def test_all_pass_all_fail_thresholds(mlp3):
    import paper_2403_14902_b300 as H
    w = mlp3["w"]
    lo = [float(mlp3["S"][:, i].min()) - 1.0 for i in range(3)]
    hi = [float(mlp3["S"][:, i].max()) + 1.0 for i in range(3)]
    for th, want in [(lo, True), (hi, False)]:
        q = make_query(w, th, batch=256)
        res = run_stream(q, mlp3["Xd"], 256)
        assert all(r[0].all() == want and (r[0].any() == want) for r in res)
        q.close()


def test_single_predicate_and_determinism(mlp3):
    w = mlp3["w"]
    runs = []
    for _ in range(2):
        q = make_query(w, mlp3["th"], batch=w.batch, preds=[1])
        res = run_stream(q, mlp3["Xd"], w.batch)
        runs.append(res)
        q.close()
    pm1 = mlp3["pm"][:, [1]]
    check_against_oracle(runs[0], pm1, w.batch, policy="rank", costs=[model_costs(w)[1]])
    for a, b in zip(*runs):
        assert np.array_equal(a[0], b[0]) and a[1].tolist() == b[1].tolist()


def test_api_errors_on_device(mlp3):
    import paper_2403_14902_b300 as H
    w = mlp3["w"]
    q = make_query(w, mlp3["th"], batch=16, max_in_flight=1)
    with pytest.raises(H.HydroError) as e:
        q.submit(mlp3["Xd"][:17])
    assert e.value.status == H.EINVAL
    bid = q.submit(mlp3["Xd"][:16])
    with pytest.raises(H.HydroError) as e:
        q.submit(mlp3["Xd"][:16])          # the only slot is busy
    assert e.value.status == H.EAGAIN
    q.poll(bid)
    with pytest.raises(H.HydroError) as e:
        q.poll(bid)                        # already polled
    assert e.value.status == H.ENOTFOUND
    with pytest.raises(H.HydroError) as e:
        q.add_mlp(D.predicate_weights(w)[0], 0.0)   # after the first submit
    assert e.value.status == H.ESTATE
    q.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_two_lanes_exact(mlp3, precision):
    import torch

    import paper_2403_14902_b300 as H
    w = mlp3["w"]
    q = H.Query("vec", dim=w.dim, max_batch=w.batch, policy="rank", precision=precision, lanes=2, max_in_flight=4)
    for i, layers in enumerate(D.predicate_weights(w)):
        q.add_mlp(layers, mlp3["th"][i])
    q.calibrate(torch.from_numpy(D.calib_tuples(w)).cuda())
    res = run_stream(q, mlp3["Xd"], w.batch, max_in_flight=4)
    check_against_oracle(res, mlp3["pm"], w.batch, policy="rank", costs=model_costs(w))
    q.close()
