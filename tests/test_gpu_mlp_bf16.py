"""GPU parity of the BF16 tensor-core MLP path: tuple rows gathered into BF16,
hidden layers on tcgen05 with the one-output last layer folded into the last
hidden layer's epilogue, then the FP32 and FP64 rechecks of the band around
each threshold.  Scores are checked against a BF16-rounding emulation of the
forward pass (FP64 arithmetic on BF16-rounded operands) and against the FP64
oracle; the pass set, orders and counts must equal the oracle's exactly."""
import numpy as np
import pytest

import datagen as D
import oracle as O
from gpu_helpers import check_against_oracle, make_query, model_costs, oracle_thresholds, run_stream

pytestmark = pytest.mark.gpu


def bf16_round(a):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_forward(X, layers):
    """The tensor-core path's rounding points: BF16 inputs, weights and
    stored hidden activations; exact accumulation; the last hidden layer's
    activation stays unrounded and meets the FP32 head weights."""
    h = bf16_round(X)
    L = len(layers)
    for l, (W, b) in enumerate(layers[:-1]):
        a = np.maximum(h @ bf16_round(W).T + np.asarray(b, np.float64), 0.0)
        h = a if l == L - 2 else bf16_round(a)
    W, b = layers[-1]
    return h @ np.asarray(W, np.float64)[0] + float(b[0])


@pytest.fixture(scope="module")
def mlp3():
    import torch
    w = D.workload("mlp3")
    th, calib = oracle_thresholds(w)
    X = D.stream_tuples(w)
    S = O.udf_scores("vec", X, D.predicate_weights(w))
    return dict(w=w, th=th, rms=np.sqrt((calib ** 2).mean(axis=0)), X=X, S=S, pm=O.pass_matrix(S, th),
                Xd=torch.from_numpy(X).cuda(), calib=torch.from_numpy(D.calib_tuples(w)).cuda())


def test_bf16_scores_match_rounding_emulation(mlp3):
    # 1,000 rows in one launch: seven full 128-row tiles and a ragged tail
    import torch
    w = mlp3["w"]
    n = 1000
    q = make_query(w, mlp3["th"], batch=n, precision="bf16")
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    weights = D.predicate_weights(w)
    for i in range(len(w.udfs)):
        q.udf_scores(i, "bf16", mlp3["Xd"][:n], out)
        s16 = out.cpu().numpy()
        emu = bf16_forward(mlp3["X"][:n], weights[i])
        s64 = mlp3["S"][:n, i]
        scale = np.maximum(np.abs(emu), mlp3["rms"][i])
        # FP32 accumulation order and the odd hidden activation rounded to the
        # neighbouring BF16 value are all that separate kernel and emulation
        assert np.max(np.abs(s16 - emu) / scale) < 2e-3, i
        # BF16 against exact: a few BF16 ulps of the score scale
        assert np.max(np.abs(s16 - s64) / np.maximum(np.abs(s64), mlp3["rms"][i])) < 0.1, i
        assert np.median(np.abs(s16 - s64) / np.maximum(np.abs(s64), mlp3["rms"][i])) < 1e-2, i
    q.close()


def test_bf16_calibrate_then_exact_stream(mlp3):
    w = mlp3["w"]
    for policy in ["rank", "static", "all"]:
        q = make_query(w, mlp3["th"], batch=w.batch, precision="bf16", policy=policy)
        info = q.calibrate(mlp3["calib"])
        for i, d in enumerate(info):
            assert 0 < d["max_err_lowp"] < 0.05 * mlp3["rms"][i]
            assert d["margin_lowp"] >= 4 * d["max_err_lowp"]
            assert d["margin_fp32"] >= 16 * d["max_err_fp32"]
        res = run_stream(q, mlp3["Xd"], w.batch)
        check_against_oracle(res, mlp3["pm"], w.batch, policy=policy, costs=model_costs(w))
        assert sum(sum(r[2]["recheck_fp32"]) for r in res) > 0
        q.close()


def test_bf16_wide_margin_rechecks_everything_and_stays_exact(mlp3):
    w = mlp3["w"]
    q = make_query(w, mlp3["th"], batch=w.batch, precision="bf16")
    q.calibrate(mlp3["calib"])
    for i in range(3):
        q.set_margins(i, 1e3, 5e-3, 1e3)
    res = run_stream(q, mlp3["Xd"], w.batch)
    check_against_oracle(res, mlp3["pm"], w.batch, policy="rank", costs=model_costs(w))
    ev = sum(sum(r[1]) for r in res)
    assert sum(sum(r[2]["recheck_fp64"]) for r in res) == ev
    q.close()


def test_bf16_edge_batches(mlp3):
    import paper_2403_14902_b300 as H
    w = mlp3["w"]
    for n in [0, 1, 127, 129, 256]:
        q = make_query(w, mlp3["th"], batch=256, precision="bf16", policy="static")
        q.calibrate(mlp3["calib"])
        bid = q.submit(mlp3["Xd"][:n], n=n)
        words, counts, info = q.poll(bid)
        assert np.array_equal(H.bits_from_words(words, n), O.result_bits(mlp3["pm"][:n]))
        assert counts.tolist() == O.static_counts(mlp3["pm"][:n], [0, 1, 2]).tolist()
        q.close()


def test_bf16_drift6_widths_sampled():
    """The drifting stream's six 512-h-1 predicates (h = 64 ... 2048, so every
    column-tile width of the kernel) on 8,192 tuples in batches of 4,096."""
    import torch
    w = D.workload("drift6", n=8192)
    th = oracle_thresholds(w)[0]
    X = D.stream_tuples(w)
    S = O.udf_scores("vec", X, D.predicate_weights(w))
    pm = O.pass_matrix(S, th)
    q = make_query(w, th, batch=w.batch, precision="bf16", policy="rank")
    q.calibrate(torch.from_numpy(D.calib_tuples(w)[:4096]).cuda())
    Xd = torch.from_numpy(X).cuda()
    out = torch.empty(w.batch, dtype=torch.float64, device="cuda")
    weights = D.predicate_weights(w)
    for i in range(len(w.udfs)):
        q.udf_scores(i, "bf16", Xd[:w.batch], out)
        emu = bf16_forward(X[:w.batch], weights[i])
        scale = np.maximum(np.abs(emu), np.sqrt((S[:, i] ** 2).mean()))
        assert np.max(np.abs(out.cpu().numpy() - emu) / scale) < 2e-3, i
    res = run_stream(q, Xd, w.batch)
    check_against_oracle(res, pm, w.batch, policy="rank", costs=model_costs(w))
    q.close()
