"""GPU parity of the CNN path (3x64x64 uint8 frames, four CNN UDFs with 2/4/6/8
conv3x3 layers) against the oracle: FP32, BF16-with-recheck and split-BF16
working precision, small streams element by element and the full
65,536-frame stream in the bench's launch configuration against the stored
oracle pass matrix of the whole stream."""
import numpy as np
import pytest

import datagen as D
import oracle as O
from gpu_helpers import (check_against_oracle, make_query, model_costs, run_stream, score_tolerance_ok,
                         stored_pass_matrix, stored_thresholds)

pytestmark = pytest.mark.gpu

N_SMALL = 72          # 4 batches of 16 + a ragged batch of 8
B_SMALL = 16


@pytest.fixture(scope="module")
def cnn4():
    import torch
    w = D.workload("cnn4")
    th = stored_thresholds("cnn4")
    F = D.stream_tuples(w, N_SMALL)
    S = O.udf_scores("frame", F, D.predicate_weights(w))
    calib = D.calib_tuples(w)
    return dict(w=w, th=th, F=F, S=S, pm=O.pass_matrix(S, th), Fd=torch.from_numpy(F).cuda(),
                calib_d=torch.from_numpy(calib[:64]).cuda(), rms=np.sqrt((S ** 2).mean(axis=0)))


@pytest.mark.parametrize("policy,precision,lanes", [("rank", "fp32", 1), ("cost", "fp32", 1), ("rank", "bf16", 2)])
def test_measured_cost_routing(cnn4, policy, precision, lanes):
    """Measured cost (device time per evaluated tuple): the orders depend on
    timing, so each batch is checked against its own reported order: exact
    pass set, evaluation and pass counts from the pass matrix under that
    order; every stage reports its time, and the 8-layer UDF costs more per
    tuple than the 2-layer one, so both policies evaluate it last."""
    w = cnn4["w"]
    # a first batch through the same kernels, so that no measured stage pays their loading
    warm = make_query(w, cnn4["th"], batch=B_SMALL, precision=precision)
    run_stream(warm, cnn4["Fd"][:B_SMALL], B_SMALL)
    warm.close()
    q = make_query(w, cnn4["th"], batch=B_SMALL, policy=policy, precision=precision, cost="measured",
                   lag=lanes - 1, lanes=lanes)
    res = run_stream(q, cnn4["Fd"], B_SMALL)
    for b, (bits, counts, info) in enumerate(res):
        pm = cnn4["pm"][b * B_SMALL:(b + 1) * B_SMALL]
        assert np.array_equal(bits, O.result_bits(pm)), f"batch {b}: pass set"
        assert sorted(info["order"]) == [0, 1, 2, 3]
        want = [len(pm)] * 4 if info["warmup"] else O.static_counts(pm, info["order"]).tolist()
        assert counts.tolist() == want, f"batch {b}: counts {counts} vs {want}"
        assert all(t > 0 for t in info["stage_ns"])
        if b == 0:
            # the first batch's stage times may include the first launch of a recheck level's
            # kernels; the routed batches below show the measured cost ordering
            assert info["warmup"]
        else:
            assert info["order"][-1] == 3, f"batch {b}: order {info['order']}"
    q.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_cnn_edge_batches(cnn4, precision):
    """Empty, one-frame and ragged batches (below one 128-pixel-row tile of
    frames, not a multiple of the 16-frame batch), static declared order."""
    import paper_2403_14902_b300 as H
    w = cnn4["w"]
    pm = cnn4["pm"]
    for n in [0, 1, 5, 16]:
        q = make_query(w, cnn4["th"], batch=B_SMALL, policy="static", precision=precision)
        bid = q.submit(cnn4["Fd"][:n], n=n)
        words, counts, _ = q.poll(bid)
        assert np.array_equal(H.bits_from_words(words, n), O.result_bits(pm[:n]))
        assert counts.tolist() == O.static_counts(pm[:n], [0, 1, 2, 3]).tolist()
        q.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("policy", ["rank", "static", "all"])
def test_small_stream_parity(cnn4, precision, policy):
    w = cnn4["w"]
    q = make_query(w, cnn4["th"], batch=B_SMALL, policy=policy, precision=precision)
    res = run_stream(q, cnn4["Fd"], B_SMALL)
    check_against_oracle(res, cnn4["pm"], B_SMALL, policy=policy, costs=model_costs(w))
    if precision == "bf16":
        assert sum(sum(r[2]["recheck_fp32"]) for r in res) >= 0
    q.close()


@pytest.mark.parametrize("policy", ["rank", "static", "all"])
def test_split_working_precision_parity(cnn4, policy):
    """Split BF16 as the working precision (FP32-class scores on the tensor
    cores, the static arm that isolates routing from precision): orders,
    counts and pass sets exact against the oracle; its calibrated margin
    sends the few close scores to the FP32 level."""
    w = cnn4["w"]
    q = make_query(w, cnn4["th"], batch=B_SMALL, policy=policy, precision="bf16x3")
    info = q.calibrate(cnn4["calib_d"])
    for d in info:
        assert 0 < d["max_err_tf32"] < 5e-3 and d["margin_tf32"] >= 8 * d["max_err_tf32"]
    res = run_stream(q, cnn4["Fd"], B_SMALL)
    check_against_oracle(res, cnn4["pm"], B_SMALL, policy=policy, costs=model_costs(w))
    assert sum(sum(r[2]["recheck_tf32"]) for r in res) == 0, "no split level after a split working level"
    q.close()


def test_split_working_precision_wide_margin(cnn4):
    """Every split-BF16 score sent on to FP32 (margin wider than the score
    spread) and every FP32 score on to FP64: the pass set does not move."""
    w = cnn4["w"]
    q = make_query(w, cnn4["th"], batch=B_SMALL, policy="rank", precision="bf16x3")
    for i in range(4):
        q.set_margins(i, 0.02, 10.0, 10.0)
    res = run_stream(q, cnn4["Fd"][:40], B_SMALL)
    check_against_oracle(res, cnn4["pm"][:40], B_SMALL, policy="rank", costs=model_costs(w))
    evaluated = sum(int(r[1].sum()) for r in res)
    assert sum(sum(r[2]["recheck_fp32"]) for r in res) == evaluated
    assert sum(sum(r[2]["recheck_fp64"]) for r in res) == evaluated
    q.close()


@pytest.mark.parametrize("precision,margins", [("bf16", None), ("bf16", (10.0, 10.0, 1e-5)),
                                               ("fp32", (0.02, 5e-3, 0.05))])
def test_recheck_graphs_match_direct_launches(cnn4, precision, margins):
    """The recheck levels replayed from captured graphs (each level an IF node
    behind a gate kernel, band tuples staged per lane) give the same orders,
    counts and pass sets as launching every level directly, on two stream
    lanes; with mostly empty bands they launch fewer kernels.  Wide margins
    drive every level of the cascade through the graphs."""
    w = cnn4["w"]
    launches = {}
    for graphs in (True, False):
        q = make_query(w, cnn4["th"], batch=B_SMALL, policy="rank", precision=precision, lanes=2, lag=1,
                       recheck_graphs=graphs)
        if margins:
            for i in range(4):
                q.set_margins(i, *margins)
        q.profile(False)
        res = run_stream(q, cnn4["Fd"], B_SMALL)
        check_against_oracle(res, cnn4["pm"], B_SMALL, policy="rank", costs=model_costs(w))
        launches[graphs] = q.profile_read()[1]
        q.close()
    assert launches[True] > 0
    if margins is None:
        assert launches[True] < launches[False], launches


@pytest.mark.parametrize("tf32_margin", [5e-3, 10.0])
def test_bf16_wide_margin_rechecks_and_stays_exact(cnn4, tf32_margin):
    # a margin wider than the score spread sends every tuple through the
    # 3xTF32 recheck (and with the wide 3xTF32 margin, all of them on through
    # the FP32 CUDA-core recheck); the pass set must not move
    w = cnn4["w"]
    q = make_query(w, cnn4["th"], batch=B_SMALL, policy="rank", precision="bf16")
    for i in range(4):
        q.set_margins(i, 10.0, tf32_margin, 1e-5)
    res = run_stream(q, cnn4["Fd"], B_SMALL)
    check_against_oracle(res, cnn4["pm"], B_SMALL, policy="rank", costs=model_costs(w))
    evaluated = sum(int(r[1].sum()) for r in res)
    assert sum(sum(r[2]["recheck_tf32"]) for r in res) == evaluated
    if tf32_margin >= 10.0:
        assert sum(sum(r[2]["recheck_fp32"]) for r in res) == evaluated
    q.close()


def test_fp32_level_both_band_conv_forms(cnn4):
    """Batches of 32 with every evaluated frame sent through the split level on
    to FP32: the FP32 bands' conv layers take the K-split form (nine partial
    planes, one per tap, summed in order) for bands of up to a tenth of the
    batch capacity (3 frames here) and the unsplit form above; both occur here
    (bands of 32, 10, 8, 3 and 1 frames), and the pass set is the oracle's."""
    w = cnn4["w"]
    q = make_query(w, cnn4["th"], batch=32, policy="rank", precision="bf16")
    for i in range(4):
        q.set_margins(i, 10.0, 10.0, 1e-5)
    res = run_stream(q, cnn4["Fd"], 32)
    check_against_oracle(res, cnn4["pm"], 32, policy="rank", costs=model_costs(w))
    bands = [n for r in res for n in r[2]["recheck_fp32"]]
    assert sum(bands) == sum(int(r[1].sum()) for r in res)
    split_frames = min(8, 32 // 10)
    assert any(0 < n <= split_frames for n in bands) and any(n > split_frames for n in bands), bands
    q.close()


@pytest.mark.parametrize("precision,margins", [("fp32", (0.02, 5e-3, 10.0)), ("bf16", (10.0, 10.0, 1e-5))])
def test_other_frame_size(cnn4, precision, margins):
    """Frames of 3 x 16 x 24 with the workload's four CNN UDFs: H*W = 384 is a
    multiple of 128 but not of 512 (the recheck levels pool each frame as one
    pixel range) and the width is not the tensor-core conv's 64, so the layers
    after the first run on CUDA cores; the first layer's tensor-core kernel
    takes tiles spanning several rows.  Margins send every evaluated frame
    through every recheck level; pass set and counts exact."""
    import torch
    import paper_2403_14902_b300 as H
    w = cnn4["w"]
    rng = np.random.default_rng(11)
    F = rng.integers(0, 48, size=(40, 3, 16, 24), dtype=np.uint8)
    weights = D.predicate_weights(w)
    S = O.udf_scores("frame", F, weights)
    th = [float(np.median(S[:, i])) for i in range(S.shape[1])]
    pm = O.pass_matrix(S, th)
    q = H.Query("frame", frame=(3, 16, 24), max_batch=16, policy="static", precision=precision)
    for i, u in enumerate(weights):
        q.add_cnn(u, th[i])
        q.set_margins(i, *margins)
    res = run_stream(q, torch.from_numpy(F).cuda(), 16)
    check_against_oracle(res, pm, 16, policy="static", costs=model_costs(w))
    evaluated = sum(int(r[1].sum()) for r in res)
    level = "recheck_fp64" if precision == "fp32" else "recheck_fp32"
    assert sum(sum(r[2][level]) for r in res) == evaluated
    q.close()


def test_fp32_wide_margin_goes_to_fp64(cnn4):
    w = cnn4["w"]
    q = make_query(w, cnn4["th"], batch=B_SMALL, policy="static", precision="fp32")
    for i in range(4):
        q.set_margins(i, 0.02, 5e-3, 0.05)
    res = run_stream(q, cnn4["Fd"], B_SMALL)
    check_against_oracle(res, cnn4["pm"], B_SMALL, policy="static", costs=model_costs(w))
    assert sum(sum(r[2]["recheck_fp64"]) for r in res) > 0
    q.close()


def test_udf_scores_error(cnn4):
    import torch
    w = cnn4["w"]
    q = make_query(w, cnn4["th"], batch=64, precision="bf16")
    n = 40
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    for i in range(4):
        s64 = cnn4["S"][:n, i]
        q.udf_scores(i, "fp32", cnn4["Fd"][:n], out)
        assert score_tolerance_ok(out.cpu().numpy(), s64, cnn4["rms"][i]).all()
        q.udf_scores(i, "fp64", cnn4["Fd"][:n], out)
        assert np.max(np.abs(out.cpu().numpy() - s64)) <= 1e-10 * max(1.0, np.abs(s64).max())
        q.udf_scores(i, "bf16", cnn4["Fd"][:n], out)
        # the BF16 error must sit well inside the 0.02 recheck margin
        assert np.max(np.abs(out.cpu().numpy() - s64)) < 0.02 / 2
        q.udf_scores(i, "tf32x3", cnn4["Fd"][:n], out)
        # 3xTF32 is FP32-accurate up to the tensor cores' accumulation
        assert score_tolerance_ok(out.cpu().numpy(), s64, cnn4["rms"][i]).all()
        assert np.max(np.abs(out.cpu().numpy() - s64)) < 5e-3
    q.close()


def test_split_bf16_recheck_level(cnn4):
    """The first recheck level in split BF16 ([hi | lo] operands, three BF16
    passes): its scores are within the FP32 tolerance like 3xTF32's, its
    calibrated margin covers its error, and the stream stays exact."""
    import torch
    w = cnn4["w"]
    q = make_query(w, cnn4["th"], batch=B_SMALL, precision="bf16", split="bf16x3")
    n = 40
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    for i in range(4):
        s64 = cnn4["S"][:n, i]
        q.udf_scores(i, "bf16x3", cnn4["Fd"][:n], out)
        e_sb = np.max(np.abs(out.cpu().numpy() - s64))
        q.udf_scores(i, "bf16", cnn4["Fd"][:n], out)
        e16 = np.max(np.abs(out.cpu().numpy() - s64))
        assert e_sb < 0.2 * e16, (i, e_sb, e16)
    info = q.calibrate(cnn4["calib_d"])
    for d in info:
        assert 0 < d["max_err_tf32"] < 5e-3 and d["margin_tf32"] >= 8 * d["max_err_tf32"]
    res = run_stream(q, cnn4["Fd"], B_SMALL)
    check_against_oracle(res, cnn4["pm"], B_SMALL, policy="rank", costs=model_costs(w))
    assert sum(sum(r[2]["recheck_tf32"]) for r in res) > 0
    q.close()


def test_calibrate_bf16(cnn4):
    w = cnn4["w"]
    q = make_query(w, cnn4["th"], batch=B_SMALL, precision="bf16")
    info = q.calibrate(cnn4["calib_d"])
    for d in info:
        assert d["max_err_lowp"] < 0.02 / 2
        assert d["margin_lowp"] >= 0.02
        assert d["margin_fp32"] >= 16 * d["max_err_fp32"]
        assert 0 < d["max_err_tf32"] < 5e-3 and d["margin_tf32"] >= 8 * d["max_err_tf32"]
    res = run_stream(q, cnn4["Fd"], B_SMALL)
    check_against_oracle(res, cnn4["pm"], B_SMALL, policy="rank", costs=model_costs(w))
    q.close()


def test_full_stream_parity_bf16():
    """The full 65,536-frame stream in the bench's launch configuration:
    batches of 1,024, rank routing, BF16 with the recheck cascade, four
    stream lanes (route lag 3), 8 batches in flight.  Every frame's result
    and every batch's order, evaluation and pass counts equal the oracle's
    (its stored FP64 pass matrix of the whole stream and its router
    simulation with lag 3)."""
    import torch
    w = D.workload("cnn4")
    th = stored_thresholds("cnn4")
    pm = stored_pass_matrix("cnn4")
    assert pm.shape == (w.n, 4)
    Fd = torch.from_numpy(D.stream_tuples(w)).cuda()
    q = make_query(w, th, batch=w.batch, policy="rank", precision="bf16", lanes=4, lag=3, max_in_flight=8)
    q.calibrate(torch.from_numpy(D.calib_tuples(w)[:64]).cuda())
    res = run_stream(q, Fd, w.batch, max_in_flight=8)
    bits = np.concatenate([r[0] for r in res])
    assert np.array_equal(bits, O.result_bits(pm)), f"{int((bits != O.result_bits(pm)).sum())} frames differ"
    check_against_oracle(res, pm, w.batch, policy="rank", costs=model_costs(w), lag=3)
    q.close()


@pytest.mark.parametrize("policy,precision,lanes,lag", [("static", "bf16x3", 4, 3), ("all", "bf16", 4, 3)])
def test_full_stream_parity_static_arms(policy, precision, lanes, lag):
    """The bench's static arms over the full stream: split BF16 as the
    working precision in declared order, and every predicate on every frame
    in BF16.  Every frame's result and every batch's counts equal the
    oracle's."""
    import torch
    w = D.workload("cnn4")
    th = stored_thresholds("cnn4")
    pm = stored_pass_matrix("cnn4")
    Fd = torch.from_numpy(D.stream_tuples(w)).cuda()
    q = make_query(w, th, batch=w.batch, policy=policy, precision=precision, lanes=lanes, lag=lag, max_in_flight=8)
    q.calibrate(torch.from_numpy(D.calib_tuples(w)[:64]).cuda())
    res = run_stream(q, Fd, w.batch, max_in_flight=8)
    check_against_oracle(res, pm, w.batch, policy=policy, costs=model_costs(w), lag=lag)
    q.close()


@pytest.mark.parametrize("precision,lanes,lag", [("bf16", 2, 1), ("fp32", 2, 1), ("bf16", 3, 2), ("bf16", 4, 3)])
def test_lanes_match_oracle(cnn4, precision, lanes, lag):
    """Batches on `lanes` stream lanes (route lag `lag`): the same orders,
    counts and pass sets as the oracle's simulation with that lag."""
    import paper_2403_14902_b300 as H
    w = cnn4["w"]
    q = H.Query("frame", frame=w.frame, max_batch=B_SMALL, policy="rank", precision=precision, lanes=lanes,
                lag=lag, max_in_flight=4)
    for i, udf in enumerate(D.predicate_weights(w)):
        q.add_cnn(udf, cnn4["th"][i])
    if precision == "bf16":
        q.calibrate(cnn4["calib_d"])
    res = run_stream(q, cnn4["Fd"], B_SMALL, max_in_flight=4)
    check_against_oracle(res, cnn4["pm"], B_SMALL, policy="rank", costs=model_costs(w), lag=lag)
    q.close()


def test_two_lanes_need_route_lag():
    import paper_2403_14902_b300 as H
    with pytest.raises(H.HydroError) as e:
        H.Query("frame", frame=(3, 64, 64), max_batch=8, lanes=2, lag=0)
    assert e.value.status == H.EINVAL


@pytest.mark.parametrize("frame", [(1, 16, 8), (3, 8, 48), (2, 4, 256), (3, 2, 512), (3, 1, 640)])
@pytest.mark.parametrize("aligned", [True, False])
def test_first_layer_geometries(frame, aligned):
    """The first conv layer over frame shapes whose 128-pixel tiles span 16
    rows down to a fraction of one row (the tensor-core layer reads a window
    of rows around each tile; 640 columns go to the CUDA-core layer), from
    16-byte-aligned frames and from frames one byte off: the BF16 scores of a
    3-32-64 CNN stay within BF16 error of the oracle's FP64 scores, and the
    FP32 scores within FP32 tolerance."""
    import torch
    import paper_2403_14902_b300 as H
    C, Hh, Wd = frame
    w = D.workload("cnn4", frame=frame, udfs=((C, 32, 64),), selectivity=(0.5,), head_gain=(8.0,))
    weights = D.cnn_weights(w, 11, (C, 32, 64), 8.0)
    n = 24
    F = D.blob_frames(w, 5, n)
    S = O.udf_scores("frame", F, [weights])[:, 0]
    buf = torch.zeros(F.size + 16, dtype=torch.uint8, device="cuda")
    off = 0 if aligned else 1
    Fd = buf[off:off + F.size].view(F.shape)
    Fd.copy_(torch.from_numpy(F))
    assert (Fd.data_ptr() % 16 == 0) == aligned
    q = H.Query("frame", frame=frame, max_batch=32, precision="bf16")
    q.add_cnn(weights, 0.0)
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    q.udf_scores(0, "fp32", Fd, out)
    assert score_tolerance_ok(out.cpu().numpy(), S, np.sqrt((S ** 2).mean())).all()
    q.udf_scores(0, "bf16", Fd, out)
    err = np.max(np.abs(out.cpu().numpy() - S))
    assert err < 0.02 * np.max(np.abs(S)), (err, np.max(np.abs(S)))
    q.close()
