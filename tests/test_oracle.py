"""Pins for the oracle: every check here ties the oracle to something other
than itself (torch float64 as an independent implementation, closed forms,
brute force over orders, and the numbers the paper prints)."""
import json
import os
from fractions import Fraction
from itertools import permutations

import numpy as np
import pytest
import torch
import torch.nn.functional as F

import datagen as D
import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _torch_mlp(X, layers):
    h = torch.from_numpy(np.asarray(X, np.float64))
    for l, (W, b) in enumerate(layers):
        h = F.linear(h, torch.from_numpy(W.astype(np.float64)), torch.from_numpy(b.astype(np.float64)))
        if l + 1 < len(layers):
            h = F.relu(h)
    return h[:, 0].numpy()


def _torch_cnn(frames, udf):
    convs, (hw, hb) = udf
    a = torch.from_numpy(frames.astype(np.float64)) / 255.0
    for W, b in convs:
        a = F.relu(F.conv2d(a, torch.from_numpy(W.astype(np.float64)),
                            torch.from_numpy(b.astype(np.float64)), padding=1))
    return (a.mean(dim=(2, 3)) @ torch.from_numpy(hw.astype(np.float64)) + hb).numpy()


# ------------------------------------------------------------ UDF scores

def test_mlp_scores_match_torch_float64():
    w = D.workload("mlp3")
    ws = D.predicate_weights(w)
    X = D.calib_tuples(w)[:128]
    for layers in ws:
        got = O.mlp_scores(X, layers)
        ref = _torch_mlp(X, layers)
        assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_mlp_random_shapes_match_torch_float64():
    g = np.random.default_rng(3)
    for dims in [(1, 1), (7, 1), (5, 3, 1), (33, 17, 9, 1)]:
        layers = [(g.standard_normal((dims[l + 1], dims[l])).astype(np.float32),
                   g.standard_normal(dims[l + 1]).astype(np.float32)) for l in range(len(dims) - 1)]
        X = g.standard_normal((11, dims[0])).astype(np.float32)
        np.testing.assert_allclose(O.mlp_scores(X, layers), _torch_mlp(X, layers), rtol=1e-12, atol=1e-12)


def test_mlp_single_layer_closed_form():
    # dims (d, 1): the score is w.x + b, summed exactly in rationals
    g = np.random.default_rng(4)
    W = g.integers(-8, 8, (1, 6)).astype(np.float32) / 4
    b = np.array([0.5], np.float32)
    X = g.integers(-5, 5, (4, 6)).astype(np.float32) / 2
    got = O.mlp_scores(X, [(W, b)])
    for r in range(4):
        exact = sum(Fraction(float(W[0, k])) * Fraction(float(X[r, k])) for k in range(6)) + Fraction(0.5)
        assert got[r] == float(exact)


def test_mlp_relu_only_on_hidden_layers():
    # negative last-layer output must survive (no ReLU on the score)
    W1 = np.eye(2, dtype=np.float32)
    b1 = np.zeros(2, np.float32)
    W2 = np.array([[-1.0, -1.0]], np.float32)
    b2 = np.array([-0.25], np.float32)
    X = np.array([[1.0, 2.0], [-3.0, 1.0]], np.float32)
    got = O.mlp_scores(X, [(W1, b1), (W2, b2)])
    assert got[0] == -3.25          # relu(1)+relu(2) = 3
    assert got[1] == -1.25          # relu(-3)=0, relu(1)=1


def test_cnn_scores_match_torch_float64():
    w = D.workload("cnn4")
    frames = D.calib_tuples(w)[:2]
    ws = D.predicate_weights(w)
    for udf in ws[:2]:
        got = O.cnn_scores(frames, udf)
        ref = _torch_cnn(frames, udf)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_cnn_small_random_match_torch_float64():
    g = np.random.default_rng(5)
    frames = g.integers(0, 256, (3, 2, 5, 7)).astype(np.uint8)   # odd, non-square
    chans = (2, 3, 4)
    convs = [(g.standard_normal((chans[l + 1], chans[l], 3, 3)).astype(np.float32),
              g.standard_normal(chans[l + 1]).astype(np.float32)) for l in range(2)]
    udf = (convs, (g.standard_normal(4).astype(np.float32), 0.75))
    np.testing.assert_allclose(O.cnn_scores(frames, udf), _torch_cnn(frames, udf), rtol=1e-12, atol=1e-12)


def test_cnn_shift_tap_closed_form():
    # one channel, only tap (ky=1, kx=2) = 1: out[y][x] = in[y][x+1], zero in
    # the last column (padding); the pooled score is then sum(in[:, 1:]) / (H*W*255)
    g = np.random.default_rng(6)
    H, W = 4, 6
    frames = g.integers(0, 256, (2, 1, H, W)).astype(np.uint8)
    Wc = np.zeros((1, 1, 3, 3), np.float32)
    Wc[0, 0, 1, 2] = 1.0
    udf = ([(Wc, np.zeros(1, np.float32))], (np.ones(1, np.float32), 0.0))
    got = O.cnn_scores(frames, udf)
    for f in range(2):
        exact = Fraction(int(frames[f, 0, :, 1:].astype(np.int64).sum()), H * W * 255)
        assert abs(got[f] - float(exact)) <= 1e-15


def test_cnn_bias_only_closed_form():
    # zero conv weights: every activation is relu(bias); score = hb + hw . relu(b_last)
    chans = (3, 2, 2)
    convs = [(np.zeros((2, 3, 3, 3), np.float32), np.array([0.5, -1.0], np.float32)),
             (np.zeros((2, 2, 3, 3), np.float32), np.array([-0.25, 2.0], np.float32))]
    udf = (convs, (np.array([3.0, 0.5], np.float32), -1.0))
    frames = np.random.default_rng(7).integers(0, 256, (2, 3, 8, 8)).astype(np.uint8)
    assert np.all(O.cnn_scores(frames, udf) == -1.0 + 3.0 * 0.0 + 0.5 * 2.0)


def test_planted_tap_transpose_is_caught():
    # plant a mistake in the oracle's input (transposed 3x3 taps): the torch
    # comparison used above must see it
    g = np.random.default_rng(8)
    frames = g.integers(0, 256, (1, 2, 6, 6)).astype(np.uint8)
    Wc = g.standard_normal((2, 2, 3, 3)).astype(np.float32)
    udf = ([(Wc, np.zeros(2, np.float32))], (np.ones(2, np.float32), 0.0))
    bad = ([(np.ascontiguousarray(Wc.transpose(0, 1, 3, 2)), np.zeros(2, np.float32))], udf[1])
    assert np.max(np.abs(O.cnn_scores(frames, bad) - _torch_cnn(frames, udf))) > 1e-6


# ------------------------------------------------------------ thresholds, pass set

@pytest.mark.parametrize("s", [0.0, 0.1, 0.2, 0.5, 0.8, 0.9, 1.0])
def test_threshold_gives_exact_calibration_selectivity(s):
    sc = np.random.default_rng(9).standard_normal(1024)
    t = O.threshold_for_selectivity(sc, s)
    assert int((sc > t).sum()) == int(round(s * 1024))


def test_bitmap_layout_lsb_first():
    bits = np.zeros(70, bool)
    bits[[0, 5, 31, 32, 69]] = True
    w = O.bitmap_words(bits)
    assert w.tolist() == [(1 << 0) | (1 << 5) | (1 << 31), 1, 1 << 5]


def test_result_is_order_invariant_bruteforce():
    # the conjunction is the same whichever order evaluates it, and the
    # short-circuit counts of a static order follow the definition tuple by tuple
    g = np.random.default_rng(10)
    for P in range(1, 6):
        pm = g.random((40, P)) < g.random(P)[None, :]
        ref = pm.all(axis=1)
        for order in permutations(range(P)):
            sim = O.simulate(pm, batch=40, policy="static", static_order=order)
            assert np.array_equal(sim[0]["bits"], ref)
            want = np.zeros(P, np.int64)
            for r in range(40):
                for i in order:
                    want[i] += 1
                    if not pm[r, i]:
                        break
            assert np.array_equal(sim[0]["counts"], want)
            assert np.array_equal(O.static_counts(pm, order), want)


# ------------------------------------------------------------ rank routing

def test_rank_order_minimises_expected_cost_bruteforce():
    # for independent predicates the ascending c/(1-s) order is optimal
    g = np.random.default_rng(11)
    for trial in range(200):
        P = int(g.integers(2, 7))
        c = [int(v) for v in g.integers(1, 1000, P)]
        s = [Fraction(int(v), 1000) for v in g.integers(0, 1000, P)]
        keys = [Fraction(c[i]) / (1 - s[i]) for i in range(P)]
        rank = O.order_by(keys)
        brute_order, brute_cost = O.best_order_bruteforce(c, [float(x) for x in s])
        rank_cost = O.expected_cost(rank, c, [float(x) for x in s])
        assert rank_cost <= brute_cost * (1 + 1e-12)


def test_expected_cost_definition_small():
    assert O.expected_cost([0, 1, 2], [1, 2, 4], [0.5, 0.25, 1.0]) == 1 + 0.5 * 2 + 0.5 * 0.25 * 4


def _golden():
    with open(os.path.join(GOLDEN, "paper_routing_examples.json")) as f:
        return json.load(f)


def test_paper_worked_example():
    ex = _golden()["worked_example"]
    c = [Fraction(v) for v in ex["cost"]]
    s = [Fraction(v) for v in ex["selectivity"]]
    rank = [c[i] / (1 - s[i]) for i in range(2)]
    assert rank == [Fraction(v) for v in ex["rank"]]
    names = ex["names"]
    assert names[O.order_by(rank)[0]] == ex["score_driven_first"]
    assert names[O.order_by(s)[0]] == ex["selectivity_driven_first"]
    assert names[O.order_by(c)[0]] == ex["cost_driven_first"]
    n = ex["units"]
    breed, color = 1, 0
    assert n * O.expected_cost([breed, color], c, s) == ex["sequential_time_breed_first"]
    assert n * O.expected_cost([color, breed], c, s) == ex["sequential_time_color_first"]
    # concurrent (two resources, pipelined): the slower stage bounds the
    # makespan from below; the paper's timelines sit at or just above it
    for first, second, printed in [(breed, color, ex["concurrent_time_breed_first"]),
                                   (color, breed, ex["concurrent_time_color_first"])]:
        fluid = max(n * c[first], n * s[first] * c[second])
        assert fluid <= printed <= fluid + c[first] + c[second]


@pytest.mark.parametrize("case", ["uc1_profiled", "table1_case1", "table1_case2"])
def test_paper_policy_choices(case):
    ex = _golden()[case]
    c = [Fraction(v) for v in ex["cost"]]
    s = [Fraction(v) for v in ex["selectivity"]]
    names = ex["names"]
    assert names[O.order_by([c[i] / (1 - s[i]) for i in range(2)])[0]] == ex["score_driven_first"]
    assert names[O.order_by(c)[0]] == ex["cost_driven_first"]
    assert names[O.order_by(s)[0]] == ex["selectivity_driven_first"]


def test_model_costs_closed_form():
    # 2 x multiply-adds written out for the three MLPs of the 256-d workload
    assert O.mlp_flops((256, 128, 1)) == 2 * (256 * 128 + 128) == 65792
    assert O.mlp_flops((256, 512, 512, 1)) == 787456
    assert O.mlp_flops((256, 1024, 1024, 1024, 1)) == 4720640
    assert O.cnn_flops((3, 32, 64)) == 2 * 64 * 64 * 9 * (3 * 32 + 32 * 64) + 2 * 64


def test_simulate_hand_worked_trace():
    # P=2, batches of 4, equal cost.  Predicate 1 passes 1 of 4, predicate 0 passes 3 of 4.
    pm = np.array([[1, 0], [1, 1], [1, 0], [0, 0]] * 4, bool)
    sim = O.simulate(pm, batch=4, policy="rank", costs=[10, 10], warmup=1, window=8, lag=1)
    # batch 0: warmup, every predicate sees all 4
    assert sim[0]["warmup"] and sim[0]["counts"].tolist() == [4, 4]
    # batch 1: nothing finished lag=1 batches earlier -> declared order 0,1
    assert sim[1]["order"] == [0, 1] and sim[1]["counts"].tolist() == [4, 3]
    # batch 2: sees batch 0: s0=(3+1)/(4+2)=2/3, s1=(1+1)/(4+2)=1/3 -> rank 30 vs 15 -> order 1,0
    assert sim[2]["order"] == [1, 0] and sim[2]["counts"].tolist() == [1, 4]
    # batch 3: window holds batches 0..1: e0=8,p0=6 -> s0=7/10; e1=7,p1=2 -> s1=3/9; order 1,0
    assert sim[3]["order"] == [1, 0]
    for b in sim:
        assert b["bits"].tolist() == [False, True, False, False]


def test_simulate_longer_lag_hand_worked():
    # the trace above with lag 3: batches 1..3 see no finished batch (declared
    # order); batch 4 sees batch 0 only -> order 1,0; batch 5 sees 0..1
    pm = np.array([[1, 0], [1, 1], [1, 0], [0, 0]] * 6, bool)
    sim = O.simulate(pm, batch=4, policy="rank", costs=[10, 10], warmup=1, window=8, lag=3)
    assert [b["order"] for b in sim[1:4]] == [[0, 1]] * 3
    assert all(b["counts"].tolist() == [4, 3] for b in sim[1:4])
    assert sim[4]["order"] == [1, 0] and sim[4]["counts"].tolist() == [1, 4]
    # batch 5: window = batches 0, 1: e0 = 8, p0 = 6, e1 = 7, p1 = 2 -> 10 * 10/3 > 10 * 9/6 -> 1,0
    assert sim[5]["order"] == [1, 0]


def test_simulate_window_and_fallback_to_warmup_stats():
    # predicate 1 is last and never reached after batch 1 -> its window count
    # is zero and the warmup statistics stand in
    P = 2
    pm = np.zeros((6 * 8, P), bool)
    pm[:8, 1] = True                   # warmup batch: predicate 1 passes all
    sim = O.simulate(pm, batch=8, policy="rank", costs=[1, 1000], warmup=1, window=1, lag=0)
    # batch 1 sees batch 0: s0 = 1/10, s1 = 9/10 -> rank 10/9 vs 10000 -> order 0,1
    assert sim[1]["order"] == [0, 1]
    assert sim[1]["counts"].tolist() == [8, 0]
    # batch 2 window = batch 1 only: e1 = 0 -> fall back to warmup (e1=8,p1=8)
    assert sim[2]["order"] == [0, 1]


def test_simulate_policies_order_keys():
    pm = np.ones((3 * 4, 3), bool)
    pm[:4, 2] = False
    for pol, want in [("cost", [1, 2, 0]), ("selectivity", [2, 0, 1]), ("static", [2, 1, 0])]:
        sim = O.simulate(pm, batch=4, policy=pol, costs=[30, 10, 20], static_order=[2, 1, 0], lag=0)
        assert sim[2]["order"] == want
    sim = O.simulate(pm, batch=4, policy="all")
    assert all(b["counts"].tolist() == [4, 4, 4] for b in sim)


def test_simulate_reuse_hand_worked_trace():
    # predicates 0 and 1 share an upstream UDF "E" (cost 100) under heads of
    # cost 1; predicate 2 costs 50 and shares nothing.  Every tuple passes.
    pm = np.ones((12, 3), bool)
    kw = dict(batch=4, policy="rank", costs=[1, 1, 50], groups=["E", "E", None], group_costs={"E": 100},
              ids=np.arange(12), warmup=1, lag=1, window=8)
    sim = O.simulate(pm, prefilled=[4, 5], **kw)
    # batch 0 (warmup, declared order): predicate 0 computes E for ids 0..3, predicate 1 reuses them
    assert sim[0]["hits"].tolist() == [0, 4, 0]
    # batch 1 (nothing visible yet: declared order): ids 4, 5 were prefilled
    assert sim[1]["order"] == [0, 1, 2] and sim[1]["hits"].tolist() == [2, 4, 0]
    # batch 2: s = 5/6 everywhere; ids 8..11 miss -> cost(0) = cost(1) = 1 + 4/4*100 = 101 > 50
    assert sim[2]["order"] == [2, 0, 1] and sim[2]["hits"].tolist() == [0, 4, 0]
    # the same stream with batch 2's ids prefilled: the heads cost 1 < 50
    sim = O.simulate(pm, prefilled=[8, 9, 10, 11], **kw)
    assert sim[2]["order"] == [0, 1, 2] and sim[2]["hits"].tolist() == [4, 4, 0]


def test_simulate_reuse_later_head_is_cheap():
    # heads 0 and 1 share "E" (cost 100) under own costs 1 and 30; predicate 2
    # costs 110; every tuple passes, so the rank keys are proportional to the
    # costs.  Batch 2 misses all 4 ids: head 0 = 101 goes first; head 1 then
    # costs 30 (its tuples are cached by head 0) < 110.  Ranking the heads
    # with the surcharge both ways would give 0, 2, 1 (101 < 110 < 130).
    pm = np.ones((12, 3), bool)
    sim = O.simulate(pm, batch=4, policy="rank", costs=[1, 30, 110], groups=["E", "E", None],
                     group_costs={"E": 100}, ids=np.arange(12), warmup=1, lag=1, window=8)
    assert sim[2]["order"] == [0, 1, 2] and sim[2]["hits"].tolist() == [0, 4, 0]
    # cost policy: the same keys without the selectivity factor
    sim = O.simulate(pm, batch=4, policy="cost", costs=[1, 30, 110], groups=["E", "E", None],
                     group_costs={"E": 100}, ids=np.arange(12), warmup=1, lag=1, window=8)
    assert sim[2]["order"] == [0, 1, 2]


def test_simulate_reuse_matches_plain_counts():
    # reuse changes costs and hits, never the pass set or which tuples reach a predicate
    g = np.random.default_rng(12)
    pm = g.random((64, 3)) < 0.6
    plain = O.simulate(pm, 8, policy="static", static_order=[1, 0, 2])
    reuse = O.simulate(pm, 8, policy="static", static_order=[1, 0, 2], groups=["E", "E", None],
                       group_costs={"E": 7}, ids=np.arange(64))
    for a, b in zip(plain, reuse):
        assert np.array_equal(a["bits"], b["bits"]) and a["counts"].tolist() == b["counts"].tolist()
        # predicate 0 runs after predicate 1 (same group) on a subset of its tuples: all hits
        assert b["hits"][0] == b["counts"][0]


def test_concurrent_worked_example_color_first():
    # Sec. 4.1 "Example comparison": color (cost 1, s 0.6) then breed (cost 2):
    # 10 units of color, six survivors to breed -> 14 time units
    ex = _golden()["worked_example"]
    assert O.concurrent_makespan([0, 1], [1, 2], [0.6, 0.1], 10) == ex["concurrent_time_color_first"]
    # breed first: the breed resource alone needs 20 units
    assert O.fluid_makespan([1, 0], [1, 2], [0.6, 0.1], 10) == ex["concurrent_time_breed_first"]
    assert O.concurrent_makespan([1, 0], [1, 2], [0.6, 0.1], 10) >= 20


def test_synthetic_sweep_claims():
    # Sec. 4.2 "Sensitive Analysis using Synthetic Queries": A costs 10, B 20;
    # s_B in {0.1, 0.5, 0.9}, s_A from 0.1 to 0.9.  Under concurrency the
    # cost-driven order (A first) is never slower than score- or
    # selectivity-driven, and selectivity-driven is the worst on average.
    c = [10, 20]
    totals = {"cost": 0.0, "score": 0.0, "selectivity": 0.0}
    for sB in (0.1, 0.5, 0.9):
        for sA in [k / 10 for k in range(1, 10)]:
            s = [sA, sB]
            orders = {"cost": O.order_by([Fraction(10), Fraction(20)]),
                      "score": O.order_by([Fraction(10) / (1 - Fraction(sA).limit_denominator(10)),
                                           Fraction(20) / (1 - Fraction(sB).limit_denominator(10))]),
                      "selectivity": O.order_by([Fraction(sA).limit_denominator(10), Fraction(sB).limit_denominator(10)])}
            t = {k: O.concurrent_makespan(o, c, s, 100) for k, o in orders.items()}
            assert t["cost"] <= t["score"] and t["cost"] <= t["selectivity"]
            for k in totals:
                totals[k] += t[k]
    assert totals["selectivity"] >= totals["score"] >= totals["cost"]
