"""GPU parity of multi-query sessions: many queries over one pool of MLP UDFs,
each step stacking every query's next chunk, against the oracle run per query
(each query alone, batches = its chunks, rank routing with lag 0)."""
import json
import os

import numpy as np
import pytest

import datagen as D
import oracle as O
from gpu_helpers import stored_pass_matrix

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def mq_thresholds():
    with open(os.path.join(GOLDEN, "mq64_thresholds.json")) as f:
        return json.load(f)["thresholds"]


def make_session(w, qs, th, *, precision="fp32", cap, graphs=True, autotune=True, warmup=1, window=8,
                 queries=None, policy="rank", tile_sched=None):
    import paper_2403_14902_b300 as H
    s = H.Session(dim=w.dim, max_step_tuples=cap, precision=precision, graphs=graphs, autotune=autotune,
                  warmup=warmup, window=window, policy=policy, tile_sched=tile_sched)
    for layers in D.mq_pool_weights(w):
        s.add_udf(layers)
    for q in (range(len(qs)) if queries is None else queries):
        s.add_query(qs[q]["udfs"], th[q])
    return s


def run_session(s, streams, chunk):
    """All steps until every stream is consumed; per step (counts, bits,
    per-query report)."""
    import torch

    import paper_2403_14902_b300 as H
    done = [0] * len(streams)
    out = []
    while any(done[q] < streams[q].shape[0] for q in range(len(streams))) or not out:
        rows, counts = D.mq_stacked_step(streams, done, chunk)
        Xd = torch.from_numpy(rows).cuda() if rows.shape[0] else torch.empty((0, streams[0].shape[1]), device="cuda")
        sid = s.submit(Xd, counts)
        words, per, ms = s.poll(sid)
        out.append((counts, H.bits_from_words(words, rows.shape[0]), per))
        done = [d + c for d, c in zip(done, counts)]
    return out


def oracle_per_query(w, qs, th, streams, chunk, queries, warmup=1, window=8, policy="rank"):
    pool = D.mq_pool_weights(w)
    sims = {}
    for k, q in enumerate(queries):
        Q = qs[q]
        S = O.udf_scores("vec", streams[k], [pool[u] for u in Q["udfs"]])
        pm = O.pass_matrix(S, th[q])
        costs = [O.mlp_flops(w.udfs[u]) for u in Q["udfs"]]
        sims[k] = O.simulate(pm, chunk, policy=policy, costs=costs, warmup=warmup, window=window, lag=0)
    return sims


def check_steps(res, sims, n_queries):
    batch_of = [0] * n_queries
    for counts, bits, per in res:
        off = 0
        for k in range(n_queries):
            c = counts[k]
            r = per[k]
            if c == 0:
                assert r["batch"] == -1 and r["n"] == 0
                continue
            b = batch_of[k]
            s = sims[k][b]
            assert r["batch"] == b
            assert np.array_equal(bits[off:off + c], s["bits"]), f"query {k} batch {b}: pass set"
            assert r["warmup"] == s["warmup"]
            assert r["order"] == s["order"], f"query {k} batch {b}: order {r['order']} vs {s['order']}"
            assert r["evaluated"] == s["counts"].tolist(), f"query {k} batch {b}: counts"
            assert r["passed"] == s["passed"].tolist(), f"query {k} batch {b}: passed"
            assert r["n_pass"] == int(s["bits"].sum())
            batch_of[k] += 1
            off += c
    for k in range(n_queries):
        assert batch_of[k] == len(sims[k])


@pytest.fixture(scope="module")
def small():
    """Ten queries of the 64-query workload, each cut to at most 2,500 of its
    tuples, chunks of 640: several steps, ragged tails, queries finishing at
    different steps."""
    w = D.workload("mq64")
    qs = D.mq_queries(w)
    th = mq_thresholds()
    queries = list(range(10))
    streams = [D.mq_tuples(w, q, min(qs[q]["n"], 300 + 220 * q), qs) for q in queries]
    chunk = 640
    sims = oracle_per_query(w, qs, th, streams, chunk, queries)
    calib = np.concatenate([D.mq_calib_tuples(w, q, qs)[:128] for q in queries])
    return dict(w=w, qs=qs, th=th, queries=queries, streams=streams, chunk=chunk, sims=sims, calib=calib)


@pytest.mark.parametrize("graphs", [True, False])
def test_session_fp32_exact(small, graphs):
    import torch
    s = make_session(small["w"], small["qs"], small["th"], cap=len(small["queries"]) * small["chunk"],
                     graphs=graphs, queries=small["queries"])
    s.calibrate(torch.from_numpy(small["calib"]).cuda())
    res = run_session(s, small["streams"], small["chunk"])
    check_steps(res, small["sims"], len(small["queries"]))
    s.close()


@pytest.mark.parametrize("tile_sched", ["static", "data_aware"])
@pytest.mark.parametrize("precision,graphs", [("bf16", True), ("bf16", False), ("fp8", True)])
def test_session_tile_schedulers_exact_and_balance(small, tile_sched, precision, graphs):
    """Both tile schedulers of the grouped tensor-core launches (static round
    robin; data-aware: heaviest tiles first, claimed by the CTA that is ready)
    give the oracle's orders, counts and pass sets, with and without graphs;
    the load-balance record covers the grouped launches: every CTA's busy
    time lies inside its launch's makespan."""
    import torch
    s = make_session(small["w"], small["qs"], small["th"], precision=precision,
                     cap=len(small["queries"]) * small["chunk"], graphs=graphs, queries=small["queries"],
                     tile_sched=tile_sched)
    s.calibrate(torch.from_numpy(small["calib"]).cuda())
    s.balance(True)
    res = run_session(s, small["streams"], small["chunk"])
    check_steps(res, small["sims"], len(small["queries"]))
    b = s.balance(False)
    assert b["launches"] > 0 and 0 < b["ctas"] <= 148
    assert 0 < b["busy_mean_ms"] <= b["busy_max_ms"] * (1 + 1e-9) <= b["makespan_ms"] * (1 + 1e-6)
    assert abs(sum(b["cta_busy_ms"]) - 0) > 0
    s.close()


@pytest.mark.parametrize("autotune", [True, False])
def test_session_bf16_exact(small, autotune):
    import torch
    s = make_session(small["w"], small["qs"], small["th"], precision="bf16",
                     cap=len(small["queries"]) * small["chunk"], autotune=autotune, queries=small["queries"])
    info = s.calibrate(torch.from_numpy(small["calib"]).cuda())
    for d in info:
        assert d["margin_lowp"] >= 4 * d["max_err_lowp"] > 0
        # the split-BF16 level is far closer to exact than BF16
        assert 0 < d["max_err_tf32"] < 0.02 * d["max_err_lowp"]
        assert d["margin_tf32"] >= 8 * d["max_err_tf32"]
    res = run_session(s, small["streams"], small["chunk"])
    check_steps(res, small["sims"], len(small["queries"]))
    split = sum(sum(r["recheck_split"]) for _, _, per in res for r in per)
    f32 = sum(sum(r["recheck_fp32"]) for _, _, per in res for r in per)
    assert split + f32 > 0
    if autotune:
        t = s.tuning()
        assert len(t) == sum(len(d) - 2 for d in small["w"].udfs)
        for rec in t:
            assert rec["tile_n"] in (64, 128, 256) and rec["N"] % rec["tile_n"] == 0
            assert rec["us"][rec["tile_n"].bit_length() - 7] == min(u for u in rec["us"] if u > 0)
    s.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_session_static_order_exact(small, precision):
    """Static policy: every batch of every query in its declared slot order,
    no warmup batch; counts are the pass matrix's static counts."""
    import torch
    s = make_session(small["w"], small["qs"], small["th"], precision=precision, policy="static",
                     cap=len(small["queries"]) * small["chunk"], queries=small["queries"])
    s.calibrate(torch.from_numpy(small["calib"]).cuda())
    res = run_session(s, small["streams"], small["chunk"])
    sims = oracle_per_query(small["w"], small["qs"], small["th"], small["streams"], small["chunk"],
                            small["queries"], policy="static")
    check_steps(res, sims, len(small["queries"]))
    assert not any(r["warmup"] for _, _, per in res for r in per)
    s.close()


def fp8_set(w):
    """Pool UDFs whose first hidden layer has >= 1,024 outputs (the default FP8 set)."""
    return [u for u, d in enumerate(w.udfs) if d[1] >= 1024]


@pytest.mark.parametrize("graphs", [True, False])
def test_session_fp8_exact(small, graphs):
    """FP8 first layers for the widest UDFs: level-0 errors grow, the
    calibrated margins grow with them, and the pass sets, orders and counts
    stay those of the oracle.  Only FP8-set slots reach the BF16 level."""
    import torch
    w = small["w"]
    q8 = fp8_set(w)
    assert q8 == [2, 3, 5, 6, 7]
    s = make_session(w, small["qs"], small["th"], precision="fp8", graphs=graphs,
                     cap=len(small["queries"]) * small["chunk"], queries=small["queries"])
    info = s.calibrate(torch.from_numpy(small["calib"]).cuda())
    for u, d in enumerate(info):
        assert d["margin_lowp"] >= 4 * d["max_err_lowp"] > 0
        assert d["margin_tf32"] >= 4 * d["max_err_tf32"] > 0
        if u in q8:    # level 0 in FP8, level 1 in BF16
            assert d["max_err_lowp"] > 2 * d["max_err_tf32"]
        else:          # level 0 is the BF16 path itself
            assert d["max_err_lowp"] == d["max_err_tf32"]
    res = run_session(s, small["streams"], small["chunk"])
    check_steps(res, small["sims"], len(small["queries"]))
    lv1 = 0
    for counts, _, per in res:
        for k, r in enumerate(per):
            udfs = small["qs"][small["queries"][k]]["udfs"]
            for slot, u in enumerate(udfs):
                if u not in q8:
                    assert r["recheck_split"][slot] == 0
                lv1 += r["recheck_split"][slot]
    assert lv1 > 0
    s.close()


def test_session_fp8_scores_against_oracle(small):
    """Level-0 scores of an FP8 session: FP8-set UDFs are further from FP64
    than their BF16 scores but within a few percent; the others are the BF16
    scores exactly."""
    import torch
    w = small["w"]
    s = make_session(w, small["qs"], small["th"], precision="fp8", cap=1000, queries=small["queries"])
    X = small["streams"][3][:1000]
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    o8 = torch.empty(X.shape[0], dtype=torch.float64, device="cuda")
    o16 = torch.empty_like(o8)
    pool = D.mq_pool_weights(w)
    for u in range(8):
        S = O.udf_scores("vec", X, [pool[u]])[:, 0]
        rms = np.sqrt((S ** 2).mean())
        s.udf_scores(u, "fp8", Xd, o8)
        s.udf_scores(u, "bf16", Xd, o16)
        r8 = np.abs(o8.cpu().numpy() - S) / np.maximum(np.abs(S), rms)
        r16 = np.abs(o16.cpu().numpy() - S) / np.maximum(np.abs(S), rms)
        if u in fp8_set(w):
            assert np.median(r16) < np.median(r8) < 5e-2, (u, np.median(r8), np.median(r16))
        else:
            assert torch.equal(o8, o16)
    s.close()


def test_session_wide_margins_recheck_everything(small):
    import torch
    s = make_session(small["w"], small["qs"], small["th"], precision="bf16",
                     cap=len(small["queries"]) * small["chunk"], queries=small["queries"])
    s.calibrate(torch.from_numpy(small["calib"]).cuda())
    for u in range(8):
        s.set_margins(u, 1e3, 1e3, 1e3)
    res = run_session(s, small["streams"], small["chunk"])
    check_steps(res, small["sims"], len(small["queries"]))
    ev = sum(sum(r["evaluated"]) for _, _, per in res for r in per)
    for key in ("recheck_fp32", "recheck_fp64"):
        assert sum(sum(r[key]) for _, _, per in res for r in per) == ev
    # the split level ran on the rounds whose band reached its minimum size
    split = sum(sum(r["recheck_split"]) for _, _, per in res for r in per)
    assert 6400 <= split < ev
    s.close()


def test_session_fp64_band_beyond_layer_parallel_capacity(small):
    """FP32 session, every score sent to FP64, chunks of 1,024: the first
    round's FP64 band (8,664 entries) exceeds the 8,192 entries run layer-
    parallel; the rest run a block per entry.  Still exact."""
    import torch
    chunk = 1024
    s = make_session(small["w"], small["qs"], small["th"], cap=len(small["queries"]) * chunk,
                     queries=small["queries"])
    for u in range(8):
        s.set_margins(u, 0.0, 0.0, 1e3)
    res = run_session(s, small["streams"], chunk)
    sims = oracle_per_query(small["w"], small["qs"], small["th"], small["streams"], chunk, small["queries"])
    check_steps(res, sims, len(small["queries"]))
    assert sum(res[0][0]) > 8192
    ev = sum(sum(r["evaluated"]) for _, _, per in res for r in per)
    assert sum(sum(r["recheck_fp64"]) for _, _, per in res for r in per) == ev
    s.close()


def test_session_scores_against_oracle(small):
    import torch
    w = small["w"]
    s = make_session(w, small["qs"], small["th"], precision="bf16", cap=1000, queries=small["queries"])
    X = small["streams"][3][:1000]
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    out = torch.empty(X.shape[0], dtype=torch.float64, device="cuda")
    pool = D.mq_pool_weights(w)
    for u in range(8):
        S = O.udf_scores("vec", X, [pool[u]])[:, 0]
        rms = np.sqrt((S ** 2).mean())
        s.udf_scores(u, "fp64", Xd, out)
        assert np.max(np.abs(out.cpu().numpy() - S)) <= 1e-9 * max(1.0, np.abs(S).max())
        s.udf_scores(u, "fp32", Xd, out)
        assert np.max(np.abs(out.cpu().numpy() - S) / np.maximum(np.abs(S), rms)) < 1e-3
        s.udf_scores(u, "bf16", Xd, out)
        assert np.median(np.abs(out.cpu().numpy() - S) / np.maximum(np.abs(S), rms)) < 1e-2
        s.udf_scores(u, "bf16x3", Xd, out)
        assert np.max(np.abs(out.cpu().numpy() - S) / np.maximum(np.abs(S), rms)) < 2e-4
    s.close()


def test_session_idle_queries_and_empty_step(small):
    """Steps where some queries sit out (count 0), a one-tuple chunk, and an
    empty step: the idle queries' batch numbers do not advance."""
    import torch
    w, qs, th = small["w"], small["qs"], small["th"]
    queries = [0, 1, 2]
    streams = [D.mq_tuples(w, q, 700, qs) for q in queries]
    plan = [[300, 0, 1], [0, 0, 0], [300, 300, 0], [100, 400, 299]]   # per step, per query
    s = make_session(w, qs, th, cap=1024, queries=queries)
    import paper_2403_14902_b300 as H
    done = [0, 0, 0]
    batches = [[] for _ in queries]
    for counts in plan:
        rows = np.concatenate([streams[k][done[k]:done[k] + c] for k, c in enumerate(counts)])
        Xd = torch.from_numpy(np.ascontiguousarray(rows)).cuda() if len(rows) else torch.empty((0, w.dim), device="cuda")
        sid = s.submit(Xd, counts)
        words, per, _ = s.poll(sid)
        bits = H.bits_from_words(words, len(rows))
        off = 0
        for k, c in enumerate(counts):
            if c:
                batches[k].append((c, bits[off:off + c], per[k]))
            else:
                assert per[k]["batch"] == -1
            off += c
            done[k] += c
    pool = D.mq_pool_weights(w)
    for k, q in enumerate(queries):
        X = np.concatenate([streams[k][:done[k]]])
        pm = O.pass_matrix(O.udf_scores("vec", X, [pool[u] for u in qs[q]["udfs"]]), th[q])
        costs = [O.mlp_flops(w.udfs[u]) for u in qs[q]["udfs"]]
        lo = 0
        for b, (c, bits, r) in enumerate(batches[k]):
            # the query's batches are its non-empty chunks, of varying size
            assert r["batch"] == b
            assert np.array_equal(bits, O.result_bits(pm[lo:lo + c]))
            if b == 0:
                assert r["warmup"] and r["evaluated"] == [c] * len(costs)
            else:
                assert r["evaluated"] == O.static_counts(pm[lo:lo + c], r["order"]).tolist()
            lo += c
    s.close()


def test_session_full_workload_exact():
    """All 64 queries (1.6 M tuples) in the bench's launch configuration:
    chunks of 4,096, 8 chunks of every query per step (route lag 7), BF16
    with graphs and autotuning.  Every tuple of every query, and every
    batch's order, evaluation and pass counts, equal the oracle's (its
    stored FP64 pass matrix of each query's whole stream and its router
    simulation of that query with lag 7)."""
    import torch
    import paper_2403_14902_b300 as H
    w = D.workload("mq64")
    qs = D.mq_queries(w)
    th = mq_thresholds()
    streams = [D.mq_tuples(w, q, None, qs) for q in range(len(qs))]
    chunk, K = w.batch, 8
    s = H.Session(dim=w.dim, max_step_tuples=len(qs) * chunk * K, precision="bf16", batches_per_step=K,
                  lag=K - 1)
    for layers in D.mq_pool_weights(w):
        s.add_udf(layers)
    for q in range(len(qs)):
        s.add_query(qs[q]["udfs"], th[q])
    calib = np.concatenate([D.mq_calib_tuples(w, q, qs)[:64] for q in range(len(qs))])
    s.calibrate(torch.from_numpy(calib).cuda())
    res = run_session_multi(s, streams, chunk, K)
    got = [[] for _ in qs]
    for counts, bits, per in res:
        off = 0
        for v, c in enumerate(counts):
            if c:
                got[v // K].append((bits[off:off + c], per[v]))
            off += c
    for q in range(len(qs)):
        pm = stored_pass_matrix("mq64", q)
        assert pm.shape[0] == streams[q].shape[0]
        sim = O.simulate(pm, chunk, policy="rank", costs=[O.mlp_flops(w.udfs[u]) for u in qs[q]["udfs"]],
                         lag=K - 1)
        assert len(got[q]) == len(sim), f"query {q}: batches"
        for b, ((bits, r), sm) in enumerate(zip(got[q], sim)):
            assert r["batch"] == b
            assert np.array_equal(bits, sm["bits"]), f"query {q} batch {b}: pass set"
            assert r["order"] == sm["order"], f"query {q} batch {b}: order {r['order']} vs {sm['order']}"
            assert r["evaluated"] == sm["counts"].tolist(), f"query {q} batch {b}: counts"
            assert r["passed"] == sm["passed"].tolist(), f"query {q} batch {b}: passed"
    s.close()


def test_session_graph_skips_empty_regions(small):
    """With graphs, each round and each recheck level is a conditional region
    that runs only when it has work: same results, fewer kernel launches than
    launching every kernel of every round."""
    import torch
    counts = {}
    for graphs in (True, False):
        s = make_session(small["w"], small["qs"], small["th"], precision="bf16",
                         cap=len(small["queries"]) * small["chunk"], graphs=graphs, queries=small["queries"])
        s.calibrate(torch.from_numpy(small["calib"]).cuda())
        s.profile(False)   # resets the launch counter
        res = run_session(s, small["streams"], small["chunk"])
        check_steps(res, small["sims"], len(small["queries"]))
        counts[graphs] = s.profile_read()[1]
        s.close()
    assert 0 < counts[True] < counts[False]


def run_session_multi(s, streams, chunk, K):
    """Steps of up to K consecutive chunks per query (entry q*K + k)."""
    import torch

    import paper_2403_14902_b300 as H
    done = [0] * len(streams)
    out = []
    while any(done[q] < streams[q].shape[0] for q in range(len(streams))):
        parts, counts = [], []
        for q, X in enumerate(streams):
            for k in range(K):
                lo = done[q]
                m = max(0, min(chunk, X.shape[0] - lo))
                parts.append(X[lo:lo + m])
                counts.append(m)
                done[q] += m
        rows = np.ascontiguousarray(np.concatenate(parts))
        sid = s.submit(torch.from_numpy(rows).cuda(), counts)
        words, per, _ = s.poll(sid)
        out.append((counts, H.bits_from_words(words, rows.shape[0]), per))
    return out


@pytest.mark.parametrize("K,lag,precision", [(2, 1, "bf16"), (3, 2, "fp32"), (2, 3, "bf16"), (16, 15, "bf16"),
                                              (4, 3, "fp8"), (32, 31, "bf16")])
def test_session_several_batches_per_step(small, K, lag, precision):
    """Each step holds up to K consecutive batches of every query, routed with
    lag >= K - 1: orders, counts and pass sets equal the oracle's per-query
    simulation with that lag."""
    import torch

    import paper_2403_14902_b300 as H
    w, qs, th = small["w"], small["qs"], small["th"]
    chunk = 320
    s = H.Session(dim=w.dim, max_step_tuples=len(small["queries"]) * chunk * K, precision=precision,
                  batches_per_step=K, lag=lag)
    for layers in D.mq_pool_weights(w):
        s.add_udf(layers)
    for q in small["queries"]:
        s.add_query(qs[q]["udfs"], th[q])
    s.calibrate(torch.from_numpy(small["calib"]).cuda())
    res = run_session_multi(s, small["streams"], chunk, K)
    pool = D.mq_pool_weights(w)
    for k, q in enumerate(small["queries"]):
        pm = O.pass_matrix(O.udf_scores("vec", small["streams"][k], [pool[u] for u in qs[q]["udfs"]]), th[q])
        sim = O.simulate(pm, chunk, policy="rank", costs=[O.mlp_flops(w.udfs[u]) for u in qs[q]["udfs"]], lag=lag)
        b = 0
        for counts, bits, per in res:
            off = sum(counts[:k * K])
            for j in range(K):
                c = counts[k * K + j]
                r = per[k * K + j]
                if c == 0:
                    assert r["batch"] == -1
                    continue
                sm = sim[b]
                assert r["batch"] == b
                assert np.array_equal(bits[off:off + c], sm["bits"])
                assert r["order"] == sm["order"], (q, b, r["order"], sm["order"])
                assert r["evaluated"] == sm["counts"].tolist()
                assert r["passed"] == sm["passed"].tolist()
                off += c
                b += 1
        assert b == len(sim)
    s.close()
