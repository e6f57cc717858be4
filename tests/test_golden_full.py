"""The stored oracle pass matrices of the whole benchmarked streams
(``tests/golden/<workload>_oracle.npz``, written by
``tests/golden/make_full_oracle.py``) against the oracle itself on sampled
tuples, and their layout: row-major [n, P] bits, LSB first, the conjunction
of every row's bits is that tuple's result (Sec. 1, Listing 1)."""
import json
import os

import numpy as np
import pytest

import datagen as D
import oracle as O

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name, q=None):
    z = np.load(os.path.join(GOLDEN, f"{name}_oracle.npz"))
    key, kn, kp = ("pm", "n", "P") if q is None else (f"pm_{q}", f"n_{q}", f"P_{q}")
    n, P = int(z[kn]), int(z[kp])
    bits = np.unpackbits(z[key], bitorder="little")
    assert bits.size >= n * P and not bits[n * P:].any(), "padding bits must be zero"
    return z, bits[:n * P].reshape(n, P).astype(bool)


def _thresholds(name):
    with open(os.path.join(GOLDEN, f"{name}_thresholds.json")) as f:
        return json.load(f)["thresholds"]


def _present(name):
    return os.path.exists(os.path.join(GOLDEN, f"{name}_oracle.npz"))


@pytest.mark.parametrize("name,sample", [("mlp3", 4096), ("uc1", 512), ("drift5", 384), ("drift6", 384),
                                         ("cnn4", 6)])
def test_stored_pass_matrix_matches_oracle_on_sample(name, sample):
    if not _present(name):
        pytest.fail(f"{name}_oracle.npz is missing: run tests/golden/make_full_oracle.py {name}")
    w = D.workload(name)
    z, pm = _load(name)
    assert pm.shape == (w.n, len(w.udfs))
    th = _thresholds(name)
    assert np.array_equal(z["thresholds"], np.asarray(th, np.float64))
    rng = np.random.default_rng(2024)
    if w.kind == "frame":
        # frames come in independent blocks, so any frame can be drawn on its own
        idx = np.sort(rng.choice(w.n, sample, replace=False))
        F = np.concatenate([D.stream_tuples(w, 1, start=int(i)) for i in idx])
        S = O.udf_scores("frame", F, D.predicate_weights(w))
    else:
        X = D.stream_tuples(w)
        idx = np.arange(w.n) if sample >= w.n else np.sort(rng.choice(w.n, sample, replace=False))
        S = O.udf_scores("vec", X[idx], D.predicate_weights(w))
    assert np.array_equal(pm[idx], O.pass_matrix(S, th))
    # pass fractions near the calibration targets (the stream and the calibration draw differ)
    frac = pm.mean(axis=0)
    assert np.all(np.abs(frac - np.asarray(w.selectivity)) < 0.35), frac


def test_stored_mq64_pass_matrices_match_oracle_on_sample():
    if not _present("mq64"):
        pytest.fail("mq64_oracle.npz is missing: run tests/golden/make_full_oracle.py mq64")
    w = D.workload("mq64")
    qs = D.mq_queries(w)
    th = _thresholds("mq64")
    pool = D.mq_pool_weights(w)
    z = np.load(os.path.join(GOLDEN, "mq64_oracle.npz"))
    assert int(z["queries"]) == len(qs)
    for q in range(len(qs)):
        _, pm = _load("mq64", q)
        assert pm.shape == (qs[q]["n"], len(qs[q]["udfs"]))
    rng = np.random.default_rng(7)
    for q in (0, 17, 40, 63):
        _, pm = _load("mq64", q)
        X = D.mq_tuples(w, q, queries=qs)
        idx = np.sort(rng.choice(X.shape[0], 128, replace=False))
        S = O.udf_scores("vec", X[idx], [pool[u] for u in qs[q]["udfs"]])
        assert np.array_equal(pm[idx], O.pass_matrix(S, th[q])), f"query {q}"


def test_stored_uc1_grids_match_oracle_on_sample():
    """The synthetic two-predicate stream: every threshold of each
    predicate's selectivity grid, and the default pair inside the grids."""
    if not _present("uc1"):
        pytest.fail("uc1_oracle.npz is missing: run tests/golden/make_full_oracle.py uc1")
    w = D.workload("uc1")
    z, pm = _load("uc1")
    with open(os.path.join(GOLDEN, "uc1_thresholds.json")) as f:
        G = json.load(f)
    n = w.n
    grids = {}
    for i, key in enumerate(("A", "B")):
        P = int(z[f"P_{key}"])
        bits = np.unpackbits(z[f"pm_{key}"], bitorder="little")
        assert not bits[n * P:].any()
        grids[key] = bits[:n * P].reshape(n, P).astype(bool)
        sel = list(w.extra[f"sel_{key}"])
        assert np.allclose(z[f"sel_{key}"], sel)
        # a lower selectivity is a higher threshold: its passes are a subset
        frac = grids[key].mean(axis=0)
        assert np.all(np.diff(frac) > 0), frac
        assert np.array_equal(grids[key][:, sel.index(w.selectivity[i])], pm[:, i])
    rng = np.random.default_rng(5)
    idx = np.sort(rng.choice(n, 256, replace=False))
    S = O.udf_scores("vec", D.stream_tuples(w)[idx], D.predicate_weights(w))
    for i, key in enumerate(("A", "B")):
        th = np.asarray([G[key][f"{v:.1f}"] for v in w.extra[f"sel_{key}"]])
        assert np.array_equal(grids[key][idx], S[:, i:i + 1] > th[None, :])
