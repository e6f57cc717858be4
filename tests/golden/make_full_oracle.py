"""Write the oracle's pass matrix of a whole benchmarked stream.

For every tuple of the workload's stream and every predicate, the FP64
oracle score is compared with the stored threshold (``<name>_thresholds.json``,
itself written by ``make_thresholds.py`` from the oracle):
pass = score > threshold (Sec. 1, the conjunction of Listing 1; the test is
strict).  The result is the [n, P] pass matrix the full-size parity tests and
the bench's exact-pass-set check compare with, and from which the best
static order of the stream is found by brute force (Sec. 4.2 "System
Variants", "Best Reordering").  Calls only ``oracle`` and ``datagen``.

Output ``<name>_oracle.npz``:
  * single-stream workloads: ``pm`` = np.packbits(pass matrix [n, P] in
    row-major order, bitorder="little"), ``n``, ``P``, ``thresholds``; the
    frame workload adds ``scores_f32`` = the FP64 scores rounded to fp32
    (its oracle takes hours; the pass bits come from the FP64 scores);
  * the many-query workload: per query ``pm_<q>`` packed the same way with
    ``n_<q>`` and ``P_<q>``;
  * the synthetic two-predicate workload: ``pm`` at its own selectivities
    plus ``pm_A`` / ``pm_B``, every threshold of each predicate's
    selectivity grid.

The frame workload is computed in chunks whose scores are kept under
``tests/golden/.partial/`` (not committed) so that an interrupted run
resumes where it stopped.

    python tests/golden/make_full_oracle.py [workload ...] [--threads N]
"""
import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import datagen as D  # noqa: E402
import oracle as O  # noqa: E402

PARTIAL = os.path.join(HERE, ".partial")
CHUNK = 1024


def _thresholds(name):
    with open(os.path.join(HERE, f"{name}_thresholds.json")) as f:
        return json.load(f)["thresholds"]


def _pack(pm):
    return np.packbits(np.asarray(pm, bool).reshape(-1), bitorder="little")


def single_stream(name, threads):
    w = D.workload(name)
    th = _thresholds(name)
    udfs = D.predicate_weights(w)
    t0 = time.time()
    extra = {}
    if w.kind == "frame":
        os.makedirs(PARTIAL, exist_ok=True)
        parts = []
        for c0 in range(0, w.n, CHUNK):
            path = os.path.join(PARTIAL, f"{name}_{c0:08d}.npy")
            if os.path.exists(path):
                S = np.load(path)
            else:
                F = D.blob_frames(w, 1, min(CHUNK, w.n - c0), start=c0)
                S = O.udf_scores(w.kind, F, udfs, threads)
                np.save(path + ".tmp.npy", S)
                os.replace(path + ".tmp.npy", path)
                print(f"{name}: frames {c0}..{c0 + S.shape[0]} done, {time.time() - t0:.0f} s", flush=True)
            parts.append(S)
        S = np.concatenate(parts)
        extra["scores_f32"] = S.astype(np.float32)
    else:
        S = O.udf_scores(w.kind, D.stream_tuples(w), udfs, threads)
    pm = O.pass_matrix(S, th)
    secs = time.time() - t0
    np.savez_compressed(os.path.join(HERE, f"{name}_oracle.npz"), pm=_pack(pm), n=w.n, P=len(th),
                        thresholds=np.asarray(th, np.float64), oracle_seconds=secs,
                        oracle_threads=threads or O.threads(), **extra)
    print(name, "pass fraction per predicate", pm.mean(axis=0).round(4).tolist(),
          "conjunction", float(O.result_bits(pm).mean()), f"{secs:.0f} s", flush=True)


def grid_stream(name, threads):
    """Synthetic two-predicate workload: the FP64 scores of A and B on the
    whole stream against every threshold of their selectivity grids;
    ``pm_A`` [n, |grid A|] and ``pm_B`` [n, |grid B|] packed like ``pm``
    (``pm`` itself at the workload's own pair of selectivities)."""
    w = D.workload(name)
    with open(os.path.join(HERE, f"{name}_thresholds.json")) as f:
        G = json.load(f)
    t0 = time.time()
    S = O.udf_scores(w.kind, D.stream_tuples(w), D.predicate_weights(w), threads)
    out = {}
    for i, key in enumerate(("A", "B")):
        th = [G[key][f"{s:.1f}"] for s in w.extra[f"sel_{key}"]]
        pm = S[:, i:i + 1] > np.asarray(th, np.float64)[None, :]
        out[f"pm_{key}"] = _pack(pm)
        out[f"P_{key}"] = len(th)
        out[f"sel_{key}"] = np.asarray(w.extra[f"sel_{key}"], np.float64)
    pm = O.pass_matrix(S, G["thresholds"])
    np.savez_compressed(os.path.join(HERE, f"{name}_oracle.npz"), pm=_pack(pm), n=w.n, P=2,
                        thresholds=np.asarray(G["thresholds"], np.float64), oracle_seconds=time.time() - t0,
                        oracle_threads=threads or O.threads(), **out)
    print(name, "pass fraction", pm.mean(axis=0).round(4).tolist(), f"{time.time() - t0:.0f} s", flush=True)


def many_queries(name, threads):
    w = D.workload(name)
    th = _thresholds(name)
    qs = D.mq_queries(w)
    pool = D.mq_pool_weights(w)
    t0 = time.time()
    out = {}
    for q, Q in enumerate(qs):
        S = O.udf_scores("vec", D.mq_tuples(w, q, queries=qs), [pool[u] for u in Q["udfs"]], threads)
        pm = O.pass_matrix(S, th[q])
        out[f"pm_{q}"] = _pack(pm)
        out[f"n_{q}"] = pm.shape[0]
        out[f"P_{q}"] = pm.shape[1]
        print(f"{name}: query {q} ({pm.shape[0]} x {pm.shape[1]}) {time.time() - t0:.0f} s", flush=True)
    np.savez_compressed(os.path.join(HERE, f"{name}_oracle.npz"), queries=len(qs),
                        oracle_seconds=time.time() - t0, oracle_threads=threads or O.threads(), **out)


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("names", nargs="*", default=["mlp3", "uc1", "drift6", "drift5", "mq64", "cnn4"])
    ap.add_argument("--threads", type=int, default=0)
    a = ap.parse_args()
    for nm in a.names:
        w = D.workload(nm)
        if w.extra and "queries" in w.extra:
            many_queries(nm, a.threads)
        elif w.extra and "sel_A" in w.extra:
            grid_stream(nm, a.threads)
        else:
            single_stream(nm, a.threads)
