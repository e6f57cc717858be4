"""Write the predicate thresholds of the seeded workloads.

Each threshold is the midpoint that leaves exactly round(s * n_calib) of the
calibration draw's FP64 oracle scores above it (s = the workload's target
selectivity).  Calls only ``oracle`` and ``datagen``.

    python tests/golden/make_thresholds.py [workload ...]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import datagen as D  # noqa: E402
import oracle as O  # noqa: E402


def mq_thresholds(name: str) -> dict:
    """Per query and slot: the threshold leaving the slot's target
    selectivity of the query's own calibration draw above it."""
    w = D.workload(name)
    t0 = time.time()
    qs = D.mq_queries(w)
    pool = D.mq_pool_weights(w)
    th = []
    for q, Q in enumerate(qs):
        S = O.udf_scores("vec", D.mq_calib_tuples(w, q, qs), [pool[u] for u in Q["udfs"]])
        th.append([O.threshold_for_selectivity(S[:, k], s) for k, s in enumerate(Q["selectivity"])])
    return {"workload": name, "n_calib": w.n_calib, "thresholds": th, "oracle_seconds": round(time.time() - t0, 1),
            "oracle_threads": O.threads()}


def grid_thresholds(name: str) -> dict:
    """Per predicate (A, B), the threshold of every selectivity of its grid
    on the calibration draw; ``thresholds`` holds the pair at the workload's
    own selectivities."""
    w = D.workload(name)
    t0 = time.time()
    S = O.udf_scores(w.kind, D.calib_tuples(w), D.predicate_weights(w))
    out = {"workload": name, "n_calib": w.n_calib}
    for i, key in enumerate(("A", "B")):
        out[key] = {f"{s:.1f}": O.threshold_for_selectivity(S[:, i], s) for s in w.extra[f"sel_{key}"]}
    out["selectivity"] = list(w.selectivity)
    out["thresholds"] = [O.threshold_for_selectivity(S[:, i], s) for i, s in enumerate(w.selectivity)]
    out["oracle_seconds"] = round(time.time() - t0, 1)
    out["oracle_threads"] = O.threads()
    return out


def thresholds(name: str) -> dict:
    w = D.workload(name)
    if w.extra and "queries" in w.extra:
        return mq_thresholds(name)
    if w.extra and "sel_A" in w.extra:
        return grid_thresholds(name)
    t0 = time.time()
    S = O.udf_scores(w.kind, D.calib_tuples(w), D.predicate_weights(w))
    th = [O.threshold_for_selectivity(S[:, i], s) for i, s in enumerate(w.selectivity)]
    return {"workload": name, "n_calib": w.n_calib, "selectivity": list(w.selectivity), "thresholds": th,
            "calib_score_min": S.min(axis=0).tolist(), "calib_score_max": S.max(axis=0).tolist(),
            "calib_score_std": S.std(axis=0).tolist(), "oracle_seconds": round(time.time() - t0, 1),
            "oracle_threads": O.threads()}


if __name__ == "__main__":
    names = sys.argv[1:] or ["mlp3", "cnn4"]
    for name in names:
        out = thresholds(name)
        with open(os.path.join(HERE, f"{name}_thresholds.json"), "w") as f:
            json.dump(out, f, indent=1)
        print(name, out["thresholds"], out["oracle_seconds"], "s")
