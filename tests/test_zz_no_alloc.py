"""The allocation-free MLP scoring entry point (for callers that cannot
allocate device memory, e.g. while recording a CUDA graph) against the
query's hydro_udf_scores on the same tuples, twice in a row.  Collected last
on purpose; self-contained so it also passes alone in a fresh process."""
import numpy as np
import pytest

import datagen as D

pytestmark = pytest.mark.gpu


def _reference_and_noalloc(q, H, pred, layers, X, out_ref, out_na):
    import torch
    q.udf_scores(pred, "fp32", X, out_ref)
    Ws = [torch.from_numpy(W).cuda() for W, _ in layers]
    bs = [torch.from_numpy(b).cuda() for _, b in layers]
    H.mlp_scores_noalloc(X, Ws, bs, out_na)
    torch.cuda.synchronize()
    return out_ref.cpu().numpy(), out_na.cpu().numpy()


def test_noalloc_matches_query_scores_two_calls():
    import torch

    import paper_2403_14902_b300 as H
    w = D.workload("mlp3")
    weights = D.predicate_weights(w)
    X = torch.from_numpy(D.stream_tuples(w)).cuda()
    q = H.Query("vec", dim=w.dim, max_batch=1024)
    for layers in weights:
        q.add_mlp(layers, 0.0)
    # scale of each predicate's scores for the relative tolerance
    calls = [(2, 1000), (0, 777)]     # widest UDF first, then a narrower one on fewer rows
    for pred, n in calls:
        out_ref = torch.empty(n, dtype=torch.float64, device="cuda")
        out_na = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        ref, na = _reference_and_noalloc(q, H, pred, weights[pred], X[:n], out_ref, out_na)
        rms = float(np.sqrt((ref ** 2).mean()))
        assert np.all(np.abs(na - ref) <= 1e-3 * np.maximum(np.abs(ref), rms)), f"pred {pred}"
    q.close()


def test_noalloc_rejects_oversized_input():
    import torch

    import paper_2403_14902_b300 as H
    w = D.workload("mlp3")
    layers = D.predicate_weights(w)[2]          # hidden width 1024
    X = torch.zeros((1025, w.dim), dtype=torch.float32, device="cuda")   # 1025 * 1024 > 1,048,576
    Ws = [torch.from_numpy(W).cuda() for W, _ in layers]
    bs = [torch.from_numpy(b).cuda() for _, b in layers]
    out = torch.empty(1025, dtype=torch.float64, device="cuda")
    with pytest.raises(H.HydroError) as e:
        H.mlp_scores_noalloc(X, Ws, bs, out)
    assert e.value.status == H.EINVAL and "static scratch" in str(e.value)
