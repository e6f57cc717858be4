"""The allocation-free MLP scoring entry point, for callers that cannot
allocate device memory once they are running (a framework that owns the
device pool, a service that cannot take a cudaMalloc's synchronisation).

Each UDF is scored twice in a row through ``hydro_mlp_scores_noalloc`` and
compared with the FP64 oracle at the 1e-3 relative tolerance of the FP32
path, and with the query's own ``hydro_udf_scores`` on the same tuples.
The UDFs cover every layer count the entry point branches on: one layer
(the dot kernel only), two, three (the last layer reads the second buffer)
and four.  Collected last on purpose; self-contained so it also passes alone
in a fresh process."""
import numpy as np
import pytest

import datagen as D
import oracle as O

pytestmark = pytest.mark.gpu


def _udfs():
    """mlp3's three UDFs (2, 3 and 4 layers) and a 1-layer 256-1 MLP."""
    w = D.workload("mlp3")
    return w, D.predicate_weights(w) + [D.mlp_weights(w, 77, (w.dim, 1))]


def _tol_ok(got, s64):
    rms = float(np.sqrt((s64 ** 2).mean()))
    return np.abs(got - s64) <= 1e-3 * np.maximum(np.abs(s64), rms)


def test_noalloc_matches_oracle_and_query_scores_two_calls():
    import torch

    import paper_2403_14902_b300 as H
    w, udfs = _udfs()
    Xh = D.stream_tuples(w)
    X = torch.from_numpy(Xh).cuda()
    q = H.Query("vec", dim=w.dim, max_batch=1024)
    for layers in udfs:
        q.add_mlp(layers, 0.0)
    # widest UDF first, then the others on other row counts; every UDF twice in a row
    for pred, n in [(2, 1000), (2, 1000), (0, 777), (0, 777), (1, 1024), (1, 1024), (3, 513), (3, 513)]:
        layers = udfs[pred]
        s64 = O.mlp_scores(Xh[:n], layers)
        out_ref = torch.empty(n, dtype=torch.float64, device="cuda")
        q.udf_scores(pred, "fp32", X[:n], out_ref)
        Ws = [torch.from_numpy(W).cuda() for W, _ in layers]
        bs = [torch.from_numpy(b).cuda() for _, b in layers]
        out_na = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        H.mlp_scores_noalloc(X[:n], Ws, bs, out_na)
        torch.cuda.synchronize()
        na, ref = out_na.cpu().numpy(), out_ref.cpu().numpy()
        assert np.isfinite(na).all(), f"pred {pred}: unwritten scores"
        assert _tol_ok(na, s64).all(), f"pred {pred}: no-alloc scores vs the FP64 oracle"
        assert _tol_ok(na, ref).all(), f"pred {pred}: no-alloc scores vs hydro_udf_scores"
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


def test_noalloc_wrapper_rejects_mismatched_tensors():
    """Shapes, dtypes and strides the C entry point cannot see are refused
    by the binding before any kernel runs."""
    import torch

    import paper_2403_14902_b300 as H
    w = D.workload("mlp3")
    layers = D.predicate_weights(w)[0]          # 256-128-1
    X = torch.zeros((8, w.dim), dtype=torch.float32, device="cuda")
    Ws = [torch.from_numpy(W).cuda() for W, _ in layers]
    bs = [torch.from_numpy(b).cuda() for _, b in layers]
    out = torch.empty(8, dtype=torch.float64, device="cuda")
    bad = [
        (X, [Ws[0].t(), Ws[1]], bs, out),                                   # transposed (non-contiguous)
        (X, [Ws[0][:, :128].contiguous(), Ws[1]], bs, out),                # wrong fan-in
        (X, Ws, [bs[0][:64], bs[1]], out),                                  # short bias
        (X, Ws, bs, out.float()),                                           # float32 output
        (X, Ws, bs, out[:4]),                                               # short output
        (X.double(), Ws, bs, out),                                          # float64 tuples
        (X, [Ws[0].double(), Ws[1]], bs, out),                              # float64 weights
    ]
    for args in bad:
        with pytest.raises(ValueError):
            H.mlp_scores_noalloc(*args)
