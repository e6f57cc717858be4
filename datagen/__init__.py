"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module only draws random numbers and lays them out: tuples, tuple ids,
UDF weights and the workload shapes.  It holds none of the method's
arithmetic (no UDF evaluation, no thresholds, no routing); thresholds are
derived from UDF scores by whichever side evaluates them.

Every stream is a counter-based Philox generator (numpy's
``np.random.Philox``) keyed by ``workload_id * 1000 + stream``.  Frame
pixels use integer arithmetic only, so the bytes are the same on every host
CPU.

Workloads (the paper's data are unavailable, Sec. 4.2 / 4.4; these stand in
for them with the shapes of the build's five configurations):

* ``mlp3``  - 4,096 x 256 fp32 tuples from an 8-cluster Gaussian mixture,
  three MLP UDFs 256-128-1, 256-512-512-1, 256-1024-1024-1024-1, target
  selectivities 0.5/0.2/0.8 on a 1,024-tuple calibration draw, batches of 256.
* ``cnn4``  - 65,536 frames of 3x64x64 uint8 (Gaussian-like blobs on noise),
  four CNN UDFs with 2/4/6/8 conv3x3 layers of 32-128 channels + global
  average pool + linear, target selectivities 0.3/0.6/0.1/0.9, batches of
  2,048.
* ``drift5`` - 1,048,576 x 512 fp32 tuples in 8 segments whose 8-cluster
  mixture weights are drawn from Dirichlet(0.5) per segment (so each
  predicate's selectivity drifts between segments); five MLP UDFs, the first
  two sharing an upstream embedding 512-1024-256 (heads 256-1 and 256-256-1),
  then 512-256-1, 512-1024-1024-1, 512-2048-1; batches of 4,096.
* ``drift6`` - the same drifting stream under six MLPs 512-h-1, h = 64 ... 2048
  (costs 1:2:4:8:16:32), for per-tuple routing by a learned proxy.
* ``uc1`` - 262,144 x 512 fp32 tuples from one isotropic Gaussian and two
  synthetic-cost MLP predicates, A = 512-1024-1 and B = 512-2048-1 (cost ratio
  1:2), with thresholds for a grid of selectivities of each, for the
  concurrent-worker (pipeline) experiments.
* ``mq64`` - 64 concurrent queries over 512-dim fp32 tuples: query q has a
  lognormal tuple count (median 20,000, clipped to 1,000 ... 200,000), its
  own Dirichlet(0.5) cluster mixture, and a conjunction of 2-6 distinct UDFs
  drawn from one shared pool of eight MLPs (hidden widths 256 ... 2048) with
  per-slot target selectivities uniform in [0.2, 0.9]; each query is routed
  in chunks of 4,096 of its own tuples.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "rng", "Workload", "WORKLOADS", "workload", "gmm_tuples", "blob_frames",
    "mlp_weights", "cnn_weights", "tuple_ids", "predicate_weights",
    "stream_tuples", "calib_tuples", "embedding_weights", "head_weights", "segment_mixes",
    "mq_queries", "mq_pool_weights", "mq_tuples", "mq_calib_tuples", "mq_stacked_step",
]


def rng(workload_id: int, stream: int) -> np.random.Generator:
    """Philox stream ``workload_id*1000 + stream``."""
    return np.random.Generator(np.random.Philox(key=workload_id * 1000 + stream))


@dataclass(frozen=True)
class Workload:
    name: str
    wid: int                      # workload id used in the seeds
    kind: str                     # "vec" (fp32 feature rows) or "frame" (uint8 CHW)
    n: int                        # stream tuples
    batch: int                    # routing batch size
    udfs: tuple                   # per predicate: MLP widths or CNN channel chain
    selectivity: tuple            # target pass fraction on the calibration draw
    n_calib: int                  # calibration draw size
    dim: int = 0                  # vec: feature dim
    frame: tuple = (3, 64, 64)    # frame: C, H, W
    n_clusters: int = 8
    cluster_spread: float = 3.0
    head_gain: tuple = ()         # per predicate scale of the last layer (default 1)
    extra: dict = field(default_factory=dict)


WORKLOADS = {
    "mlp3": Workload(
        name="mlp3", wid=1, kind="vec", n=4096, batch=256, dim=256,
        udfs=((256, 128, 1), (256, 512, 512, 1), (256, 1024, 1024, 1024, 1)),
        selectivity=(0.5, 0.2, 0.8), n_calib=1024),
    "cnn4": Workload(
        name="cnn4", wid=2, kind="frame", n=65536, batch=2048,
        udfs=((3, 32, 64), (3, 32, 64, 64, 128), (3, 32, 64, 64, 128, 128, 128),
              (3, 32, 64, 64, 128, 128, 128, 128, 128)),
        selectivity=(0.3, 0.6, 0.1, 0.9), n_calib=256, head_gain=(8.0, 8.0, 6.0, 4.0)),
    "drift5": Workload(
        name="drift5", wid=3, kind="vec", n=1048576, batch=4096, dim=512,
        udfs=((512, 1024, 256, 1), (512, 1024, 256, 256, 1), (512, 256, 1), (512, 1024, 1024, 1), (512, 2048, 1)),
        selectivity=(0.5, 0.4, 0.5, 0.6, 0.5), n_calib=1024,
        extra={"segments": 8, "dirichlet": 0.5, "embedding": (512, 1024, 256), "emb_preds": (0, 1)}),
    # the same drifting stream (workload id 3, same streams) under six MLPs
    # 512-h-1 with h = 64 * 2^k, so costs grow 1:2:4:8:16:32
    "drift6": Workload(
        name="drift6", wid=3, kind="vec", n=1048576, batch=4096, dim=512,
        udfs=tuple((512, 64 << k, 1) for k in range(6)),
        selectivity=(0.6, 0.5, 0.4, 0.5, 0.3, 0.5), n_calib=1024,
        extra={"segments": 8, "dirichlet": 0.5, "weight_stream": 40, "proxy_hidden": 64, "refresh": 16}),
    # two synthetic-cost predicates for the concurrent-worker experiments: A = 512-1024-1 and
    # B = 512-2048-1 (cost ratio 1:2), tuples from one isotropic Gaussian, thresholds for each
    # selectivity of the grids below (Sec. 4.1 "Example comparison", "Sensitive Analysis
    # using Synthetic Queries")
    "uc1": Workload(
        name="uc1", wid=6, kind="vec", n=262144, batch=4096, dim=512,
        udfs=((512, 1024, 1), (512, 2048, 1)), selectivity=(0.6, 0.1), n_calib=4096, n_clusters=1,
        cluster_spread=0.0,
        extra={"sel_A": (0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9), "sel_B": (0.1, 0.5, 0.9)}),
    # 64 queries over one pool of eight MLP UDFs; ``n`` caps a query's
    # tuple count, ``batch`` is the per-query chunk of one step
    "mq64": Workload(
        name="mq64", wid=5, kind="vec", n=200000, batch=4096, dim=512,
        udfs=((512, 256, 1), (512, 512, 1), (512, 1024, 1), (512, 2048, 1), (512, 512, 256, 1),
              (512, 1024, 512, 1), (512, 2048, 1024, 1), (512, 1024, 1024, 1)),
        selectivity=(), n_calib=1024,
        extra={"queries": 64, "median": 20000, "sigma": 1.0, "min_n": 1000, "min_p": 2, "max_p": 6,
               "sel_lo": 0.2, "sel_hi": 0.9, "dirichlet": 0.5}),
}


def workload(name: str, **overrides) -> Workload:
    """A workload by name; keyword overrides give reduced-size variants
    (e.g. ``n=512``) that keep every other field, so seeds stay the same."""
    w = WORKLOADS[name]
    if not overrides:
        return w
    d = dict(w.__dict__)
    d.update(overrides)
    return Workload(**d)


# ----------------------------------------------------------------- tuples

def _cluster_means(w: Workload) -> np.ndarray:
    g = rng(w.wid, 0)
    return (g.standard_normal((w.n_clusters, w.dim)) * w.cluster_spread).astype(np.float64)


ROW_BLOCK = 4096   # rows per Philox counter block of a vector stream


def gmm_tuples(w: Workload, stream: int, n: int, mix: np.ndarray | None = None) -> np.ndarray:
    """``n`` fp32 rows of an isotropic unit-variance Gaussian mixture with
    ``w.n_clusters`` components (uniform weights unless ``mix``).  Rows come
    in blocks of ``ROW_BLOCK``, each from its own Philox counter range, so
    the first n rows do not depend on how many are drawn."""
    means = _cluster_means(w)
    p = np.full(w.n_clusters, 1.0 / w.n_clusters) if mix is None else np.asarray(mix, np.float64)
    out = np.empty((n, w.dim), np.float32)
    for b0 in range(0, n, ROW_BLOCK):
        bg = np.random.Philox(key=w.wid * 1000 + stream)
        bg.advance((b0 // ROW_BLOCK) << 40)
        g = np.random.Generator(bg)
        comp = g.choice(w.n_clusters, size=ROW_BLOCK, p=p)
        x = means[comp] + g.standard_normal((ROW_BLOCK, w.dim))
        m = min(ROW_BLOCK, n - b0)
        out[b0:b0 + m] = x[:m]
    return out


FRAME_BLOCK = 256   # frames per Philox counter block of a frame stream


def _frame_block(w: Workload, stream: int, blk: int) -> np.ndarray:
    """Frames ``blk*FRAME_BLOCK ...`` of a frame stream, [FRAME_BLOCK, C, H, W]."""
    C, H, W = w.frame
    m = FRAME_BLOCK
    bg = np.random.Philox(key=w.wid * 1000 + stream)
    bg.advance(blk << 24)                    # disjoint counter range per block
    g = np.random.Generator(bg)
    noise = g.integers(0, 48, size=(m, C, H, W), dtype=np.uint8)
    active = (g.random((m, 4)) < 0.75).astype(np.float32)
    cy = g.integers(0, H, size=(m, 4)).astype(np.float32)
    cx = g.integers(0, W, size=(m, 4)).astype(np.float32)
    rad = g.integers(6, 24, size=(m, 4)).astype(np.float32)
    amp = g.integers(30, 208, size=(m, 4, C)).astype(np.float32)
    yy = np.arange(H, dtype=np.float32)[:, None]
    xx = np.arange(W, dtype=np.float32)[None, :]
    acc = noise.astype(np.float32)
    for k in range(4):
        dy = yy[None] - cy[:, k, None, None]
        dx = xx[None] - cx[:, k, None, None]
        r2 = (rad[:, k] * rad[:, k])[:, None, None]
        t = np.maximum(r2 - (dy * dy + dx * dx), np.float32(0)) / r2
        shape = (t * t)[:, None, :, :]
        acc += (amp[:, k, :] * active[:, k, None])[:, :, None, None] * shape
    return np.minimum(np.floor(acc), 255).astype(np.uint8)


def blob_frames(w: Workload, stream: int, n: int, start: int = 0) -> np.ndarray:
    """``n`` uint8 frames [n, 3, H, W] starting at frame ``start``: uniform
    noise in [0, 48) plus up to four bright blobs.  A blob of radius R centred
    at (cy, cx) adds ``amp_c * ((R^2 - d^2) / R^2)^2`` to channel c where
    d^2 < R^2 (a smooth bump); the sum is floored and clipped to 255.  Only
    IEEE add, subtract, multiply and divide are used (no transcendental calls,
    fixed summation order), so the bytes are identical on every host.

    Frames come in blocks of ``FRAME_BLOCK``, each drawn from its own Philox
    counter range, so any slice of the stream can be generated on its own."""
    C, H, W = w.frame
    out = np.empty((n, C, H, W), np.uint8)
    if n == 0:
        return out
    b0, b1 = start // FRAME_BLOCK, (start + n - 1) // FRAME_BLOCK

    def fill(blk):
        f = _frame_block(w, stream, blk)
        lo = max(start, blk * FRAME_BLOCK)
        hi = min(start + n, (blk + 1) * FRAME_BLOCK)
        out[lo - start:hi - start] = f[lo - blk * FRAME_BLOCK:hi - blk * FRAME_BLOCK]

    blocks = list(range(b0, b1 + 1))
    if len(blocks) == 1:
        fill(b0)
    else:
        with ThreadPoolExecutor(max_workers=min(len(blocks), os.cpu_count() or 1)) as ex:
            list(ex.map(fill, blocks))
    return out


def tuple_ids(n: int, start: int = 0) -> np.ndarray:
    """Dense int64 tuple ids ``start .. start+n-1``."""
    return np.arange(start, start + n, dtype=np.int64)


# ----------------------------------------------------------------- weights

def _gain(w: Workload, pred: int) -> float:
    return float(w.head_gain[pred]) if pred < len(w.head_gain) else 1.0


def mlp_weights(w: Workload, stream: int, dims, gain: float = 1.0) -> list:
    """Per linear layer (W [out, in] fp32, b [out] fp32).  Hidden layers use a
    He-uniform bound sqrt(6/fan_in) (keeps activations' second moment through
    ReLU); biases and the last layer use 1/sqrt(fan_in), the last layer scaled
    by ``gain``."""
    g = rng(w.wid, stream)
    layers = []
    for l in range(len(dims) - 1):
        fi, fo = dims[l], dims[l + 1]
        last = l == len(dims) - 2
        bound = (1.0 / math.sqrt(fi)) * gain if last else math.sqrt(6.0 / fi)
        W = ((g.random((fo, fi)) * 2.0 - 1.0) * bound).astype(np.float32)
        b = ((g.random(fo) * 2.0 - 1.0) / math.sqrt(fi)).astype(np.float32)
        layers.append((np.ascontiguousarray(W), b))
    return layers


def cnn_weights(w: Workload, stream: int, chans, gain: float = 1.0) -> tuple:
    """Conv layers (W [Cout, Cin, 3, 3] fp32, b [Cout] fp32), He-uniform with
    fan_in = 9*Cin, then the head (w [C_last] fp32, b float).  Head weights are
    drawn from U(0, gain/sqrt(C_last)): non-negative, so the score follows the
    frame content that all pooled channels share instead of cancelling it (a
    zero-mean head leaves the deep UDFs with a score spread close to BF16
    rounding error)."""
    g = rng(w.wid, stream)
    convs = []
    for l in range(len(chans) - 1):
        ci, co = chans[l], chans[l + 1]
        fi = 9 * ci
        W = ((g.random((co, ci, 3, 3)) * 2.0 - 1.0) * math.sqrt(6.0 / fi)).astype(np.float32)
        b = ((g.random(co) * 2.0 - 1.0) / math.sqrt(fi)).astype(np.float32)
        convs.append((np.ascontiguousarray(W), b))
    C = chans[-1]
    hw = (g.random(C) * (gain / math.sqrt(C))).astype(np.float32)
    hb = np.float32((g.random() * 2.0 - 1.0) / math.sqrt(C))
    return convs, (hw, float(hb))


def embedding_weights(w: Workload):
    """Layers of the shared upstream embedding (stream 30): hidden layers
    only, so every layer is followed by ReLU; None if the workload has none."""
    dims = w.extra.get("embedding") if w.extra else None
    if not dims:
        return None
    g = rng(w.wid, 30)
    layers = []
    for l in range(len(dims) - 1):
        fi, fo = dims[l], dims[l + 1]
        W = ((g.random((fo, fi)) * 2.0 - 1.0) * math.sqrt(6.0 / fi)).astype(np.float32)
        b = ((g.random(fo) * 2.0 - 1.0) / math.sqrt(fi)).astype(np.float32)
        layers.append((np.ascontiguousarray(W), b))
    return layers


def head_weights(w: Workload, i: int):
    """Head layers of predicate i on top of the embedding (stream 10+i)."""
    emb = w.extra["embedding"]
    head_dims = w.udfs[i][len(emb) - 1:]
    return mlp_weights(w, 10 + i, head_dims, _gain(w, i))


def predicate_weights(w: Workload):
    """Full layer lists of every predicate, predicate i on stream 10+i.  A
    predicate on the shared embedding is the embedding's layers followed by
    its head's layers (one plain MLP)."""
    if w.kind == "vec":
        shared = set(w.extra.get("emb_preds", ())) if w.extra else set()
        emb = embedding_weights(w) if shared else None
        base = w.extra.get("weight_stream", 10) if w.extra else 10
        return [emb + head_weights(w, i) if i in shared else mlp_weights(w, base + i, d, _gain(w, i))
                for i, d in enumerate(w.udfs)]
    return [cnn_weights(w, 10 + i, c, _gain(w, i)) for i, c in enumerate(w.udfs)]


def segment_mixes(w: Workload) -> np.ndarray:
    """[segments, clusters] mixture weights, one Dirichlet(alpha) draw per
    segment (stream 5)."""
    S = max(w.extra["segments"], 64)
    g = rng(w.wid, 5)
    return g.dirichlet(np.full(w.n_clusters, w.extra["dirichlet"]), size=S)


def stream_tuples(w: Workload, n: int | None = None, start: int = 0) -> np.ndarray:
    """The workload's tuple stream (stream 1); frames may be sliced by
    ``start``.  A drifting stream is cut into ``segments`` equal segments,
    segment s drawn from its own mixture (``segment_mixes``) on stream 100+s;
    its prefix of n tuples is the first n tuples of that full stream."""
    n = w.n if n is None else n
    if w.kind == "vec" and w.extra and "segments" in w.extra:
        assert start == 0
        S = w.extra["segments"]
        seg = w.extra.get("segment_len") or (WORKLOADS[w.name].n // S if w.name in WORKLOADS else w.n // S)
        S = max(S, -(-n // seg))
        mixes = segment_mixes(w)
        parts, left = [], n
        for s in range(S):
            if left <= 0:
                break
            m = min(seg, left)
            parts.append(gmm_tuples(w, 100 + s, m, mixes[s]))
            left -= m
        return np.ascontiguousarray(np.concatenate(parts)) if parts else np.zeros((0, w.dim), np.float32)
    if w.kind == "vec":
        assert start == 0
        return gmm_tuples(w, 1, n)
    return blob_frames(w, 1, n, start=start)


def calib_tuples(w: Workload) -> np.ndarray:
    """The calibration draw (stream 2), independent of the stream tuples."""
    if w.kind == "vec":
        return gmm_tuples(w, 2, w.n_calib)
    return blob_frames(w, 2, w.n_calib)


# ----------------------------------------------------------------- many queries

def mq_queries(w: Workload) -> list:
    """The concurrent queries of a pool workload (stream 6): per query its
    tuple count ``n``, pool UDF ids ``udfs`` (distinct, in slot order),
    target selectivities ``selectivity`` per slot and cluster mixture ``mix``."""
    e = w.extra
    g = rng(w.wid, 6)
    out = []
    for _ in range(e["queries"]):
        n = int(round(e["median"] * math.exp(e["sigma"] * g.standard_normal())))
        n = min(max(n, e["min_n"]), w.n)
        P = int(g.integers(e["min_p"], e["max_p"] + 1))
        udfs = [int(u) for u in g.permutation(len(w.udfs))[:P]]
        sel = [float(v) for v in g.uniform(e["sel_lo"], e["sel_hi"], size=P)]
        mix = g.dirichlet(np.full(w.n_clusters, e["dirichlet"]))
        out.append(dict(n=n, udfs=udfs, selectivity=sel, mix=mix))
    return out


def mq_pool_weights(w: Workload) -> list:
    """Layers of every pool UDF, UDF u on stream 10+u."""
    return [mlp_weights(w, 10 + u, d) for u, d in enumerate(w.udfs)]


def mq_tuples(w: Workload, q: int, n: int | None = None, queries=None) -> np.ndarray:
    """Query q's tuple stream (stream 100+q), its first ``n`` tuples."""
    qs = mq_queries(w) if queries is None else queries
    n = qs[q]["n"] if n is None else n
    return gmm_tuples(w, 100 + q, n, qs[q]["mix"])


def mq_calib_tuples(w: Workload, q: int, queries=None) -> np.ndarray:
    """Query q's calibration draw (stream 400+q), from its own mixture."""
    qs = mq_queries(w) if queries is None else queries
    return gmm_tuples(w, 400 + q, w.n_calib, qs[q]["mix"])


def mq_stacked_step(streams, counts_done, chunk: int):
    """One step's input: the next ``chunk`` (or fewer) tuples of every query
    stacked query after query.  Returns (stacked rows, per-query counts)."""
    parts, counts = [], []
    for q, X in enumerate(streams):
        lo = counts_done[q]
        m = max(0, min(chunk, X.shape[0] - lo))
        parts.append(X[lo:lo + m])
        counts.append(m)
    dim = streams[0].shape[1] if streams else 0
    rows = np.concatenate(parts) if parts else np.zeros((0, dim), np.float32)
    return np.ascontiguousarray(rows), counts
