"""Benchmark: query tuples/sec at an exact pass set, adaptive vs static order.

Workload: the 65,536-frame stream (3x64x64 uint8, seeded Gaussian-like blobs
on noise), four random-init CNN UDF predicates (2/4/6/8 conv3x3 layers of
32-128 channels + global average pool + linear head) with target
selectivities 0.3/0.6/0.1/0.9, routing batches of 1,024, rank c/(1-s)
routing, BF16 tensor-core inference with FP32 accumulation and an FP32/FP64
recheck of every score within 0.02 of its threshold.

One step = the whole stream through the query (64 batches submitted and
polled).  Inputs (805 MB) exceed L2 (126 MB), so no flush is needed between
steps.  Printed as one JSON line on rank 0.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica of the
workload on its own GPU (the path shards by tuples with no exchange step);
value = tuples of all ranks / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import datagen as D  # noqa: E402

METRIC = "query tuples/sec at exact pass set: adaptive vs static order, same B300"
WORKLOAD = "cnn4"
PEAKS_FALLBACK = {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return dict(PEAKS_FALLBACK), "fallback"


def thresholds(name):
    with open(os.path.join(ROOT, "tests", "golden", f"{name}_thresholds.json")) as f:
        return json.load(f)["thresholds"]


# ---------------------------------------------------------------- distributed

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def dist_init(backend):
    import torch.distributed as dist
    ws, rank, _ = dist_env()
    if ws > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return ws, rank


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(x: float, device=None) -> float:
    """Max of a float over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(units_per_rank: int, steps: int, seconds_max: float, world: int) -> float:
    """Whole-job throughput: units all ranks processed / slowest rank's time."""
    return units_per_rank * steps * world / seconds_max


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, reasons)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- our arm

def build_query(H, w, th, *, policy, precision, stream, max_in_flight=8):
    q = H.Query(w.kind, frame=w.frame, max_batch=w.batch, policy=policy, precision=precision,
                max_in_flight=max_in_flight, stream=stream)
    for i, udf in enumerate(D.predicate_weights(w)):
        q.add_cnn(udf, th[i])
    return q


def run_step(q, X, batch, max_in_flight):
    """The whole stream through the query; returns total passing tuples."""
    pending, n_pass = [], 0
    for b0 in range(0, X.shape[0], batch):
        pending.append(q.submit(X[b0:b0 + batch]))
        if len(pending) >= max_in_flight:
            n_pass += q.poll(pending.pop(0))[2]["n_pass"]
    for b in pending:
        n_pass += q.poll(b)[2]["n_pass"]
    return n_pass


def run_step_host(q, Xh, bufs, batch, max_in_flight, stream):
    """End to end through the public API from pinned HOST frames: each batch
    is copied host->device on the query's stream, submitted and polled (the
    poll reads the bitmap and counts back to the host)."""
    import torch
    pending, n_pass, k = [], 0, 0
    with torch.cuda.stream(stream):
        for b0 in range(0, Xh.shape[0], batch):
            buf = bufs[k % len(bufs)]
            k += 1
            m = min(batch, Xh.shape[0] - b0)
            buf[:m].copy_(Xh[b0:b0 + m], non_blocking=True)
            pending.append(q.submit(buf[:m]))
            if len(pending) >= max_in_flight:
                n_pass += q.poll(pending.pop(0))[2]["n_pass"]
        for b in pending:
            n_pass += q.poll(b)[2]["n_pass"]
    return n_pass


def timed(fn, steps, stream, device):
    import torch
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = [fn() for _ in range(steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    return e0.elapsed_time(e1) / 1000.0, out


def cpu_baseline(w, th, n_frames=32, start=0):
    """The oracle as it stands (FP64, every predicate on every tuple) on a
    bounded sample of the stream, on this host's cores."""
    import oracle as O
    F = D.stream_tuples(w, n_frames, start=start)
    t0 = time.perf_counter()
    S = O.udf_scores(w.kind, F, D.predicate_weights(w))
    dt = time.perf_counter() - t0
    O.result_bits(O.pass_matrix(S, th))
    return {"value": n_frames / dt, "unit": "tuples/s", "cores": O.threads(), "kind": "oracle",
            "sample": f"{n_frames} frames of the {w.n}-frame stream, all 4 UDFs in FP64 ({dt:.1f} s)"}


def ours(args):
    import torch
    ws, rank = dist_init("nccl")
    _, _, local = dist_env()
    torch.cuda.set_device(local)
    import paper_2403_14902_b300 as H
    w = D.workload(WORKLOAD)
    th = thresholds(WORKLOAD)
    Xh = torch.from_numpy(D.stream_tuples(w))
    X = Xh.cuda()
    stream = torch.cuda.Stream()
    mif = 8
    q = build_query(H, w, th, policy="rank", precision="bf16", stream=stream, max_in_flight=mif)
    calib = q.calibrate(torch.from_numpy(D.calib_tuples(w)[:64]).cuda())
    step = lambda: run_step(q, X, w.batch, mif)  # noqa: E731
    for _ in range(args.warmup):
        step()
    clocks = ClockSampler(local)
    clocks.start()
    q.profile(True)
    secs, npass = timed(step, args.steps, stream, local)
    prof, launches = q.profile_read()
    q.profile(False)
    clk = clocks.stop()
    secs_max = max_over_ranks(secs, device=torch.device("cuda", local))
    value = aggregate(w.n, args.steps, secs_max, ws)

    # end to end from pinned host memory
    Xp = Xh.pin_memory()
    bufs = [torch.empty((w.batch,) + tuple(w.frame), dtype=torch.uint8, device="cuda") for _ in range(mif)]
    hstep = lambda: run_step_host(q, Xp, bufs, w.batch, mif, stream)  # noqa: E731
    hstep()
    esecs, _ = timed(hstep, max(1, min(args.steps, 3)), stream, local)
    esecs = max_over_ranks(esecs, device=torch.device("cuda", local))
    e2e_steps = max(1, min(args.steps, 3))
    stats = q.stats()
    q.close()

    # static-order FP32 baseline (declared order, the paper's "No Reordering")
    qs = build_query(H, w, th, policy="static", precision="fp32", stream=stream, max_in_flight=mif)
    qs.calibrate(torch.from_numpy(D.calib_tuples(w)[:16]).cuda())
    sstep = lambda: run_step(qs, X, w.batch, mif)  # noqa: E731
    sstep()
    s_steps = 1
    ssecs, snpass = timed(sstep, s_steps, stream, local)
    ssecs = max_over_ranks(ssecs, device=torch.device("cuda", local))
    qs.close()
    assert snpass[0] == npass[0], "static FP32 and adaptive BF16 pass sets differ in size"

    if rank != 0:
        return None
    peaks, src = load_peaks()
    dom = max(prof.items(), key=lambda kv: kv[1]["total_ms"]) if prof else (None, None)
    roof = None
    if dom[0]:
        name, d = dom
        achieved = d["flops"] / (d["total_ms"] / 1000.0) / 1e12
        peak = float(peaks["bf16_tflops_sustained"])
        roof = {"bound": "tensor", "kernel": name, "achieved": round(achieved, 2), "peak": peak,
                "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": None,
                "peak_source": f"bf16_tflops_sustained ({src})", "launches": d["launches"],
                "avg_launch_ms": round(d["total_ms"] / max(1, d["launches"]), 4)}
    h2d = int(np.prod(Xh.shape))
    nb = (w.n + w.batch - 1) // w.batch
    d2h = nb * (4 * ((w.batch + 31) // 32) + 64 + 32 * 8)
    out = {
        "metric": METRIC, "value": round(value, 1), "unit": "tuples/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(secs_max / args.steps * 1000.0, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": f"{WORKLOAD}: {w.n} frames 3x64x64 uint8, 4 CNN UDF predicates (2/4/6/8 conv3x3 "
                               f"layers, 32-128 ch), selectivities 0.3/0.6/0.1/0.9, batches of {w.batch}, rank "
                               "c/(1-s) routing, BF16 tensor cores + FP32/FP64 recheck within 0.02",
                   "global_batch": w.n, "routing_batch": w.batch, "parallelism": f"replicas{ws}",
                   "l2": "inputs 805 MB > 126 MB L2, no flush"},
        "roofline": roof,
        "cpu_baseline": cpu_baseline(w, th),
        "e2e": {"value": round(aggregate(w.n, e2e_steps, esecs, ws), 1), "unit": "tuples/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": clk,
        "baselines": {"static_fp32_declared_order": {
            "value": round(aggregate(w.n, s_steps, ssecs, ws), 1), "unit": "tuples/s",
            "ms_per_step": round(ssecs / s_steps * 1000.0, 3)}},
        "speedup_vs_static_fp32": round(value / aggregate(w.n, s_steps, ssecs, ws), 3),
        "pass_count_per_step": int(npass[0]),
        "kernels": {k: {"launches": v["launches"], "total_ms": round(v["total_ms"], 3),
                        "tflops": round(v["flops"] / max(v["total_ms"], 1e-9) / 1e9, 2)} for k, v in prof.items()},
        "recheck": {"tf32x3": [s["recheck_tf32"] for s in stats], "fp32": [s["recheck_fp32"] for s in stats],
                    "fp64": [s["recheck_fp64"] for s in stats],
                    "calib_max_err_bf16": [round(c["max_err_lowp"], 6) for c in calib],
                    "calib_max_err_tf32x3": [float("%.3g" % c["max_err_tf32"]) for c in calib],
                    "calib_max_err_fp32": [float("%.3g" % c["max_err_fp32"]) for c in calib]},
    }
    return out


# ---------------------------------------------------------------- reference arm

def reference(args):
    """The oracle (plain FP64 CPU, every predicate on every tuple) timed on the
    host cores on a bounded sample of the same workload per step."""
    ws, rank = dist_init("gloo")
    if rank != 0:
        return None
    import oracle as O
    w = D.workload(WORKLOAD)
    th = thresholds(WORKLOAD)
    n = 8
    F = D.stream_tuples(w, n)
    ws_ = D.predicate_weights(w)
    for _ in range(args.warmup):
        O.udf_scores(w.kind, F[:1], ws_)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.result_bits(O.pass_matrix(O.udf_scores(w.kind, F, ws_), th))
    dt = time.perf_counter() - t0
    value = n * args.steps / dt
    return {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "tuples/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1000.0, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{WORKLOAD}: oracle on {n} frames of the {w.n}-frame stream per step"},
            "cpu_baseline": {"value": round(value, 3), "unit": "tuples/s", "cores": O.threads(), "kind": "oracle",
                             "sample": f"{n} frames per step, all 4 UDFs in FP64"},
            "e2e": {"value": round(value, 3), "unit": "tuples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    args = ap.parse_args(argv)
    out = reference(args) if args.impl == "reference" else ours(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
