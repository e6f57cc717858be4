"""The N > 1 path of bench.py on CPU: two gloo ranks on 127.0.0.1.  Every
rank runs an independent replica (the path shards by tuples with no exchange
step); the only collectives are the barrier and the max over ranks of the
timed region, and rank 0 alone prints the JSON line."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, secs, out_path, fail_rank):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import datetime

    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", timeout=datetime.timedelta(seconds=20))
    if rank == fail_rank:
        os._exit(3)   # leaves between steps, before the barrier: the other rank must fail, not hang
    try:
        bench.barrier()
        m = bench.max_over_ranks(secs[rank])
        v = bench.aggregate(1000, 4, m, world)
        with open(f"{out_path}.{rank}", "w") as f:
            json.dump({"max": m, "value": v}, f)
    except Exception as e:   # noqa: BLE001
        with open(f"{out_path}.{rank}", "w") as f:
            json.dump({"error": type(e).__name__}, f)
    finally:
        if dist.is_initialized():
            try:
                dist.destroy_process_group()
            except Exception:   # noqa: BLE001
                pass


def _spawn(tmp_path, secs, fail_rank=-1):
    import torch.multiprocessing as mp
    out = str(tmp_path / "r")
    ctx = mp.get_context("spawn")
    port = free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, secs, out, fail_rank)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(not p.is_alive() for p in procs)
    res = {}
    for r in range(2):
        if os.path.exists(f"{out}.{r}"):
            with open(f"{out}.{r}") as f:
                res[r] = json.load(f)
    return procs, res


def test_max_over_ranks_and_whole_job_value(tmp_path):
    procs, res = _spawn(tmp_path, [0.5, 2.0])
    assert [p.exitcode for p in procs] == [0, 0]
    for r in range(2):
        assert res[r]["max"] == 2.0
        # 1,000 tuples x 4 steps on each of 2 ranks over the slowest rank's 2 s
        assert res[r]["value"] == pytest.approx(1000 * 4 * 2 / 2.0)


def test_rank_that_leaves_fails_the_other_rank_instead_of_hanging(tmp_path):
    procs, res = _spawn(tmp_path, [1.0, 1.0], fail_rank=1)
    assert procs[1].exitcode == 3
    assert "error" in res.get(0, {}), res


def test_reference_arm_under_torchrun_prints_one_line():
    port = free_port()
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
                        "--workload", "cnn4", "--gpus", "2", "--steps", "1", "--warmup", "1"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
