"""The C-ABI library loads and exports every entry point include/hydro.h
declares, the ctypes structs match the header's layout, and argument
checking that needs no GPU behaves (no compute calls here)."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2403_14902_b300 as H

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hydro.h")


def _declared():
    with open(HEADER) as f:
        src = f.read()
    return sorted(set(re.findall(r"HYDRO_API[^;(]*?\b(hydro_\w+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = H.load()
    names = _declared()
    assert set(names) == set(H.EXPORTED)
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", H.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (hydro_\w+)", out))
    assert set(names) <= exported


def test_struct_layouts_match_header(tmp_path):
    prog = tmp_path / "sizes.c"
    prog.write_text(r'''
#include <stddef.h>
#include <stdio.h>
#include "hydro.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(hydro_query_config), sizeof(hydro_udf_desc),
         sizeof(hydro_batch_info), sizeof(hydro_pred_stats), sizeof(hydro_calib_info));
  printf("%zu %zu %zu %zu\n", offsetof(hydro_query_config, stream), offsetof(hydro_udf_desc, head_bias),
         offsetof(hydro_batch_info, device_ms), offsetof(hydro_pred_stats, margin_fp32));
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(hydro_session_config), offsetof(hydro_session_config, stream),
         sizeof(hydro_step_query), offsetof(hydro_step_query, evaluated), sizeof(hydro_tile_choice),
         offsetof(hydro_tile_choice, us));
  return 0;
}
''')
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    a, b, c = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")[:3]
    assert [int(x) for x in a.split()] == [ctypes.sizeof(H.QueryConfig), ctypes.sizeof(H.UdfDesc),
                                          ctypes.sizeof(H.BatchInfo), ctypes.sizeof(H.PredStats),
                                          ctypes.sizeof(H.CalibInfo)]
    assert [int(x) for x in b.split()] == [H.QueryConfig.stream.offset, H.UdfDesc.head_bias.offset,
                                          H.BatchInfo.device_ms.offset, H.PredStats.margin_fp32.offset]
    assert [int(x) for x in c.split()] == [ctypes.sizeof(H.SessionConfig), H.SessionConfig.stream.offset,
                                          ctypes.sizeof(H.StepQuery), H.StepQuery.evaluated.offset,
                                          ctypes.sizeof(H.TileChoice), H.TileChoice.us.offset]


def test_session_defaults_and_rejections_without_a_device():
    L = H.load()
    cfg = H.SessionConfig()
    L.hydro_session_default_config(ctypes.byref(cfg))
    assert (cfg.precision, cfg.warmup_batches, cfg.stats_window, cfg.use_graphs, cfg.autotune,
            cfg.max_in_flight) == (0, 1, 8, 1, 1, 2)
    h = ctypes.c_void_p()
    cfg.max_step_tuples = 1024
    cfg.dim = 100                      # not a multiple of 64
    assert L.hydro_session_create(ctypes.byref(cfg), ctypes.byref(h)) == H.EINVAL
    assert b"dim" in L.hydro_last_error()
    cfg.dim = 512
    cfg.max_step_tuples = 0
    assert L.hydro_session_create(ctypes.byref(cfg), ctypes.byref(h)) == H.EINVAL
    cfg.max_step_tuples = 1024
    cfg.max_in_flight = 9
    assert L.hydro_session_create(ctypes.byref(cfg), ctypes.byref(h)) == H.EINVAL
    cfg.max_in_flight = 2
    assert cfg.fp8_min_width == 0
    cfg.precision = H.PRECISIONS["fp8"]
    cfg.dim = 192                      # FP8 sessions: E4M3 rows in 128-byte K slices
    assert L.hydro_session_create(ctypes.byref(cfg), ctypes.byref(h)) == H.EINVAL
    assert b"FP8" in L.hydro_last_error()
    cfg.dim = 512
    cfg.fp8_min_width = -1
    assert L.hydro_session_create(ctypes.byref(cfg), ctypes.byref(h)) == H.EINVAL
    cfg.precision = H.PRECISIONS["bf16"]
    cfg.policy = H.POLICIES["all"]     # sessions route by rank or keep the declared order
    assert L.hydro_session_create(ctypes.byref(cfg), ctypes.byref(h)) == H.EINVAL
    cfg.policy = H.POLICIES["static"]
    cfg.learned = 1                    # a learned session falls back to rank routing
    assert L.hydro_session_create(ctypes.byref(cfg), ctypes.byref(h)) == H.EINVAL
    cfg.learned = 0
    cfg.policy = H.POLICIES["rank"]
    cfg.precision = 6                  # no such precision
    cfg.fp8_min_width = 0
    assert L.hydro_session_create(ctypes.byref(cfg), ctypes.byref(h)) == H.EINVAL
    assert L.hydro_session_create(None, ctypes.byref(h)) == H.EINVAL
    assert L.hydro_session_destroy(None) == H.EINVAL
    assert L.hydro_session_poll(None, 0, None, None, None, 0) == H.EINVAL
    sid = ctypes.c_int64()
    assert L.hydro_session_submit(None, None, None, ctypes.byref(sid)) == H.EINVAL


def test_default_config():
    cfg = H.QueryConfig()
    H.load().hydro_default_config(ctypes.byref(cfg))
    assert (cfg.policy, cfg.precision, cfg.warmup_batches, cfg.stats_window, cfg.route_lag,
            cfg.max_in_flight, cfg.proxy_hidden, cfg.proxy_refresh) == (0, 0, 1, 8, 1, 4, 64, 16)


def test_create_rejects_bad_config_without_touching_a_device():
    L = H.load()
    cfg = H.QueryConfig()
    L.hydro_default_config(ctypes.byref(cfg))
    h = ctypes.c_void_p()
    cfg.dim = 0
    cfg.max_batch = 16
    assert L.hydro_create_query(ctypes.byref(cfg), ctypes.byref(h)) == H.EINVAL
    assert b"dim" in L.hydro_last_error()
    cfg.dim = 8
    cfg.max_batch = 0
    assert L.hydro_create_query(ctypes.byref(cfg), ctypes.byref(h)) == H.EINVAL
    cfg.max_batch = 16
    cfg.route_lag = 8
    assert L.hydro_create_query(ctypes.byref(cfg), ctypes.byref(h)) == H.EINVAL
    cfg.route_lag = 1
    cfg.lanes = 3                      # more lanes than route_lag + 1
    assert L.hydro_create_query(ctypes.byref(cfg), ctypes.byref(h)) == H.EINVAL
    cfg.lanes = 9
    cfg.route_lag = 7
    assert L.hydro_create_query(ctypes.byref(cfg), ctypes.byref(h)) == H.EINVAL
    cfg.lanes = 1
    cfg.cost_source = 2                # no such cost source
    assert L.hydro_create_query(ctypes.byref(cfg), ctypes.byref(h)) == H.EINVAL
    cfg.cost_source = H.COSTS["measured"]
    cfg.warmup_batches = 0             # measured cost needs the warmup statistics
    assert L.hydro_create_query(ctypes.byref(cfg), ctypes.byref(h)) == H.EUNSUPPORTED
    cfg.warmup_batches = 1
    cfg.policy = H.POLICIES["static"]
    assert L.hydro_create_query(ctypes.byref(cfg), ctypes.byref(h)) == H.EUNSUPPORTED
    cfg.policy = H.POLICIES["rank"]
    cfg.cost_source = H.COSTS["model"]
    assert L.hydro_create_query(None, ctypes.byref(h)) == H.EINVAL


def test_null_query_handles():
    L = H.load()
    assert L.hydro_destroy_query(None) == H.EINVAL
    assert L.hydro_poll_result(None, 0, None, None, None, 0) == H.EINVAL
    bid = ctypes.c_int64()
    assert L.hydro_submit_batch(None, None, None, 0, ctypes.byref(bid)) == H.EINVAL


def test_create_without_device_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    with pytest.raises(H.HydroError) as e:
        H.Query("vec", dim=8, max_batch=16)
    assert e.value.status == H.ECUDA
