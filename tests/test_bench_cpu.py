"""Host logic of bench.py that decides whether the recorded ncu traffic still
describes the timed kernel: the source hash ignores comments and whitespace
but not code, and a record taken on other code, another workload or another
tile size is not reported."""
import importlib.util
import json
import os
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b


@pytest.fixture
def tree(tmp_path):
    """A copy of the hashed sources and the traffic record, with bench.py's
    ROOT pointed at it."""
    b = _bench()
    for f in b.RASTER_SOURCES:
        os.makedirs(tmp_path / os.path.dirname(f), exist_ok=True)
        shutil.copy(os.path.join(ROOT, f), tmp_path / f)
    os.makedirs(tmp_path / "profiles")
    shutil.copy(os.path.join(ROOT, "profiles", "ncu_traffic.json"), tmp_path / "profiles" / "ncu_traffic.json")
    b.ROOT = str(tmp_path)
    return b, tmp_path


def _edit(path, fn):
    with open(path) as f:
        s = f.read()
    with open(path, "w") as f:
        f.write(fn(s))


def test_hash_ignores_comments_and_whitespace_not_code(tree):
    b, root = tree
    h0 = b.raster_source_hash()
    src = root / b.RASTER_SOURCES[0]
    _edit(src, lambda s: "// a new comment line\n/* and a\n   block */\n" + s.replace("\n", "\n  ", 5))
    assert b.raster_source_hash() == h0
    _edit(src, lambda s: s + "\nstatic const int kChanged = 1;\n")
    assert b.raster_source_hash() != h0


def test_traffic_reported_only_for_the_recorded_code_workload_and_tile(tree):
    b, root = tree
    rec = json.load(open(root / "profiles" / "ncu_traffic.json"))["k_raster_bwd"]
    cfg = rec["config"]
    # the committed record matches the committed sources
    traffic, note = b.measured_traffic("k_raster_bwd", rec["workload"], cfg)
    assert traffic == rec["dram_bytes_per_launch"] and note == rec["command"]
    # the batch depth does not change the backward's traffic; the tile size does
    tile = cfg.split("/")[0]
    assert b.measured_traffic("k_raster_bwd", rec["workload"], tile + "/64")[0] == traffic
    assert b.measured_traffic("k_raster_bwd", rec["workload"], "8x8/128")[0] is None
    assert b.measured_traffic("k_raster_bwd", "another_workload", cfg)[0] is None
    # code changed since the capture
    _edit(root / b.RASTER_SOURCES[-1], lambda s: s + "\nstatic const int kChanged = 1;\n")
    traffic, note = b.measured_traffic("k_raster_bwd", rec["workload"], cfg)
    assert traffic is None and "changed" in note


def test_traffic_scaled_to_another_workload_by_algorithmic_bytes(tree):
    b, root = tree
    path = root / "profiles" / "ncu_traffic.json"
    recs = json.load(open(path))
    rec = recs["k_raster_bwd"]
    rec["algorithmic_bytes"] = 1000
    json.dump(recs, open(path, "w"))
    traffic, note = b.measured_traffic("k_raster_bwd", "another_workload", rec["config"], 3000)
    assert traffic == 3 * rec["dram_bytes_per_launch"] and "scaled" in note
    assert b.measured_traffic("k_raster_bwd", "another_workload", rec["config"])[0] is None


def test_stage_bytes_and_report_use_every_stage():
    b = _bench()

    class A:
        depth_loss, ssim_lambda = "kl", 0.0
    u = dict(N=100, views=2, pairs=200, visible=50, instances=400, listed=300, tiles=10, pix=1000, lidar=20,
             touched=40, sh_coeffs=16, pixel_entries=5000, pixel_blends=2000, tile_entries=100, tile_active=80)
    kern = {k: 0.01 for k in ("project", "compact", "depth_sort", "emit", "tile_sort", "ranges", "raster_fwd",
                               "image_l1", "depth_loss", "zero_grad", "raster_bwd", "project_bwd")}
    alu = {"fp32_fma": 60.0, "fp32x2_fma": 70.0}
    rep = b.roofline_report(u, kern, 0.2, 6000.0, "test", alu, A, 16, 16)
    assert set(rep["stages"]) == set(kern)
    bw = rep["roofline"]
    assert bw["peak"] == 70.0
    assert bw["flops"] == 5000 * b.EVAL_FLOPS + 2000 * b.BWD_BLEND_FLOPS
    P = 4 * (11 + 48)
    assert rep["bytes"]["project_bwd"] == P * 40 + (P + 8) * 100 + 72 * 50
    assert rep["bytes"]["project"] == 44 * 100 + (P - 44) * 40 + 12 * 200 + 88 * 50
    B = 3 * 40 * P + 260 * 50 + 52 * 400 + 88 * 1000 + 20 * 20 + 8 * 40
    assert rep["step"]["algorithmic_bytes"] == B
    assert abs(rep["step"]["frac"] - B / 0.2e-3 / 1e9 / 6000.0) < 1e-12
