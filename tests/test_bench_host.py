"""Host-side logic of the benchmark (no GPU): the timing spread summary, the raycast's instruction-issue roofline and
its gate on the stored capture's source hash, the stored DRAM-traffic ratios and their gate, and the constant-level
networks that bound the learned predictor."""
import json

import numpy as np
import pytest

import bench
import oracle
from paper_2511_21459_b300 import MLP_LEVELS, MLP_PARAMS
from paper_2511_21459_b300 import predictor


def test_spread_summary():
    s = bench.spread([1.0, 2.0, 3.0, 2.0])
    assert s["mean"] == 2.0 and s["min"] == 1.0 and s["max"] == 3.0 and s["n"] == 4
    assert s["spread"] == pytest.approx((3.0 - 1.0) / 2.0)


def test_raycast_roofline_arithmetic(tmp_path, monkeypatch):
    """achieved = instructions per ray x rays / launch time; peak = SMs x 4 schedulers x clock."""
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    csrc = tmp_path / "paper_2511_21459_b300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.RAYCAST_SOURCES:
        (csrc / f).write_text("source " + f)
    (tmp_path / "paper_2511_21459_b300" / "build.py").write_text("flags")
    rec = {"source_sha256": bench.source_sha256(bench.RAYCAST_SOURCES, with_build=True),
           "warp_instructions_per_ray": 1000.0, "active_threads": 16.0, "sm_mhz": 2000.0}
    (prof / "raycast_rgbd.json").write_text(json.dumps(rec))
    r = bench.raycast_roofline(ray_ms_avg=0.5, rays_per_launch=100_000, clk={"sm_max_mhz": 2000.0}, n_sms=100)
    assert r["bound"] == "alu"
    assert r["peak"] == pytest.approx(100 * 4 * 2000e6 / 1e9)
    assert r["achieved"] == pytest.approx(1000.0 * 100_000 / 0.5e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-3)
    # a source or flag change since the capture: no roofline from a stale count
    (tmp_path / "paper_2511_21459_b300" / "build.py").write_text("other flags")
    assert bench.raycast_roofline(0.5, 100_000, {"sm_max_mhz": 2000.0}, 100) is None


def test_stored_traffic_scales_and_gates(tmp_path, monkeypatch):
    """traffic = the capture's DRAM bytes per algorithmic byte x this run's algorithmic bytes per launch, only while
    the kernel sources hash as they did when the capture was taken."""
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    csrc = tmp_path / "paper_2511_21459_b300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.BATCH_FUSE_SOURCES:
        (csrc / f).write_text("source " + f)
    rec = {"source_sha256": bench.source_sha256(bench.BATCH_FUSE_SOURCES), "dram_bytes_per_algorithmic_byte": 0.8}
    (prof / "batch_fuse_traffic.json").write_text(json.dumps(rec))
    assert bench.stored_traffic("batch_fuse_traffic", bench.BATCH_FUSE_SOURCES, 1_000_000) == 800_000
    assert bench.stored_traffic("missing_traffic", bench.BATCH_FUSE_SOURCES, 1_000_000) is None
    (csrc / "mrh_batch.cu").write_text("changed")
    assert bench.stored_traffic("batch_fuse_traffic", bench.BATCH_FUSE_SOURCES, 1_000_000) is None


@pytest.mark.parametrize("level", range(MLP_LEVELS))
def test_constant_level_weights_answer_their_level(level):
    w = predictor.constant_level_weights(level)
    assert w.dtype == np.uint16 and w.size == MLP_PARAMS
    x = np.random.default_rng(level).standard_normal((200, 16)).astype(np.float32)
    logits = oracle.mlp_forward(w, x)
    assert np.all(np.argmax(logits, axis=1) == level)
