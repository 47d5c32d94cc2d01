"""The ncu captures the benchmark scales its roofline figures by (profiles/*.json) were taken from the kernel sources
as they are now: each stored source hash equals the hash of the current files (the bench drops a figure whose hash no
longer matches, so a stale capture would silently turn a reported traffic or instruction count into null)."""
import json
import os

import pytest

import bench

CAPTURES = {
    "fuse_depth_rgbd.json": (bench.source_sha256, ()),
    "raycast_rgbd.json": (bench.source_sha256, (bench.RAYCAST_SOURCES, True)),
    "lidar_fusion_traffic.json": (bench.source_sha256, (bench.LIDAR_FUSION_SOURCES,)),
    "batch_fuse_traffic.json": (bench.source_sha256, (bench.BATCH_FUSE_SOURCES,)),
}


@pytest.mark.parametrize("name", sorted(CAPTURES))
def test_stored_capture_matches_current_sources(name):
    path = os.path.join(bench.ROOT, "profiles", name)
    with open(path) as f:
        rec = json.load(f)
    fn, args = CAPTURES[name]
    assert rec["source_sha256"] == fn(*args), f"{name} was captured from other kernel sources: re-take it"
