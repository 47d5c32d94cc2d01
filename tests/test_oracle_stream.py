"""Pins for capacity-driven streaming (Sec. 3.3). Streaming only moves blocks between the map and its archive, so a map
that streams and a control map that does not must hold the same blocks, bit for bit: every resident block equals the
control's, and resident plus archived keys are the control's keys. The eviction set is checked against direct
geometry (the view cone or the radius, in double with a margin so that only clear cases are asserted)."""
import numpy as np
import pytest

import oracle
import synth

MB = (600, 400, 400)


def _rgbd():
    wl = synth.rgbd()
    return wl, wl.scene()


def _map(wl):
    return oracle.OracleMap(oracle.params_from(wl, "f32s"))


def _centres(keys, E):
    return (keys.astype(np.float64) + 0.5) * E


def _voxels(ex, blocks):
    """Positions, in the extract's voxel arrays, of the voxels of the given blocks (in that block order)."""
    starts = ex["offsets"][blocks]
    lens = ex["offsets"][blocks + 1] - starts
    first = np.cumsum(lens) - lens
    return np.repeat(starts - first, lens) + np.arange(int(lens.sum()))


def _match(a, b):
    """Indices into b of a's blocks (every key of a must be in b)."""
    kb = {tuple(k): i for i, k in enumerate(b["keys"].tolist())}
    return np.array([kb[tuple(k)] for k in a["keys"].tolist()], dtype=np.int64)


def test_nothing_moves_below_the_capacity_fraction():
    wl, sc = _rgbd()
    m = _map(wl)
    m.set_streaming(0.85, 0.0, (10 ** 9,) * 3)
    K = oracle.pinhole_from(wl)
    for k in (0, 100):
        d, c, T = synth.render_depth(wl, k, scene=sc)
        st = m.integrate_depth(K, T, d, c)
        assert st["evicted"] == 0 and st["restored"] == 0
    assert m.archived() == 0


def test_camera_streaming_moves_blocks_without_changing_any():
    wl, sc = _rgbd()
    K = oracle.pinhole_from(wl)
    seq = [0, 2, 4, 150, 152, 2, 4]  # the opposite side of the orbit, then back
    frames = {k: synth.render_depth(wl, k, scene=sc) for k in set(seq)}
    ctl, m = _map(wl), _map(wl)
    m.set_streaming(0.85, 0.0, MB)
    E = wl.base_voxel * 2  # block edge: 8 finest voxels of a quarter of the coarsest voxel
    ev = rs = 0
    for k in seq:
        d, c, T = frames[k]
        ctl.integrate_depth(K, T, d, c)
        st = m.integrate_depth(K, T, d, c)
        ev += st["evicted"]
        rs += st["restored"]
        if st["evicted"]:
            # blocks that stayed are inside this frame's view cone, give or take the margin
            ex = m.extract()
            cen = _centres(ex["keys"], E)
            R, t = T[:3, :3], T[:3, 3]
            xc = (cen - t) @ R
            r = np.sqrt(3) / 2 * E
            tx = max(K.cx, K.width - K.cx) / K.fx
            far_out = (xc[:, 2] + r < K.min_depth - 1e-3) | (np.abs(xc[:, 0]) > xc[:, 2] * tx + r * np.sqrt(1 + tx * tx) + 1e-3)
            assert not far_out.any()
    assert ev > 1000 and rs > 100
    a, b = m.extract(), ctl.extract()
    idx = _match(a, b)
    assert np.array_equal(a["levels"], b["levels"][idx])
    pa, pb = _voxels(a, np.arange(len(idx))), _voxels(b, idx)
    for f in ("D", "W", "S2"):
        assert np.array_equal(a[f][pa], b[f][pb]), f
    assert len(a["keys"]) + m.archived() == len(b["keys"])


def test_lidar_streaming_keeps_the_radius_and_the_blocks():
    wl = synth.lidar()
    wl.n_beams, wl.n_azimuth = 32, 256
    sc = wl.scene()
    ctl, m = _map(wl), _map(wl)
    m.set_streaming(0.5, 25.0, (300, 300, 300))
    ev = 0
    for f in range(0, 24, 3):
        xyz, T = synth.render_lidar(wl, f, scene=sc)
        ctl.integrate_points(T, xyz)
        st = m.integrate_points(T, xyz)
        ev += st["evicted"]
        if st["evicted"]:
            cen = _centres(m.extract()["keys"], wl.base_voxel * 2)
            # a resident block farther than the radius (plus a margin) can only have been allocated by this scan
            far = np.linalg.norm(cen - T[:3, 3], axis=1) > 25.0 + 1e-3
            assert far.sum() <= st["new_blocks"]
    assert ev > 0
    a, b = m.extract(), ctl.extract()
    assert len(a["keys"]) + m.archived() == len(b["keys"])
    idx = _match(a, b)
    assert np.array_equal(a["D"][_voxels(a, np.arange(len(idx)))], b["D"][_voxels(b, idx)])
