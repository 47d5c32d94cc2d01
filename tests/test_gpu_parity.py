"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle on the same seeded inputs.

Keys, levels and weights bit-exact; D, sigma^2 and colour within 1e-4 relative (tests/parity.py); the raycast against
the oracle's definition within the bounds of tests/raycast_check.py (same bracket: within h / 8; other brackets and
hit / miss disagreements at most 0.1 % of the pixels; normals and colours at the kernel's hit points). Sizes span many CTA tiles with ragged tails; the RGB-D and
LiDAR cases run the full-size frames of the benchmark configuration.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.parity import compare_extracts
from tests.raycast_check import check_raycast, check_shading, grid_step

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_21459_b300 import build
    build.build()


def mrh():
    import paper_2511_21459_b300 as m
    return m


def gpu_map(wl, **kw):
    m = mrh()
    return m.Map(m.params_from(wl, **kw))


def orc_map(wl, **kw):
    return oracle.OracleMap(oracle.params_from(wl, "f32s", **kw))


def run_camera(wl, frames, gmap, omap, check_each=False, theta0=None, raycast_frames=()):
    K_g, K_o = mrh().pinhole_from(wl), oracle.pinhole_from(wl)
    theta0 = wl.var_threshold[0] if theta0 is None else theta0
    reports = []
    for f, (depth, rgb, T) in enumerate(frames):
        d_t = torch.from_numpy(depth).cuda()
        c_t = torch.from_numpy(rgb).cuda()
        gmap.integrate_depth(K_g, T, d_t, c_t)
        st_o = omap.integrate_depth(K_o, T, depth, rgb)
        st_g = gmap.stats()
        assert st_g["status_code"] == 0, st_g
        for k in ("valid_rays", "touched", "new_blocks", "merged", "split", "observations", "updated_voxels"):
            assert st_g[k] == st_o[k], (f, k, st_g[k], st_o[k])
        if check_each or f == len(frames) - 1:
            reports.append(compare_extracts(gmap.extract(), omap.extract(), wl.truncation, theta0,
                                            check_color=wl.has_color))
        if f in raycast_frames:
            color = bool(wl.has_color)
            out_g = [x.cpu().numpy() for x in gmap.raycast(K_g, T, normals=True, rgb=color)]
            out_o = omap.raycast(K_o, T, normals=True, rgb=color)
            check_raycast(out_g[0], out_o[0], grid_step(wl))
            check_shading(out_g, omap, K_o, T)
    return reports


def test_tiny_single_frame():
    wl = synth.tiny()
    frames = [synth.render_depth(wl, 0)]
    rep = run_camera(wl, frames, gpu_map(wl), orc_map(wl), raycast_frames=(0,))
    assert rep[-1]["D_bit_exact"] and rep[-1]["S2_bit_exact"]


def test_tiny_repeated_views_relevel_bit_exact():
    """Ten noisy views from one pose (seeds 0-9): blocks merge once k_min views accumulate, some split back; keys,
    levels and every voxel field match the oracle after every frame."""
    wl = synth.tiny()
    frames = [synth.render_depth(wl, 0, seed=s) for s in range(10)]
    g, o = gpu_map(wl), orc_map(wl)
    reps = run_camera(wl, frames, g, o, check_each=True, raycast_frames=(9,))
    st = o.block_stats()
    assert (st["levels"] == 1).sum() > 100  # merges happened
    assert all(r["D_bit_exact"] for r in reps)


def test_tiny_noise_free_views_merge_everything_observed():
    wl = synth.tiny(noise=False)
    frames = [synth.render_depth(wl, 0)] * 6
    g, o = gpu_map(wl), orc_map(wl)
    run_camera(wl, frames, g, o, check_each=True)
    assert g.stats()["live_blocks"][1] > 1000


def test_fp16_storage_matches_oracle_half_mode():
    wl = synth.tiny()
    wl.fp16 = True
    frames = [synth.render_depth(wl, 0, seed=s) for s in range(8)]
    run_camera(wl, frames, gpu_map(wl), orc_map(wl), check_each=True, raycast_frames=(7,))


def test_rgbd_full_size_prefix():
    """The benchmark's RGB-D configuration (640x480, 3 levels, 2^20 hash): first 6 frames of the sequence, full
    comparison after every frame, raycast at frames 0 and 5."""
    wl = synth.rgbd()
    scene = wl.scene()
    frames = [synth.render_depth(wl, k, scene=scene) for k in range(6)]
    reps = run_camera(wl, frames, gpu_map(wl), orc_map(wl), check_each=True, raycast_frames=(0, 5))
    assert reps[-1]["D_max_abs"] <= 1e-4 * wl.truncation


def test_rgbd_late_sequence_window():
    """The benchmark's RGB-D configuration and thresholds, 40 frames spread over the whole orbit (every 7th pose), so
    the map holds most of what it holds at the end of the sequence, with merges at the benchmark's thresholds and
    raycasts that read across levels: counters after every frame, then the full map and a raycast from the last
    pose against the oracle."""
    wl = synth.rgbd()
    scene = wl.scene()
    frames = [synth.render_depth(wl, 7 * k, scene=scene) for k in range(40)]
    g, o = gpu_map(wl), orc_map(wl)
    run_camera(wl, frames, g, o, raycast_frames=(39,))
    st = o.block_stats()
    assert (st["levels"] > 0).sum() > 100


def test_rgbd_sparse_frames_and_relevel():
    """Every 10th pose of the sequence (bigger motion between frames) with a threshold that makes both merges and
    splits happen."""
    wl = synth.rgbd()
    wl.var_threshold = (2e-4, 8e-4)
    wl.min_obs = 2
    wl.split_hysteresis = 1.5
    scene = wl.scene()
    frames = [synth.render_depth(wl, 10 * k, scene=scene) for k in range(6)]
    g, o = gpu_map(wl), orc_map(wl)
    run_camera(wl, frames, g, o, check_each=True)
    st = o.block_stats()
    assert (st["levels"] > 0).sum() > 100


def test_ragged_image_and_invalid_depth():
    wl = synth.tiny()
    wl.width, wl.height, wl.cx, wl.cy = 161, 117, 79.5, 58.25
    depth, rgb, T = synth.render_depth(wl, 0)
    depth[::7, ::5] = 0.0
    depth[3::11, 2::13] = np.nan
    depth[50:60, 20:40] = 100.0  # beyond max_depth
    run_camera(wl, [(depth, rgb, T)], gpu_map(wl), orc_map(wl), raycast_frames=(0,))


def test_empty_frame_allocates_nothing():
    wl = synth.tiny()
    g = gpu_map(wl)
    K = mrh().pinhole_from(wl)
    g.integrate_depth(K, np.eye(4), torch.zeros((wl.height, wl.width), device="cuda"), None)
    assert g.count() == (0, 0)
    st = g.stats()
    assert st["touched"] == 0 and st["status_code"] == 0
    ex = g.extract()
    assert ex["keys"].shape[0] == 0
    assert torch.all(g.raycast(K, np.eye(4)) == 0)


def test_determinism_bitwise():
    wl = synth.rgbd()
    scene = wl.scene()
    frames = [synth.render_depth(wl, k, scene=scene) for k in range(2)]
    outs = []
    for _ in range(2):
        g = gpu_map(wl)
        for depth, rgb, T in frames:
            g.integrate_depth(mrh().pinhole_from(wl), T, torch.from_numpy(depth).cuda(), torch.from_numpy(rgb).cuda())
        outs.append({k: v.cpu().numpy() for k, v in g.extract().items()})
        g.close()
    for k in outs[0]:
        np.testing.assert_array_equal(outs[0][k], outs[1][k])


# ------------------------------------------------------------------------------------------------ LiDAR

def run_lidar(wl, n_frames, check_each=True, scene=None):
    g, o = gpu_map(wl), orc_map(wl)
    scene = wl.scene() if scene is None else scene
    for f in range(n_frames):
        xyz, T = synth.render_lidar(wl, f, scene=scene)
        g.integrate_points(T, torch.from_numpy(xyz).cuda())
        st_o = o.integrate_points(T, xyz)
        st_g = g.stats()
        assert st_g["status_code"] == 0, st_g
        for k in ("valid_rays", "touched", "new_blocks", "merged", "split", "observations", "updated_voxels"):
            assert st_g[k] == st_o[k], (f, k, st_g[k], st_o[k])
        if check_each or f == n_frames - 1:
            compare_extracts(g.extract(), o.extract(), wl.truncation, wl.var_threshold[0], check_color=False)
    return g, o


def test_lidar_small_scans_fp16():
    wl = synth.lidar()
    wl.n_beams, wl.n_azimuth = 32, 256
    wl.min_obs = 2
    run_lidar(wl, 5)


def test_lidar_small_scans_fp32_with_relevel():
    wl = synth.lidar()
    wl.fp16 = False
    wl.n_beams, wl.n_azimuth = 64, 512
    wl.min_obs = 2
    wl.var_threshold = (2e-3, 8e-3)
    wl.split_hysteresis = 1.5
    g, o = run_lidar(wl, 4)
    assert (o.block_stats()["levels"] > 0).sum() > 10


def test_lidar_long_bands_take_the_restage_path():
    """A truncation band of 3.2 m at 5 cm voxels gives oblique points more observation entries than the per-point
    stage holds: those points are written by the second walk, with the same result."""
    wl = synth.lidar()
    wl.n_beams, wl.n_azimuth = 32, 256
    wl.truncation = 1.6  # the largest band allowed: 2 tau = 8 blocks
    wl.min_obs = 2
    g, o = run_lidar(wl, 3)
    assert g.stats()["lidar_restaged"] > 0


def test_lidar_map_raycast_normals_fp16():
    """Raycast of a LiDAR-fused map (FP16 storage, no colour) from a pinhole looking along the sensor's heading:
    depth and normals match the oracle; asking for colour from a map without colour is an argument error."""
    wl = synth.lidar()
    wl.n_beams, wl.n_azimuth = 128, 1024
    wl.min_obs = 2
    g, o = run_lidar(wl, 3, check_each=False)
    c, s = np.cos(0.3), np.sin(0.3)          # optical axis along the heading, pitched 0.3 rad down
    cam_from_sensor = np.eye(4)
    cam_from_sensor[:3, :3] = [[0.0, -s, c], [-1.0, 0.0, 0.0], [0.0, -c, -s]]
    T = synth.lidar_pose(2) @ cam_from_sensor
    K_g, K_o = mrh().Pinhole(), oracle.Pinhole()
    for K in (K_g, K_o):
        K.fx = K.fy = 160.0
        K.cx, K.cy, K.width, K.height = 160.0, 60.0, 320, 120
        K.min_depth, K.max_depth = 0.5, 40.0
    out_g = [x.cpu().numpy() for x in g.raycast(K_g, T, normals=True)]
    out_o = o.raycast(K_o, T, normals=True)
    check_raycast(out_g[0], out_o[0], grid_step(wl))
    assert (out_o[0] > 0).mean() > 0.5
    check_shading(out_g, o, K_o, T)
    with pytest.raises(mrh().MrhError):
        g.raycast(K_g, T, rgb=True)


def test_lidar_dense_patch_many_points_per_block():
    """Points on a 0.5 m x 0.5 m patch 1 m in front of the sensor (128 x 128 per scan, seeded range noise): a block
    receives thousands of points and a voxel hundreds of observations per scan, far beyond the 16 that are ordered in
    registers (the long lists are applied in passes of 8 smallest point indices), and with a high threshold the
    blocks merge to the coarse levels, whose voxels collect more still. Counters after every scan and the whole map
    against the oracle."""
    wl = synth.lidar()
    wl.fp16 = False
    wl.min_obs = 2
    wl.var_threshold = (5e-2, 2e-1)
    wl.split_hysteresis = 0.0
    g, o = gpu_map(wl), orc_map(wl)
    rng = np.random.default_rng(17)
    n = 128
    a, b = np.meshgrid(np.linspace(-0.25, 0.25, n), np.linspace(-0.25, 0.25, n))
    most = 0
    for f in range(4):
        dirs = np.stack([np.ones(n * n), a.ravel(), b.ravel()], -1)
        dirs /= np.linalg.norm(dirs, axis=-1, keepdims=True)
        rng_m = 1.0 / dirs[:, 0] + rng.normal(0.0, 0.01, n * n)
        xyz = (dirs * rng_m[:, None]).astype(np.float32)
        T = np.eye(4)
        g.integrate_points(T, torch.from_numpy(xyz).cuda())
        st_o = o.integrate_points(T, xyz)
        st_g = g.stats()
        assert st_g["status_code"] == 0, st_g
        for k in ("valid_rays", "touched", "new_blocks", "merged", "split", "observations", "updated_voxels"):
            assert st_g[k] == st_o[k], (f, k, st_g[k], st_o[k])
        most = max(most, st_g["lidar_max_voxel_obs"])
        compare_extracts(g.extract(), o.extract(), wl.truncation, wl.var_threshold[0], check_color=False)
    assert most > 300, most
    assert (o.block_stats()["levels"] > 0).sum() > 0


def test_lidar_full_scans():
    """Six full 128 x 2048 scans of the benchmark's LiDAR configuration (FP16 storage)."""
    wl = synth.lidar()
    run_lidar(wl, 6, check_each=False)


# ------------------------------------------------------------------------------------------------ errors

def test_hash_full_sets_status_and_map_stays_usable():
    wl = synth.tiny()
    wl.hash_log2 = 10  # 1024 slots for ~4700 blocks
    g = gpu_map(wl)
    depth, rgb, T = synth.render_depth(wl, 0)
    K = mrh().pinhole_from(wl)
    g.integrate_depth(K, T, torch.from_numpy(depth).cuda(), torch.from_numpy(rgb).cuda())
    st = g.stats()
    assert st["status_code"] == 3
    g.clear_status()
    g.integrate_depth(K, T, torch.zeros_like(torch.from_numpy(depth)).cuda(), None)
    assert g.stats()["status_code"] == 0


def test_pool_empty_and_list_full_set_status():
    wl = synth.tiny()
    wl.max_blocks = (100, 100, 100)
    g = gpu_map(wl)
    depth, rgb, T = synth.render_depth(wl, 0)
    K = mrh().pinhole_from(wl)
    g.integrate_depth(K, T, torch.from_numpy(depth).cuda(), torch.from_numpy(rgb).cuda())
    assert g.stats()["status_code"] == 4
    assert g.count()[0] == 100
    wl2 = synth.tiny()
    wl2.max_touched = 64
    g2 = gpu_map(wl2)
    g2.integrate_depth(K, T, torch.from_numpy(depth).cuda(), torch.from_numpy(rgb).cuda())
    assert g2.stats()["status_code"] == 5


def test_invalid_arguments_are_rejected_on_host():
    m = mrh()
    wl = synth.tiny()
    g = gpu_map(wl)
    K = m.pinhole_from(wl)
    d = torch.zeros((wl.height, wl.width), device="cuda")
    bad = m.Pinhole.from_buffer_copy(K)
    bad.fx = 0.0
    with pytest.raises(m.MrhError) as e:
        g.integrate_depth(bad, np.eye(4), d)
    assert e.value.code == 1
    T = np.eye(4)
    T[0, 3] = np.nan
    with pytest.raises(m.MrhError):
        g.integrate_depth(K, T, d)
    with pytest.raises(m.MrhError):
        g.raycast(K, T)
