"""Pins for the oracle's fusion: Eq. 2 (camera), Eq. 1 (LiDAR), Eq. 3 (running mean) and the Welford S2 (Sec. 3.2.1).

Truth comes from outside the oracle: analytic ranges of the synthetic scene (tests/analytic.py), numpy two-pass means
and variances, and closed forms for a single LiDAR ray at normal incidence.
"""
import numpy as np
import pytest

import oracle
import synth
from tests import analytic

NO_RELEVEL = dict(var_threshold=(-1.0, -1.0), split_hysteresis=0.0)


def _tiny_map(precision, noise=False, **kw):
    wl = synth.tiny(noise=noise)
    m = oracle.OracleMap(oracle.params_from(wl, precision, **{**NO_RELEVEL, **kw}))
    return wl, m


@pytest.mark.parametrize("precision,tol", [("f64", 1e-6), ("f32s", 4e-6)])
def test_camera_tsdf_equals_analytic_range(precision, tol):
    """Noise-free frame: every voxel gets clip(rho_true(u,v) - |x|, tau) where (u, v) is its nearest pixel, and
    exactly the voxels more than tau behind the surface (or outside the image) stay unobserved."""
    wl, m = _tiny_map(precision)
    depth, rgb, T = synth.render_depth(wl, 0)
    m.integrate_depth(oracle.pinhole_from(wl), T, depth, rgb)
    ex = m.extract()
    x, _ = analytic.voxel_centres(ex, wl)
    zc = x[:, 2]
    front = zc > 0
    u = np.floor(wl.fx * x[:, 0] / np.where(front, zc, 1) + wl.cx + 0.5)
    v = np.floor(wl.fy * x[:, 1] / np.where(front, zc, 1) + wl.cy + 0.5)
    inside = front & (u >= 0) & (u < wl.width) & (v >= 0) & (v < wl.height)
    z_true = np.zeros(len(x))
    z_true[inside] = analytic.pixel_z_depth(wl, wl.scene(), T, u[inside], v[inside])
    qn = np.sqrt(((u - wl.cx) / wl.fx) ** 2 + ((v - wl.cy) / wl.fy) ** 2 + 1)
    eta = z_true * qn - np.linalg.norm(x, axis=1)
    tau = np.float32(wl.truncation)
    observed = inside & (z_true > 0) & (eta >= -tau)
    borderline = np.abs(eta + tau) < 1e-5
    assert np.all((ex["W"] > 0)[~borderline] == observed[~borderline])
    sel = observed & (ex["W"] > 0)
    expected = np.minimum(eta[sel], tau)
    assert sel.sum() > 100000
    np.testing.assert_allclose(ex["D"][sel], expected, rtol=0, atol=tol)
    assert np.all(ex["W"][sel] == 1.0) and np.all(ex["S2"] == 0.0)
    # the optical-axis pixel sees the sphere front at exactly z = 1.0
    assert abs(float(depth[60, 80]) - 1.0) < 1e-7


def test_camera_colour_is_running_mean():
    wl, m = _tiny_map("f64")
    depth, rgb, T = synth.render_depth(wl, 0)
    m.integrate_depth(oracle.pinhole_from(wl), T, depth, rgb)
    m.integrate_depth(oracle.pinhole_from(wl), T, depth, np.zeros_like(rgb))
    ex = m.extract()
    obs = ex["W"] == 2
    # first frame writes the pixel colour, the second (black) halves it: C = c/2
    x, _ = analytic.voxel_centres(ex, wl)
    u = np.floor(wl.fx * x[obs, 0] / x[obs, 2] + wl.cx + 0.5).astype(int)
    v = np.floor(wl.fy * x[obs, 1] / x[obs, 2] + wl.cy + 0.5).astype(int)
    np.testing.assert_allclose(ex["C"][obs], rgb[v, u].astype(np.float64) / 2.0, rtol=0, atol=1e-12)


def _per_voxel(ex):
    """dict (key tuple, voxel index) -> row, for level-0 extracts."""
    out = {}
    for b in range(len(ex["levels"])):
        k = tuple(ex["keys"][b])
        o0, o1 = ex["offsets"][b], ex["offsets"][b + 1]
        out[k] = (o0, o1)
    return out


@pytest.mark.parametrize("precision", ["f64", "f32s"])
def test_welford_equals_two_pass(precision):
    """Five noisy views: D == mean of the per-frame d, S2 / W == population variance (numpy two-pass), W == count."""
    wl = synth.tiny(noise=True)
    K = oracle.pinhole_from(wl)
    frames = [synth.render_depth(wl, 0, seed=s) for s in range(5)]
    multi = oracle.OracleMap(oracle.params_from(wl, precision, **NO_RELEVEL))
    singles = []
    for depth, rgb, T in frames:
        multi.integrate_depth(K, T, depth, rgb)
        s = oracle.OracleMap(oracle.params_from(wl, precision, **NO_RELEVEL))
        s.integrate_depth(K, T, depth, rgb)
        singles.append(s.extract())
    ex = multi.extract()
    idx = _per_voxel(ex)
    nv = ex["offsets"][-1]
    samples = np.full((5, nv), np.nan)
    for f, sx in enumerate(singles):
        for b in range(len(sx["levels"])):
            k = tuple(sx["keys"][b])
            o0, o1 = idx[k]
            s0, s1 = sx["offsets"][b], sx["offsets"][b + 1]
            w = sx["W"][s0:s1]
            samples[f, o0:o1] = np.where(w > 0, sx["D"][s0:s1], np.nan)
    cnt = np.sum(~np.isnan(samples), axis=0)
    np.testing.assert_array_equal(ex["W"], cnt)
    obs = cnt > 0
    mean = np.nanmean(samples[:, obs], axis=0)
    var = np.nanvar(samples[:, obs], axis=0)
    atol_d, atol_v = (1e-15, 1e-18) if precision == "f64" else (2e-7, 2e-12)
    np.testing.assert_allclose(ex["D"][obs], mean, rtol=0, atol=atol_d)
    np.testing.assert_allclose(ex["S2"][obs] / ex["W"][obs], var, rtol=1e-9 if precision == "f64" else 2e-4,
                               atol=atol_v)
    assert np.all(ex["S2"] >= 0)
    assert (var > 1e-8).sum() > 1000


def test_weights_monotone_and_variance_nonnegative():
    wl = synth.tiny(noise=True)
    K = oracle.pinhole_from(wl)
    m = oracle.OracleMap(oracle.params_from(wl, "f32s", **NO_RELEVEL))
    prev = None
    for s in range(4):
        depth, rgb, T = synth.render_depth(wl, 0, seed=s)
        m.integrate_depth(K, T, depth, rgb)
        ex = m.extract()
        assert np.all(ex["S2"] >= 0)
        if prev is not None:
            idx = _per_voxel(ex)
            for b in range(len(prev["levels"])):
                o0, o1 = idx[tuple(prev["keys"][b])]
                p0, p1 = prev["offsets"][b], prev["offsets"][b + 1]
                assert np.all(ex["W"][o0:o1] >= prev["W"][p0:p1])
        prev = ex


def test_repeated_noise_free_views_have_zero_variance_and_merge():
    """Identical noise-free views: S2 stays exactly 0, and once every observed voxel has W >= k_min all observed
    blocks merge to the coarser level (Sec. 3.2.1 merge rule with v_bar = 0 < theta)."""
    wl = synth.tiny(noise=False)
    K = oracle.pinhole_from(wl)
    depth, rgb, T = synth.render_depth(wl, 0)
    m = oracle.OracleMap(oracle.params_from(wl, "f32s"))
    for f in range(wl.min_obs):
        st = m.integrate_depth(K, T, depth, rgb)
        ex = m.extract()
        assert np.all(ex["S2"] == 0.0)
        if f < wl.min_obs - 1:
            assert st["merged"] == 0 and np.all(ex["levels"] == 0)
    bs = m.block_stats()
    observed = bs["n_obs"] > 0
    assert st["merged"] == observed.sum() > 1000
    assert np.all(bs["levels"][observed] == 1) and np.all(bs["levels"][~observed] == 0)


def test_fp16_storage_rounds_d_and_colour():
    wl = synth.tiny(noise=True)
    K = oracle.pinhole_from(wl)
    depth, rgb, T = synth.render_depth(wl, 0)
    m16 = oracle.OracleMap(oracle.params_from(wl, "f32s", fp16=True, **NO_RELEVEL))
    m32 = oracle.OracleMap(oracle.params_from(wl, "f32s", fp16=False, **NO_RELEVEL))
    m16.integrate_depth(K, T, depth, rgb)
    m32.integrate_depth(K, T, depth, rgb)
    a, b = m16.extract(), m32.extract()
    np.testing.assert_array_equal(a["W"], b["W"])
    np.testing.assert_array_equal(a["D"], b["D"].astype(np.float32).astype(np.float16).astype(np.float64))
    np.testing.assert_array_equal(a["C"], b["C"].astype(np.float32).astype(np.float16).astype(np.float64))


# ---------------------------------------------------------------------------------------------------------- LiDAR

def _lidar_wl():
    wl = synth.lidar()
    wl.fp16 = False
    return wl


@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f32s", 2e-6)])
def test_lidar_normal_incidence_is_plane_sdf(precision, tol):
    """One point 10 m ahead on +x: every crossed voxel gets d = clip(10 - x_centre, tau), the exact signed distance
    to the plane x = 10 (Eq. 1 with n = +x), and the crossed voxels are one row along x covering the band."""
    wl = _lidar_wl()
    m = oracle.OracleMap(oracle.params_from(wl, precision, **NO_RELEVEL))
    T = np.eye(4)
    m.integrate_points(T, np.array([[10.0, 0.0, 0.0]], np.float32))
    ex = m.extract()
    x, _ = analytic.voxel_centres(ex, wl)
    obs = ex["W"] > 0
    v0 = float(np.float32(wl.base_voxel)) / 4
    assert np.all(np.abs(x[obs, 1] - v0 / 2) < 1e-9) and np.all(np.abs(x[obs, 2] - v0 / 2) < 1e-9)
    xs = np.sort(x[obs, 0])
    assert xs[0] <= 10 - wl.truncation + v0 and xs[-1] >= 10 + wl.truncation - v0
    np.testing.assert_allclose(np.diff(xs), v0, atol=1e-9)
    tau = np.float32(wl.truncation)
    np.testing.assert_allclose(ex["D"][obs], np.clip(10.0 - x[obs, 0], -tau, tau), rtol=0, atol=tol)


def test_lidar_along_ray_values_match_geometry():
    """A small noise-free scan: each observed voxel's D is the mean over crossing rays of (p - x) . n, clipped.
    With a single scan and the ground plane only, we check the single-observation voxels against that formula
    evaluated independently in float64, within the float rounding of the ray's length and direction."""
    wl = _lidar_wl()
    wl.n_beams, wl.n_azimuth = 16, 64
    wl.range_noise = 0.0
    prims = synth.lidar_scene(2)[:1]  # ground plane only
    xyz, T = synth.render_lidar(wl, 0, scene=prims)
    m = oracle.OracleMap(oracle.params_from(wl, "f64", **NO_RELEVEL))
    st = m.integrate_points(T, xyz)
    assert st["valid_rays"] > 0
    ex = m.extract()
    x, _ = analytic.voxel_centres(ex, wl)
    one = ex["W"] == 1
    o = T[:3, 3]
    p = xyz.astype(np.float64) + o
    ok = np.isfinite(p[:, 0])
    p = p[ok]
    n = (p - o) / np.linalg.norm(p - o, axis=1, keepdims=True)
    # for each single-observation voxel find the rays whose band passes within half a voxel diagonal; the value
    # must equal clip((p - x) . n) for one of them
    tau = float(np.float32(wl.truncation))  # the map takes tau as a float
    xv = x[one]
    dvals = ex["D"][one]
    proj = (p[None, :, :] - xv[:, None, :])
    along = np.einsum("vrk,rk->vr", proj, n)
    perp = np.linalg.norm(proj - along[..., None] * n[None], axis=2)
    # the cell walk runs on endpoints rounded to 1/65536 of a block, so allow that much extra distance
    near = perp < np.sqrt(3) * wl.voxel0 / 2 + 2 * 0.4 / 65536
    err = np.where(near, np.abs(np.clip(along, -tau, tau) - dvals[:, None]), np.inf).min(axis=1)
    # the map takes the ray's length and direction in float (double only for the pose and the band's end points):
    # |d error| <= float rounding of rho (2 ulp) + |x - o| times that of the direction (3 ulp), < 6 * 2^-24 * range
    rng = np.linalg.norm(p - o, axis=1).max()
    assert np.all(err < 6 * 2.0 ** -24 * rng)
    assert np.median(err) < 1e-6
