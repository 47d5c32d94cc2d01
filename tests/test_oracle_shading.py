"""Pins for the raycast's surface attributes (normal and colour at the hit; the rendering branch of Fig. 2).

The paper renders through splats and defines neither, so both are readings: the normal is the normalised gradient of
the same trilinear interpolant whose zero crossing gives the depth, and the colour is the trilinear mean of the
stored voxel colours at the hit. What pins them independently of the oracle's own code:
- a TSDF and a colour that are linear in space, written block by block: the trilinear interpolant of a linear field is
  that field, so the hit depth is the ray-plane intersection, the normal is the plane's unit normal and the colour is
  the colour field at the intersection, in closed form, at every level;
- a frame of one constant colour: every observed voxel's running mean equals it, so every shaded pixel shows it;
- fused noise-free frames of the analytic scene: unit normals facing the camera away from depth edges.
"""
import numpy as np
import pytest

import oracle
import synth

E = 0.08                                     # block edge of the RGB-D configuration (8 voxels of 1 cm)
N_HAT = np.array([0.25, -0.15, -1.0]) / np.linalg.norm([0.25, -0.15, -1.0])   # points towards the camera
P0 = np.array([0.02, -0.01, 1.0])
C0 = np.array([120.0, 80.0, 160.0])
GC = np.array([[100.0, 0.0, 20.0], [0.0, -80.0, 10.0], [30.0, 30.0, -40.0]])   # colour gradient per channel [1/m]


def _pinhole():
    K = oracle.Pinhole()
    K.fx = K.fy = 200.0
    K.cx, K.cy = 16.0, 12.0
    K.width, K.height = 32, 24
    K.min_depth, K.max_depth = 0.1, 3.0
    return K


def _linear_map(precision, level):
    """Blocks x, y in [-2, 1], z in [10, 14] (the slab 0.8 m <= z < 1.2 m) at ``level``, D = n.(x - p0), W = 1,
    colour C0 + GC x, all sampled at the voxel centres of that level."""
    m = oracle.OracleMap(oracle.params_from(synth.rgbd(), precision))
    n = 8 >> level
    vl = 0.01 * (1 << level)
    i = np.arange(n ** 3)
    loc = np.stack([i % n, (i // n) % n, i // (n * n)], axis=1) + 0.5
    for bx in range(-2, 2):
        for by in range(-2, 2):
            for bz in range(10, 15):
                X = np.array([bx, by, bz]) * E + loc * vl
                D = (X - P0) @ N_HAT
                C = C0 + X @ GC.T
                m.set_block((bx, by, bz), level, D, np.ones(n ** 3), None, C)
    return m


def _expected(K):
    u, v = np.meshgrid(np.arange(K.width), np.arange(K.height))
    q = np.stack([(u - K.cx) / K.fx, (v - K.cy) / K.fy, np.ones(u.shape)], -1)
    z = (P0 @ N_HAT) / (q @ N_HAT)           # z-depth of the ray-plane intersection (q_z = 1)
    X = q * z[..., None]
    return z, X


@pytest.mark.parametrize("precision,atol_z,atol_n", [("f64", 1e-7, 1e-7), ("f32s", 3e-6, 2e-5)])  # outputs are float32
@pytest.mark.parametrize("level", [0, 1, 2])
def test_linear_field_gives_plane_depth_normal_and_colour(precision, atol_z, atol_n, level):
    K = _pinhole()
    m = _linear_map(precision, level)
    d, nrm, rgb = m.raycast(K, np.eye(4), normals=True, rgb=True)
    z, X = _expected(K)
    assert np.all(d > 0)
    np.testing.assert_allclose(d, z, rtol=0, atol=atol_z)
    np.testing.assert_allclose(nrm, np.broadcast_to(N_HAT, nrm.shape), rtol=0, atol=atol_n)
    c = C0 + X @ GC.T
    ref = np.floor(c + 0.5)
    diff = np.abs(rgb.astype(np.float64) - ref)
    if precision == "f64":
        assert np.all(diff == 0)
    else:                                    # float rounding may move a value across .5
        near = np.abs(c + 0.5 - np.round(c + 0.5)) < 1e-3
        assert np.all(diff[~near] == 0) and np.all(diff <= 1)


def test_linear_field_misses_without_normal_or_colour():
    """Rays that leave the allocated slab without a crossing report depth 0, normal 0 and colour 0."""
    K = _pinhole()
    m = _linear_map("f32s", 0)
    T = np.eye(4)
    T[:3, 3] = [0.0, 0.0, 2.0]               # camera behind the slab, looking away from it
    d, nrm, rgb = m.raycast(K, T, normals=True, rgb=True)
    assert np.all(d == 0) and np.all(nrm == 0) and np.all(rgb == 0)


@pytest.mark.parametrize("fp16", [False, True])
def test_constant_colour_frame_is_rendered_exactly(fp16):
    wl = synth.tiny(noise=False)
    m = oracle.OracleMap(oracle.params_from(wl, "f32s", fp16=fp16))
    K = oracle.pinhole_from(wl)
    depth, rgb, T = synth.render_depth(wl, 0)
    col = np.empty_like(rgb)
    col[...] = (200, 100, 50)
    m.integrate_depth(K, T, depth, col)
    d, nrm, out = m.raycast(K, T, normals=True, rgb=True)
    shaded = np.linalg.norm(nrm, axis=-1) > 0
    assert shaded.mean() > 0.95
    assert np.all(out[shaded] == (200, 100, 50))
    assert np.all(out[~shaded] == 0)


def test_fused_frame_normals_are_unit_and_face_the_camera():
    """On a fused noise-free frame every shaded normal has unit length and points back along the ray. (At scales
    below one pixel footprint the projective distance of Eq. 2 is the range to a constant per-pixel value, whose
    gradient runs along the ray, so the normal of a fused surface leans from the surface normal towards the viewing
    direction; the sphere, whose footprint is close to the voxel size, keeps it within a few degrees on average.)"""
    wl = synth.tiny(noise=False)
    m = oracle.OracleMap(oracle.params_from(wl, "f32s"))
    K = oracle.pinhole_from(wl)
    depth, rgb, T = synth.render_depth(wl, 0)
    m.integrate_depth(K, T, depth, rgb)
    d, nrm = m.raycast(K, T, normals=True)
    shaded = np.linalg.norm(nrm, axis=-1) > 0
    assert np.all(d[shaded] > 0)
    np.testing.assert_allclose(np.linalg.norm(nrm[shaded], axis=-1), 1.0, atol=3e-7)
    u, v = np.meshgrid(np.arange(wl.width), np.arange(wl.height))
    q = np.stack([(u - wl.cx) / wl.fx, (v - wl.cy) / wl.fy, np.ones(u.shape)], -1)
    q /= np.linalg.norm(q, axis=-1, keepdims=True)
    # away from depth edges (room corners, sphere silhouette), where the band mixes two surfaces
    zpad = np.pad(depth, 1, mode="edge")
    jump = np.max(np.abs(np.stack([zpad[1:-1, 2:], zpad[1:-1, :-2], zpad[2:, 1:-1], zpad[:-2, 1:-1]]) - depth), 0)
    smooth = shaded & (jump < 0.02)
    assert smooth.sum() > 12000
    assert np.all(np.sum(nrm * q, -1)[smooth] < 0)
    # sphere pixels seen near head-on: mean angle to the analytic normal
    X = q * (d / q[..., 2])[..., None]
    rad = X - np.array([0.0, 0.0, 1.5])
    on = shaded & (np.abs(np.linalg.norm(rad, axis=-1) - 0.5) < 0.01)
    rad = rad / np.linalg.norm(rad, axis=-1, keepdims=True)
    head_on = on & (-np.sum(rad * q, -1) > 0.7)
    assert head_on.sum() > 2000
    ang = np.degrees(np.arccos(np.clip(np.sum(nrm * rad, -1), -1, 1)))[head_on]
    assert ang.mean() < 8.0
