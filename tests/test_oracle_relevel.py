"""Pins for re-levelling (Sec. 3.2.1 merge; split is the inverse extension) and the raycast of the adaptive grid.

Merge and split payloads are readings of the paper; what pins them is exactness on linear distance fields (the mean
of 8 symmetric children is the value at the parent centre; trilinear interpolation reproduces a linear field), the
variance bookkeeping (sigma^2 pooled with weights W, S2 = sigma^2 W_max), and the noise-free raycast of analytic
geometry.
"""
import numpy as np
import pytest

import oracle
import synth
from tests import analytic


def _grid(n):
    i = np.arange(n ** 3)
    return np.stack([i % n, (i // n) % n, i // (n * n)], axis=1).astype(np.float64)


@pytest.fixture(scope="module")
def rgbd_map():
    wl = synth.rgbd()
    return wl, oracle.OracleMap(oracle.params_from(wl, "f64"))


@pytest.mark.parametrize("level", [0, 1])
def test_merge_of_linear_field_is_exact(rgbd_map, level):
    wl, m = rgbd_map
    n = 8 >> level
    g = _grid(n) + 0.5                       # fine centres in fine-voxel units
    a = np.array([0.013, -0.021, 0.007])
    D = g @ a + 0.004
    rng = np.random.default_rng(level)
    W = rng.integers(1, 9, n ** 3).astype(np.float64)
    sig2 = rng.uniform(0, 1e-5, n ** 3)
    S2 = sig2 * W
    C = np.stack([g[:, 0] * 3.0, g[:, 1] * 2.0, 100 + g[:, 2]], axis=1)
    W_eq = np.full(n ** 3, 5.0)
    out_eq = m.resample_block(level, +1, D, W_eq, sig2 * W_eq, C)
    gc = _grid(n // 2) * 2 + 1.0            # coarse centres in fine-voxel units
    np.testing.assert_allclose(out_eq["D"], gc @ a + 0.004, rtol=0, atol=1e-15)
    np.testing.assert_allclose(out_eq["C"][:, 0], gc[:, 0] * 3.0, rtol=0, atol=1e-12)
    # unequal weights: weighted pooling, W = max child weight, S2 = pooled sigma^2 * W
    out = m.resample_block(level, +1, D, W, S2, C)
    for c in range(len(gc)):
        ch = np.where(np.all(np.floor(g / 2) == np.floor(gc[c] / 2), axis=1))[0]
        assert len(ch) == 8
        w = W[ch]
        assert out["W"][c] == w.max()
        np.testing.assert_allclose(out["D"][c], (w * D[ch]).sum() / w.sum(), rtol=1e-14)
        np.testing.assert_allclose(out["S2"][c], (S2[ch].sum() / w.sum()) * w.max(), rtol=1e-14)


def test_merge_skips_unobserved_children(rgbd_map):
    wl, m = rgbd_map
    D = np.full(512, 0.05)
    W = np.zeros(512)
    W[0] = 2.0                               # one observed child in coarse voxel 0
    D[1:] = 9.0                              # unobserved garbage must not leak
    out = m.resample_block(0, +1, D, W, np.zeros(512))
    assert out["W"][0] == 2.0 and out["D"][0] == 0.05
    assert np.all(out["W"][1:] == 0) and np.all(out["D"][1:] == 0)


@pytest.mark.parametrize("level", [1, 2])
def test_split_of_linear_field_is_exact_inside(rgbd_map, level):
    wl, m = rgbd_map
    n = 8 >> level
    gc = _grid(n)
    a = np.array([0.011, 0.017, -0.005])
    D = (gc + 0.5) @ a * 2 - 0.03           # linear in fine-voxel units (coarse centre = 2 (i + 0.5))
    W = np.arange(1, n ** 3 + 1, dtype=np.float64)
    S2 = 0.25 * W
    out = m.resample_block(level, -1, D, W, S2)
    gf = _grid(2 * n)
    expected = (gf + 0.5) @ a - 0.03
    interior = np.all((gf >= 1) & (gf <= 2 * n - 2), axis=1)
    np.testing.assert_allclose(out["D"][interior], expected[interior], rtol=0, atol=1e-15)
    parent = (np.floor(gf[:, 0] / 2) + n * (np.floor(gf[:, 1] / 2) + n * np.floor(gf[:, 2] / 2))).astype(int)
    np.testing.assert_array_equal(out["W"], W[parent])
    np.testing.assert_array_equal(out["S2"], S2[parent])


def test_merge_then_split_of_linear_field_round_trips(rgbd_map):
    wl, m = rgbd_map
    g = _grid(8) + 0.5
    a = np.array([0.002, 0.003, -0.004])
    D = g @ a
    W = np.full(512, 3.0)
    up = m.resample_block(0, +1, D, W, np.zeros(512))
    down = m.resample_block(1, -1, up["D"], up["W"], up["S2"])
    interior = np.all((g >= 1.5) & (g <= 6.5), axis=1)
    np.testing.assert_allclose(down["D"][interior], D[interior], rtol=0, atol=1e-15)


def _tiny_normals(wl, z, u, v):
    """Analytic unit normals of the tiny scene (sphere or room wall) at the pixel hits, and the unit pixel rays."""
    q = np.stack([(u - wl.cx) / wl.fx, (v - wl.cy) / wl.fy, np.ones_like(u, dtype=np.float64)], -1)
    X = q * z[..., None]
    c = np.array([0.0, 0.0, 1.5])
    on_sphere = np.abs(np.linalg.norm(X - c, axis=-1) - 0.5) < 1e-6
    n = np.where(on_sphere[..., None], (X - c) / 0.5, 0.0)
    for a, (lo, hi) in enumerate([(-1.5, 1.5), (-1.5, 1.5), (0.0, 3.0)]):
        on = (~on_sphere) & ((np.abs(X[..., a] - lo) < 1e-6) | (np.abs(X[..., a] - hi) < 1e-6))
        e = np.zeros(3)
        e[a] = 1.0
        n = np.where(on[..., None], e, n)
    return n, q / np.linalg.norm(q, axis=-1, keepdims=True), np.linalg.norm(q, axis=-1)


def test_noise_free_raycast_matches_analytic_depth():
    """One noise-free tiny frame, raycast from the same pose: the depth follows the true surface. Eq. 2 reads the
    range of the voxel's nearest pixel, whose ray is up to half a pixel diagonal (delta = 0.71 / f rad) off the
    voxel's own direction; on a surface at incidence theta that shifts the zero crossing by at most
    rho tan(theta) delta. On the curved sphere the nearest-pixel range also differs by the sag of one pixel footprint,
    (z / f)^2 / R = 0.14 mm at z = 1 m. Every hit pixel away from depth edges stays inside rho tan(theta) delta plus
    0.25 mm; on the flat, head-on back wall near the optical axis the depth is exact to 20 um."""
    wl = synth.tiny(noise=False)
    m = oracle.OracleMap(oracle.params_from(wl, "f64"))
    K = oracle.pinhole_from(wl)
    depth, rgb, T = synth.render_depth(wl, 0)
    m.integrate_depth(K, T, depth, rgb)
    rc = m.raycast(K, T)
    u, v = np.meshgrid(np.arange(wl.width), np.arange(wl.height))
    z_true = analytic.pixel_z_depth(wl, wl.scene(), T, u.ravel(), v.ravel()).reshape(depth.shape)
    hit = rc > 0
    assert hit.mean() > 0.97
    n, rhat, qn = _tiny_normals(wl, z_true, u, v)
    cos = np.clip(np.abs(np.sum(n * rhat, -1)), 1e-6, 1.0)
    tan = np.sqrt(1 - cos ** 2) / cos
    bound = z_true * qn * tan * (0.71 / wl.fx) + 2.5e-4
    zpad = np.pad(z_true, 1, mode="edge")
    jump = np.max(np.abs(np.stack([zpad[1:-1, 2:], zpad[1:-1, :-2], zpad[2:, 1:-1], zpad[:-2, 1:-1]]) - z_true), 0)
    sel = hit & (jump < 0.02) & (cos > 0.3)
    assert sel.sum() > 12000
    assert np.all(np.abs(rc - z_true)[sel] <= bound[sel])
    # room only: the back wall z = 3 is a fronto-parallel plane
    room = wl.scene()[:1]
    m2 = oracle.OracleMap(oracle.params_from(wl, "f64"))
    depth2, rgb2, _ = synth.render_depth(wl, 0, scene=room)
    m2.integrate_depth(K, T, depth2, rgb2)
    rc2 = m2.raycast(K, T)
    centre = (np.abs(u - wl.cx) < 10) & (np.abs(v - wl.cy) < 10)
    assert np.all(rc2[centre] > 0)
    assert np.max(np.abs(rc2[centre] - 3.0)) < 2e-5


def test_raycast_misses_when_map_is_empty():
    wl = synth.tiny(noise=False)
    m = oracle.OracleMap(oracle.params_from(wl, "f32s"))
    assert np.all(m.raycast(oracle.pinhole_from(wl), np.eye(4)) == 0)
