"""Pins for the raycast's search (the rendering branch of Fig. 2; the paper gives no raycaster, so the definition is a
reading): the first +/- crossing of the trilinear TSDF along the pixel ray, found on the grid t_j = t_min + j h
(h = min(v_0, tau / 2); a level-l block sampled every 2^l grid steps from its first sample), then narrowed to
convergence.

What pins the search independently of the oracle's own march:
- isolated negative voxels ("pockets") in front of a wall: on a ray through a pocket's voxel centre along an axis the
  trilinear field is tau (2 |s| / v_0 - 1) at distance s from the centre, so it is non-positive on a closed segment
  of length v_0 = h that always holds a grid sample, and the crossing is half a voxel before the centre, in closed
  form, whatever the grid's alignment; a search that skips samples misses some pockets and reports the wall;
- a brute force over every grid sample of the ray (no jumps over unallocated blocks, the field read point by point
  through the oracle's probe hook): on a fused noisy frame from another pose, the oracle's crossing lies in the first
  bracket of consecutive valid samples and it misses exactly where the brute force finds none;
- a pocket in the second voxel layer after an unallocated stretch: found exactly when the first grid sample past the
  entry face has a field (closed form per grid alignment);
- positive blocks, a gap (a missing block, or unobserved voxels), negative blocks: no crossing (no two consecutive
  samples with a field straddle the gap);
- mutation tests: copies of the oracle source with one planted mistake each (a skipped sample, a jump that lands one
  sample late, a bracket across a sample without a field) are compiled and each fails one of these pins.
"""
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
import synth

TAU = 0.08          # tiny configuration: 1 / 2 cm levels, tau = 8 cm
V0 = np.float64(np.float32(np.float32(0.02) / np.float32(2.0)))
H = min(V0, 0.5 * np.float64(np.float32(TAU)))
WALL_Z = 1.0        # D = -tau from z = 1.0 m on
POCKETS = [(2, 3, 60), (5, 5, 70), (1, 6, 75), (6, 2, 81)]   # voxel (i, j, k) of a pocket, k along z (level 0)
ENTRY_POCKET = (3, 4, 33)   # second voxel layer of the first allocated block (its entry face is z = 0.32 m)


def _one_ray_camera(x, y, z0, min_depth=0.05):
    """A 1 x 1 pinhole whose only ray runs along +z from (x, y, z0)."""
    K = oracle.Pinhole()
    K.fx = K.fy = 100.0
    K.cx = K.cy = 0.0
    K.width = K.height = 1
    K.min_depth, K.max_depth = min_depth, 2.0
    T = np.eye(4)
    T[:3, 3] = [x, y, z0]
    return K, T


def _pocket_map():
    """Level-0 blocks over x, y in [0, 8 cm), z in [0.32, 1.2 m): D = +tau before the wall, -tau from it, W = 1; the
    voxels in POCKETS hold -tau."""
    m = oracle.OracleMap(oracle.params_from(synth.tiny(), "f64"))
    n = 8
    i = np.arange(n ** 3)
    loc = np.stack([i % n, (i // n) % n, i // (n * n)], axis=1)
    for bz in range(4, 15):
        z_c = (bz * n + loc[:, 2] + 0.5) * V0
        D = np.where(z_c < WALL_Z, TAU, -TAU)
        for (pi, pj, pk) in POCKETS + [ENTRY_POCKET]:
            if pk // n == bz:
                D[(loc[:, 0] == pi) & (loc[:, 1] == pj) & (loc[:, 2] == pk % n)] = -TAU
        m.set_block((0, 0, bz), 0, D, np.ones(n ** 3))
    # a second column of blocks with a gap: positive at z in [0.32, 0.56), nothing in [0.56, 0.64), negative behind
    for bz in list(range(4, 7)) + list(range(8, 15)):
        m.set_block((1, 0, bz), 0, np.full(n ** 3, TAU if bz < 7 else -TAU), np.ones(n ** 3))
    # a third column, allocated throughout: positive before z = 0.56, unobserved (W = 0) up to 0.64, negative behind
    for bz in range(4, 15):
        z_c = (bz * n + loc[:, 2] + 0.5) * V0
        hole = (z_c > 0.56) & (z_c < 0.64)
        m.set_block((2, 0, bz), 0, np.where(z_c < 0.56, TAU, np.where(hole, 0.0, -TAU)), np.where(hole, 0.0, 1.0))
    return m


def check_pockets(m):
    """Every pocket is found, at half a voxel before its centre, for five grid alignments each."""
    for (pi, pj, pk) in POCKETS:
        cx, cy, cz = (pi + 0.5) * V0, (pj + 0.5) * V0, (pk + 0.5) * V0
        for k in range(5):
            z0 = 0.1 + k * H / 5.0
            K, T = _one_ray_camera(cx, cy, z0)
            d = float(m.raycast(K, T)[0, 0])
            assert abs(d - (cz - 0.5 * V0 - z0)) < 1e-7, (pi, pj, pk, k, d, cz - 0.5 * V0 - z0)


def check_entry_pocket(m):
    """A ray along z through ENTRY_POCKET's column enters the allocated blocks at z = 0.32 m. The field exists from
    the first voxel centre (0.325 m) on, is positive up to 0.33 m and non-positive on [0.33, 0.34]: the crossing at
    0.33 m is found when the first grid sample past the entry face has a field (z >= 0.325 m), else the next samples
    sit in the pocket without a positive sample before them and the ray goes on to the wall."""
    pi, pj, pk = ENTRY_POCKET
    cx, cy = (pi + 0.5) * V0, (pj + 0.5) * V0
    for k in range(5):
        z0 = 0.1 + (k + 0.3) * H / 5.0
        K, T = _one_ray_camera(cx, cy, z0)
        first = z0 + np.float64(np.float32(K.min_depth)) + 17 * H      # first grid sample past z = 0.32
        assert 0.32 < first < 0.33
        expect = (0.33 if first >= 0.325 else WALL_Z) - z0
        d = float(m.raycast(K, T)[0, 0])
        assert abs(d - expect) < 1e-7, (k, first, d, expect)


def test_pockets_are_found_at_their_entry():
    m = _pocket_map()
    check_pockets(m)
    check_entry_pocket(m)


def check_gap(m):
    """Positive blocks, an unallocated block, negative blocks: no two consecutive samples with a field bracket a
    sign change (the field ends half a voxel before the gap and starts half a voxel after it), so the ray misses."""
    K, T = _one_ray_camera(11.5 * V0, 3.5 * V0, 0.1)
    assert float(m.raycast(K, T)[0, 0]) == 0.0


def check_hole(m):
    """The same with an unobserved stretch inside allocated blocks instead of a missing block."""
    K, T = _one_ray_camera(19.5 * V0, 3.5 * V0, 0.1)
    assert float(m.raycast(K, T)[0, 0]) == 0.0


def test_gap_between_positive_and_negative_blocks_is_no_crossing():
    m = _pocket_map()
    check_gap(m)
    check_hole(m)


def test_ray_between_pockets_reaches_the_wall():
    m = _pocket_map()
    K, T = _one_ray_camera(3.5 * V0, 0.5 * V0, 0.1)
    assert abs(float(m.raycast(K, T)[0, 0]) - (WALL_Z - 0.1)) < 1e-7


def _rays(K, T, pix):
    """Pixel rays exactly as the oracle forms them (double; pinhole fields are float32)."""
    u = (pix % K.width).astype(np.float64)
    v = (pix // K.width).astype(np.float64)
    qx = (u - np.float64(np.float32(K.cx))) / np.float64(np.float32(K.fx))
    qy = (v - np.float64(np.float32(K.cy))) / np.float64(np.float32(K.fy))
    nq = np.sqrt((qx * qx + qy * qy) + 1.0)
    rc = np.stack([qx / nq, qy / nq, 1.0 / nq], -1)
    R = T[:3, :3]
    r = np.stack([(R[a, 0] * rc[:, 0] + R[a, 1] * rc[:, 1]) + R[a, 2] * rc[:, 2] for a in range(3)], -1)
    return nq, rc, r


def brute_force_brackets(m, K, T, pix, h):
    """First bracket [t_j, t_j+1] of consecutive valid grid samples with F_j > 0 >= F_j+1 per pixel (None: none)."""
    nq, rc, r = _rays(K, T, pix)
    o = T[:3, 3]
    out = []
    for i in range(pix.size):
        t_min = np.float64(np.float32(K.min_depth)) * nq[i]
        t_max = np.float64(np.float32(K.max_depth)) * nq[i]
        j = np.arange(int((t_max - t_min) / h) + 2)
        t = t_min + j.astype(np.float64) * h
        t = t[t <= t_max]
        x = np.stack([o[a] + t * r[i, a] for a in range(3)], -1)
        F, ok, _, _ = m.probe(x)
        b = np.flatnonzero(ok[:-1] & ok[1:] & (F[:-1] > 0) & ~(F[1:] > 0))
        out.append((t[b[0]], t[b[0] + 1]) if b.size else None)
    return out, rc


def check_brute_force(m, K, T, n_pix=500, seed=3):
    pix = np.random.default_rng(seed).choice(K.width * K.height, n_pix, replace=False)
    br, rc = brute_force_brackets(m, K, T, pix, H)
    d = m.raycast_pixels(K, T, pix).astype(np.float64)
    hits = 0
    for i in range(pix.size):
        if br[i] is None:
            assert d[i] == 0.0, (i, d[i])
            continue
        hits += 1
        t = d[i] / rc[i, 2]
        # the float32 output rounds the z-depth by 2^-24 relative
        slack = 2e-7 * t
        assert br[i][0] - slack <= t <= br[i][1] + slack, (i, t, br[i])
    return hits


def _fused_tiny(precision="f32s", frames=4):
    wl = synth.tiny()
    wl.var_threshold = (-1.0,)  # every block stays at level 0: the brute force samples every grid point
    m = oracle.OracleMap(oracle.params_from(wl, precision))
    K = oracle.pinhole_from(wl)
    for s in range(frames):
        depth, rgb, T = synth.render_depth(wl, 0, seed=s)
        m.integrate_depth(K, T, depth, rgb)
    return m, K


def _side_pose():
    T = np.eye(4)
    c, s = np.cos(0.35), np.sin(0.35)
    T[:3, :3] = [[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]]
    T[:3, 3] = [-0.45, 0.05, 0.1]
    return T


@pytest.mark.parametrize("precision", ["f32s", "f64"])
def test_brute_force_search_on_a_fused_frame_from_another_pose(precision):
    m, K = _fused_tiny(precision)
    hits = check_brute_force(m, K, _side_pose())
    assert hits > 300


def brute_force_levels(m, K, T, pix, h, E, levels):
    """The same brute force on a map with coarse blocks: every grid sample is classified by its block (dict of key ->
    level); a level-l block's samples are those 2^l apart from its first grid sample; samples without a block break
    the chain of consecutive samples."""
    nq, rc, r = _rays(K, T, pix)
    o = T[:3, 3]
    out = []
    for i in range(pix.size):
        t_min = np.float64(np.float32(K.min_depth)) * nq[i]
        t_max = np.float64(np.float32(K.max_depth)) * nq[i]
        j = np.arange(int((t_max - t_min) / h) + 2)
        t = t_min + j.astype(np.float64) * h
        t = t[t <= t_max]
        x = np.stack([o[a] + t * r[i, a] for a in range(3)], -1)
        keys = np.floor(x / E).astype(np.int64)
        F, ok, _, _ = m.probe(x)
        found, prev, first = None, None, {}
        for q in range(t.size):
            k = tuple(keys[q])
            if k not in levels:
                prev = None
                continue
            q0 = first.setdefault(k, q)
            if (q - q0) % (1 << levels[k]):
                continue
            if prev is not None and ok[prev] and ok[q] and F[prev] > 0 and not F[q] > 0:
                found = (t[prev], t[q])
                break
            prev = q
        out.append(found)
    return out, rc


def test_brute_force_search_with_coarse_blocks():
    """Ten noisy views of the tiny scene, merges on: level-1 blocks are sampled at their own pitch (two grid steps)."""
    wl = synth.tiny()
    m = oracle.OracleMap(oracle.params_from(wl, "f32s"))
    K = oracle.pinhole_from(wl)
    for s in range(10):
        depth, rgb, T = synth.render_depth(wl, 0, seed=s)
        m.integrate_depth(K, T, depth, rgb)
    st = m.block_stats()
    levels = {tuple(k): int(l) for k, l in zip(st["keys"].tolist(), st["levels"].tolist())}
    assert sum(levels.values()) > 100
    E = np.float64(np.float32(V0 * 8))
    T = _side_pose()
    pix = np.random.default_rng(5).choice(K.width * K.height, 400, replace=False)
    br, rc = brute_force_levels(m, K, T, pix, H, E, levels)
    d = m.raycast_pixels(K, T, pix).astype(np.float64)
    hits = 0
    for i in range(pix.size):
        if br[i] is None:
            assert d[i] == 0.0, (i, d[i])
            continue
        hits += 1
        t = d[i] / rc[i, 2]
        assert br[i][0] - 2e-7 * t <= t <= br[i][1] + 2e-7 * t, (i, t, br[i])
    assert hits > 200


# ------------------------------------------------------------------------------------------------ mutation tests

MUTANTS = {
    # a sample skipped after every sample
    "skip_sample": ("        continue;\n      }\n      ++j;\n", "        continue;\n      }\n      j += 2;\n"),
    # the first grid sample past an unallocated block's exit face skipped
    "late_jump": ("        j = jn > j ? jn : j + 1;\n", "        j = jn + 1 > j ? jn + 1 : j + 1;\n"),
    # the last sample with a field kept across samples without one (brackets across unobserved stretches)
    "prev_validity": ("      have_prev = valid;\n      t_prev = t;\n      F_prev = F;\n",
                      "      if (valid) {\n        have_prev = true;\n        t_prev = t;\n        F_prev = F;\n      }\n"),
}


def _build_mutant(name, tmp):
    src_path = os.path.join(os.path.dirname(oracle.__file__), "mrh_oracle.cpp")
    src = open(src_path).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation site of {name} not found exactly once"
    path = os.path.join(tmp, "mrh_oracle.cpp")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    others = [s for s in oracle._SRCS if not s.endswith("mrh_oracle.cpp")]
    so = os.path.join(tmp, f"libmut_{name}.so")
    subprocess.check_call(["g++", *oracle.CFLAGS, "-o", so, path, *others])
    return so


def _pins_fail():
    failed = []
    for pin in (lambda: check_pockets(_pocket_map()), lambda: check_entry_pocket(_pocket_map()),
                lambda: check_gap(_pocket_map()), lambda: check_hole(_pocket_map()),
                lambda: check_brute_force(*_fused_tiny("f32s"), T=_side_pose())):
        try:
            pin()
        except AssertionError:
            failed.append(pin)
    return len(failed) > 0


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_search_mistake_fails_a_pin(name):
    with tempfile.TemporaryDirectory() as tmp:
        so = _build_mutant(name, tmp)
        with oracle.use_library(so):
            assert _pins_fail(), f"mutant {name} passed every pin"
