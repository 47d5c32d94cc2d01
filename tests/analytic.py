"""Analytic ground truth for the test scenes, in numpy float64 (independent of both the oracle and the library).

Ray/primitive intersection of the synthetic scenes, used to pin fused distances (Eq. 1/2) and raycast depth to the
true geometry.
"""
import numpy as np

import synth


def ray_scene_hit(prims: np.ndarray, o: np.ndarray, d: np.ndarray) -> np.ndarray:
    """Smallest s > 0 with o + s d on a primitive, for rays o (3,) and directions d (N, 3); inf where none."""
    o = np.asarray(o, dtype=np.float64)
    d = np.asarray(d, dtype=np.float64)
    best = np.full(d.shape[0], np.inf)
    for p in prims:
        kind = int(p[0])
        if kind in (synth.PRIM_ROOM, synth.PRIM_BOX):
            lo, hi = p[1:4], p[4:7]
            with np.errstate(divide="ignore", invalid="ignore"):
                ta = (lo - o) / d
                tb = (hi - o) / d
            t0 = np.nanmax(np.minimum(ta, tb), axis=1)
            t1 = np.nanmin(np.maximum(ta, tb), axis=1)
            ok = t0 <= t1
            s = np.where(ok, t1 if kind == synth.PRIM_ROOM else t0, np.inf)
        elif kind == synth.PRIM_SPHERE:
            c, r = p[1:4], p[4]
            oc = o - c
            a = np.sum(d * d, axis=1)
            b = 2.0 * (d @ oc)
            cc = oc @ oc - r * r
            disc = b * b - 4 * a * cc
            with np.errstate(invalid="ignore"):
                s = np.where(disc >= 0, (-b - np.sqrt(np.maximum(disc, 0))) / (2 * a), np.inf)
        else:
            with np.errstate(divide="ignore", invalid="ignore"):
                s = np.where(d[:, 2] < 0, -o[2] / d[:, 2], np.inf)
        s = np.where(s > 1e-9, s, np.inf)
        best = np.minimum(best, s)
    return best


def pixel_z_depth(wl, prims, T_wc, u, v):
    """Noise-free z-depth seen by pixels (u, v) of a pinhole workload (0 where no hit)."""
    q = np.stack([(np.asarray(u, np.float64) - wl.cx) / wl.fx, (np.asarray(v, np.float64) - wl.cy) / wl.fy,
                  np.ones(np.shape(u))], axis=1)
    d = q @ T_wc[:3, :3].T
    s = ray_scene_hit(prims, T_wc[:3, 3], d)
    return np.where(np.isfinite(s), s, 0.0)


def voxel_centres(ex, wl):
    """World centres (V, 3) and level (V,) of every voxel of an extract, voxel i of a side-n block at x + n(y + nz)."""
    # voxel edges are defined from the float32 base voxel (both the oracle and the library take a float)
    v0 = float(np.float32(wl.base_voxel)) / (1 << (wl.n_levels - 1))
    cents, levels = [], []
    for b in range(len(ex["levels"])):
        l = int(ex["levels"][b])
        n = 8 >> l
        vl = v0 * (1 << l)
        idx = np.arange(n ** 3)
        ijk = np.stack([idx % n, (idx // n) % n, idx // (n * n)], axis=1)
        cents.append((ex["keys"][b].astype(np.float64) * n + ijk + 0.5) * vl)
        levels.append(np.full(n ** 3, l))
    return np.concatenate(cents), np.concatenate(levels)
