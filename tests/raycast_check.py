"""Comparison of a library raycast with the CPU oracle's raycast (the rendering branch of Fig. 2).

The oracle computes the definition: on the sample grid t_j = t_min + j h, h = min(v_0, tau / 2), the first two
consecutive samples that both have a field with F_j > 0 >= F_j+1 bracket the crossing, narrowed to convergence by
bisection, in double. The kernel reaches the same bracket with fewer samples and narrows it by three bisections and a
linear root, in float. The bounds this gives:
- the same bracket: the kernel's crossing and the oracle's lie in the same last bracket of width h / 8 (the oracle's
  bisection continues inside the bracket where the kernel's stopped; a sign decision at a midpoint with |F| near
  float rounding can only move the result next to that midpoint), so |dz| <= h / 8 plus float rounding of the
  position (2e-6 z);
- a different bracket: a stride through truncated free space that passed a thin negative dip, or a float / double
  disagreement on whether a sample near a block face or a grid sample near F = 0 has a field or a sign: counted,
  together with hit / miss disagreements, against an allowance of 0.1 % of the pixels;
- typical accuracy: the linear root of a bracket of h / 8 is within 1e-4 of the depth except where the field bends
  sharply inside it (a cell face, two roots): at least 98 % of the common hits.
Normals and colours are compared at the kernel's own hit point (the oracle's probe hook evaluates its normal and
colour there), so they check the shading and not the root: the shaded / unshaded decision agrees on all but 0.1 % of
the hits, normals within 1e-4 on 99.5 % of them (1e-7 m of position rounding moves the gradient by far less; the
exceptions are points within that distance of a cell face, where the trilinear gradient jumps), colours within 1.
"""
import numpy as np


def grid_step(wl) -> float:
    v0 = np.float32(np.float32(wl.base_voxel) / np.float32(2 ** (wl.n_levels - 1)))
    return float(min(np.float64(v0), 0.5 * np.float64(np.float32(wl.truncation))))


def pixel_rays(K, T):
    """Unit pixel rays of a pinhole in the camera (rc) and world (r) frames, double, for every pixel (v, u)."""
    u, v = np.meshgrid(np.arange(K.width, dtype=np.float64), np.arange(K.height, dtype=np.float64))
    qx = (u - np.float64(np.float32(K.cx))) / np.float64(np.float32(K.fx))
    qy = (v - np.float64(np.float32(K.cy))) / np.float64(np.float32(K.fy))
    nq = np.sqrt(qx * qx + qy * qy + 1.0)
    rc = np.stack([qx / nq, qy / nq, 1.0 / nq], -1)
    r = rc @ np.asarray(T, np.float64)[:3, :3].T
    return rc, r


def check_raycast(rc_g, rc_o, h, max_mismatch=1e-3, typical=0.98):
    rc_g = np.asarray(rc_g, np.float64)
    rc_o = np.asarray(rc_o, np.float64)
    hit_g, hit_o = rc_g > 0, rc_o > 0
    both = hit_g & hit_o
    assert both.sum() > 0.5 * hit_o.sum()
    err = np.abs(rc_g - rc_o)
    same = both & (err <= h / 8.0 + 2e-6 * rc_o)
    other = np.mean(hit_g != hit_o) + np.mean(both & ~same)
    assert other <= max_mismatch, (np.mean(hit_g != hit_o), np.mean(both & ~same))
    close = np.mean(err[same] <= 1e-4 * rc_o[same])
    assert close >= typical, close
    return {"mismatch": float(other), "within_1e-4": float(close), "max_same_bracket": float(err[same].max(initial=0))}


def check_shading(out_g, omap, K, T):
    """out_g = (depth, normal[, rgb]) from the library; the oracle's normal and colour at the library's hit points."""
    depth = np.asarray(out_g[0], np.float64)
    hit = depth > 0
    rc, r = pixel_rays(K, T)
    t = depth[hit] / rc[hit][:, 2]
    x = np.asarray(T, np.float64)[:3, 3] + t[:, None] * r[hit]
    _, _, n_o, c_o = omap.probe(x)
    n_g = np.asarray(out_g[1])[hit]
    sh_g, sh_o = np.any(n_g != 0, -1), np.any(n_o != 0, -1)
    assert np.mean(sh_g != sh_o) <= 1e-3, np.mean(sh_g != sh_o)
    both = sh_g & sh_o
    assert both.mean() > 0.9
    np.testing.assert_allclose(np.linalg.norm(n_g[both], axis=-1), 1.0, atol=1e-6)
    dn = np.abs(n_g[both] - n_o[both]).max(-1)
    assert np.mean(dn <= 1e-4) >= 0.995, np.mean(dn <= 1e-4)
    if len(out_g) > 2:
        c_g = np.asarray(out_g[2])[hit][both].astype(np.int32)
        dc = np.abs(c_g - c_o[both].astype(np.int32)).max(-1)
        assert np.mean(dc <= 1) >= 0.999, np.mean(dc <= 1)
        assert np.mean(dc == 0) > 0.99
