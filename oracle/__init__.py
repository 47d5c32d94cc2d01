"""CPU oracle for the variance-adaptive hashed TSDF map (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg import this package. It shares no code
with the CUDA library: ``mrh_oracle.cpp`` is plain C++ compiled here with ``g++ -O2 -ffp-contract=off``.

Parity status of each function (what pins it, see ``tests/test_oracle_*.py``):
  segment cells (allocation)   pinned: brute force == ordered walk, closed forms, exact-rational spot checks
  camera fusion (Eq. 2)        pinned: analytic ranges of a sphere / plane, Euclidean bound, f64 vs f32s
  LiDAR fusion (Eq. 1)         pinned: normal-incidence plane, analytic along-ray values
  Welford (Eq. 5/6)            pinned: two-pass variance, S2 >= 0, W monotone, S2 == 0 for repeated noise-free views
  merge / split payloads       pinned on linear fields (exact); the rule itself is a reading: parity unpinned
  thresholds                   chosen values: parity unpinned
  raycast                      pinned: analytic plane / sphere depth; step constants are a reading
  mesh (Marching Cubes)        pinned: case table against brute-force checks (triangle count of the plane cases,
                               every inside corner cut off, orientation towards the outside); linear fields give
                               vertices on the plane at every level; closed single-level surfaces are watertight
                               with Euler characteristic 2; the resolution-boundary rule is a reading;
                               vertex collapse: representatives are members within their cluster cell, exact
                               duplicates only at a tiny spacing (closed sphere keeps Euler characteristic 2)
  streaming (Sec. 3.3)         pinned: nothing moves below the capacity fraction; above it exactly the blocks outside
                               the view cone / radius (checked by direct geometry) leave, and a block allocated again
                               comes back bit for bit; LiDAR and camera policies; the rule itself is a reading
  quadtree (Sec. 3.5, Eq. 10)  pinned: closed-form contrast of two-colour and constant regions (byte units);
                               leaves tile the image; thresholds below zero / above the maximum give single pixels /
                               one leaf; a hand-built image gives the hand-counted leaves
  splats (Sec. 3.5, Eqs. 7-9)  pinned: projection against the closed form on the optical axis and a finite-difference
                               Jacobian off axis; invariance under moving camera and Gaussians together; one
                               Gaussian gives a C at its centre, a exp(-q/2) C around it, nothing beyond three
                               standard deviations; two Gaussians blend in depth order whatever their index; an opaque
                               front Gaussian hides the back one; the cut-off is a reading
  raycast normal / colour      pinned: a linear TSDF and colour field set block by block gives the plane's unit
                               normal and the colour field at the hit (trilinear is exact on linear fields);
                               analytic walls of a fused noise-free frame; constant-colour frames
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mrh_oracle.cpp")
_SRCS = [_SRC, os.path.join(_HERE, "level_predictor.cpp"), os.path.join(_HERE, "quadtree.cpp"),
         os.path.join(_HERE, "splat.cpp")]
_SO = os.path.join(_HERE, "libmrh_oracle.so")
_lib = None

CFLAGS = ["-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile libmrh_oracle.so if it is missing or older than its source."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(os.path.getmtime(s) for s in _SRCS):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", *CFLAGS, "-o", tmp, *_SRCS])
        os.replace(tmp, _SO)
    return _SO


class Params(ctypes.Structure):
    _fields_ = [("base_voxel", ctypes.c_float), ("n_levels", ctypes.c_int), ("truncation", ctypes.c_float),
                ("var_threshold", ctypes.c_double * 2), ("split_hysteresis", ctypes.c_double),
                ("min_obs", ctypes.c_int), ("precision", ctypes.c_int), ("fp16", ctypes.c_int),
                ("has_color", ctypes.c_int), ("min_range", ctypes.c_float), ("max_range", ctypes.c_float)]


class Pinhole(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("width", ctypes.c_int), ("height", ctypes.c_int), ("min_depth", ctypes.c_float),
                ("max_depth", ctypes.c_float)]


class FrameStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in
                ("valid_rays", "touched", "new_blocks", "merged", "split", "fp64_rechecks", "observations",
                 "updated_voxels", "evicted", "restored")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


def _load(path: str | None = None):
    global _lib
    if path is not None or _lib is None:
        lib = ctypes.CDLL(path or build())
        vp = ctypes.c_void_p
        lib.orc_create.restype = vp
        lib.orc_create.argtypes = [ctypes.POINTER(Params)]
        lib.orc_destroy.argtypes = [vp]
        lib.orc_integrate_depth.argtypes = [vp, ctypes.POINTER(Pinhole), vp, vp, vp, ctypes.POINTER(FrameStats)]
        lib.orc_integrate_points.argtypes = [vp, vp, vp, ctypes.c_int64, ctypes.POINTER(FrameStats)]
        lib.orc_raycast.argtypes = [vp, ctypes.POINTER(Pinhole), vp, vp, vp, vp]
        lib.orc_raycast_pixels.argtypes = [vp, ctypes.POINTER(Pinhole), vp, ctypes.c_int64, vp, vp, vp, vp]
        lib.orc_probe_points.argtypes = [vp, ctypes.c_int64, vp, vp, vp, vp, vp]
        lib.orc_set_block.argtypes = [vp, vp, ctypes.c_int, vp, vp, vp, vp]
        lib.orc_extract_mesh.restype = ctypes.c_int64
        lib.orc_extract_mesh.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int64]
        lib.orc_mc_table.argtypes = [vp, vp, vp]
        lib.orc_set_streaming.argtypes = [vp, ctypes.c_float, ctypes.c_float, vp]
        lib.orc_archived.restype = ctypes.c_int64
        lib.orc_archived.argtypes = [vp]
        lib.orc_qt_contrast.restype = ctypes.c_double
        lib.orc_qt_contrast.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.orc_quadtree.restype = ctypes.c_int64
        lib.orc_quadtree.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, vp, ctypes.c_int64]
        lib.orc_splat_project.restype = ctypes.c_int
        lib.orc_splat_project.argtypes = [vp, vp, vp, vp, vp]
        lib.orc_splat_render.restype = ctypes.c_int64
        lib.orc_splat_render.argtypes = [ctypes.c_int64, vp, vp, vp, vp, vp, vp, ctypes.c_int, ctypes.c_int, vp, vp]
        lib.orc_splat_pixels.restype = ctypes.c_int64
        lib.orc_splat_pixels.argtypes = [ctypes.c_int64, vp, vp, vp, vp, vp, vp, ctypes.c_int64, vp, vp, vp]
        lib.orc_weld_mesh.restype = ctypes.c_int64
        lib.orc_weld_mesh.argtypes = [vp, ctypes.c_int64, ctypes.c_float, vp, ctypes.c_int64, vp, ctypes.c_int64,
                                      ctypes.POINTER(ctypes.c_int64)]
        lib.orc_count_blocks.restype = ctypes.c_int64
        lib.orc_count_blocks.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
        lib.orc_extract.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
        lib.orc_block_stats.argtypes = [vp, vp, vp, vp, vp, vp]
        lib.orc_segment_cells.restype = ctypes.c_int64
        lib.orc_segment_cells.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_int, vp, ctypes.c_int64]
        lib.orc_resample_block.argtypes = [vp, ctypes.c_int, ctypes.c_int] + [vp] * 8
        lib.orc_half_round.restype = ctypes.c_float
        lib.orc_half_round.argtypes = [ctypes.c_float]
        for name in ("orc_bf16_round", "orc_exp_cw", "orc_erf_as", "orc_gelu"):
            getattr(lib, name).restype = ctypes.c_float
            getattr(lib, name).argtypes = [ctypes.c_float]
        lib.orc_mlp_forward.argtypes = [vp, vp, ctypes.c_int64, vp]
        lib.orc_block_features.restype = ctypes.c_int
        lib.orc_block_features.argtypes = [ctypes.POINTER(Pinhole), vp, vp, vp, ctypes.c_float, ctypes.c_float,
                                           ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, vp, ctypes.c_int, vp, vp]
        lib.orc_lidar_block_features.argtypes = [vp, vp, ctypes.c_float, ctypes.c_float, ctypes.c_int64,
                                                 ctypes.c_int64, ctypes.c_int64, vp, ctypes.c_int, vp, vp]
        lib.orc_set_predictor.argtypes = [vp, vp, ctypes.c_int64]
        lib.orc_set_capture.argtypes = [vp, ctypes.c_int]
        lib.orc_get_features.restype = ctypes.c_int64
        lib.orc_get_features.argtypes = [vp, vp, vp, ctypes.c_int64]
        if path is not None:
            return lib
        _lib = lib
    return _lib


class use_library:
    """Test hook: maps created inside ``with oracle.use_library(path):`` run on another build of the oracle source
    (the mutation tests compile copies with one deliberate mistake each and check that a pin catches it)."""

    def __init__(self, path: str):
        self.lib = _load(path)

    def __enter__(self):
        global _lib
        self._saved, _lib = _lib, self.lib
        return self.lib

    def __exit__(self, *exc):
        global _lib
        _lib = self._saved
        return False


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def params_from(wl, precision: str = "f32s", fp16: bool | None = None, var_threshold=None, split_hysteresis=None,
                min_obs=None) -> Params:
    """Oracle parameters for a ``synth.Workload``."""
    p = Params()
    p.base_voxel = wl.base_voxel
    p.n_levels = wl.n_levels
    p.truncation = wl.truncation
    th = list(wl.var_threshold if var_threshold is None else var_threshold) + [0.0, 0.0]
    p.var_threshold[0], p.var_threshold[1] = th[0], th[1]
    p.split_hysteresis = wl.split_hysteresis if split_hysteresis is None else split_hysteresis
    p.min_obs = wl.min_obs if min_obs is None else min_obs
    p.precision = 1 if precision == "f64" else 0
    p.fp16 = int(wl.fp16 if fp16 is None else fp16) if precision != "f64" else 0
    p.has_color = int(wl.has_color)
    p.min_range, p.max_range = wl.r_min, wl.r_max
    return p


def pinhole_from(wl) -> Pinhole:
    k = Pinhole()
    k.fx, k.fy, k.cx, k.cy = wl.fx, wl.fy, wl.cx, wl.cy
    k.width, k.height = wl.width, wl.height
    k.min_depth, k.max_depth = wl.min_depth, wl.max_depth
    return k


class OracleMap:
    """One oracle map. ``precision`` is "f32s" (float, literal op order) or "f64" (double truth)."""

    def __init__(self, params: Params):
        self._lib = _load()
        self.params = params
        self._h = self._lib.orc_create(ctypes.byref(params))
        if not self._h:
            raise ValueError("invalid oracle parameters")

    def close(self):
        if self._h:
            self._lib.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def integrate_depth(self, K: Pinhole, T_wc: np.ndarray, depth: np.ndarray, rgb: np.ndarray | None = None):
        T = np.ascontiguousarray(T_wc, dtype=np.float64)
        d = np.ascontiguousarray(depth, dtype=np.float32)
        c = None if rgb is None else np.ascontiguousarray(rgb, dtype=np.uint8)
        st = FrameStats()
        self._lib.orc_integrate_depth(self._h, ctypes.byref(K), _p(T), _p(d), _p(c), ctypes.byref(st))
        return st.as_dict()

    def integrate_points(self, T_ws: np.ndarray, xyz: np.ndarray):
        T = np.ascontiguousarray(T_ws, dtype=np.float64)
        x = np.ascontiguousarray(xyz, dtype=np.float32)
        st = FrameStats()
        self._lib.orc_integrate_points(self._h, _p(T), _p(x), x.shape[0], ctypes.byref(st))
        return st.as_dict()

    def raycast(self, K: Pinhole, T_wc: np.ndarray, normals: bool = False, rgb: bool = False):
        """z-depth (h, w) float32; with normals / rgb also the unit normal (h, w, 3) float32 (world frame, towards
        positive TSDF) and the colour (h, w, 3) uint8 at the hit, zero where there is none."""
        T = np.ascontiguousarray(T_wc, dtype=np.float64)
        out = np.zeros((K.height, K.width), dtype=np.float32)
        nrm = np.zeros((K.height, K.width, 3), dtype=np.float32) if normals else None
        col = np.zeros((K.height, K.width, 3), dtype=np.uint8) if rgb else None
        self._lib.orc_raycast(self._h, ctypes.byref(K), _p(T), _p(out), _p(nrm), _p(col))
        if not (normals or rgb):
            return out
        return (out,) + ((nrm,) if normals else ()) + ((col,) if rgb else ())

    def raycast_pixels(self, K: Pinhole, T_wc: np.ndarray, pix, normals: bool = False, rgb: bool = False):
        """The raycast of the listed pixels only (flat indices v * width + u): z-depth (n,) and optionally normals
        (n, 3) and colours (n, 3), as ``raycast`` gives them for those pixels."""
        T = np.ascontiguousarray(T_wc, dtype=np.float64)
        pix = np.ascontiguousarray(pix, dtype=np.int64).ravel()
        out = np.zeros(pix.size, dtype=np.float32)
        nrm = np.zeros((pix.size, 3), dtype=np.float32) if normals else None
        col = np.zeros((pix.size, 3), dtype=np.uint8) if rgb else None
        self._lib.orc_raycast_pixels(self._h, ctypes.byref(K), _p(T), pix.size, _p(pix), _p(out), _p(nrm), _p(col))
        if not (normals or rgb):
            return out
        return (out,) + ((nrm,) if normals else ()) + ((col,) if rgb else ())

    def probe(self, xyz: np.ndarray):
        """The raycast's field at world points (n, 3): F (n,) float64, valid (n,) bool, and the unit normal (n, 3)
        and colour (n, 3) uint8 the raycast reports for a hit at each point (zeros where it reports none)."""
        x = np.ascontiguousarray(np.asarray(xyz, dtype=np.float64).reshape(-1, 3))
        n = x.shape[0]
        F = np.zeros(n)
        ok = np.zeros(n, np.int8)
        nrm = np.zeros((n, 3), np.float32)
        col = np.zeros((n, 3), np.uint8)
        self._lib.orc_probe_points(self._h, n, _p(x), _p(F), _p(ok), _p(nrm), _p(col))
        return F, ok.astype(bool), nrm, col

    def set_streaming(self, fraction: float, radius: float, max_blocks):
        """Capacity-driven streaming (Sec. 3.3): before each frame, when some level holds more than fraction of
        max_blocks[level] blocks, the blocks outside the frame's view (camera) or farther than radius [m] from the
        scan origin (LiDAR) move to the archive; a block allocated again returns from it. fraction 0 disables."""
        mb = np.ascontiguousarray(list(max_blocks) + [0] * (3 - len(max_blocks)), dtype=np.int64)
        self._lib.orc_set_streaming(self._h, fraction, radius, _p(mb))

    def archived(self) -> int:
        return int(self._lib.orc_archived(self._h))

    def extract_mesh(self) -> np.ndarray:
        """Multi-resolution Marching Cubes triangle soup (n, 3, 3) float32: blocks in key order, voxels in index
        order, triangles facing increasing distance."""
        n = self._lib.orc_extract_mesh(self._h, 1, None, 0)
        out = np.zeros((n, 3, 3), np.float32)
        self._lib.orc_extract_mesh(self._h, 0, _p(out), n)
        return out

    def set_block(self, key, level: int, D, W, S2=None, C=None):
        """Test hook: create or overwrite block ``key`` at ``level`` with the given voxel payload (x fastest)."""
        nv = (8 >> level) ** 3
        a = [np.ascontiguousarray(np.broadcast_to(np.asarray(x, dtype=np.float64), (nv,)))
             for x in (D, W, np.zeros(nv) if S2 is None else S2)]
        c = None if C is None else np.ascontiguousarray(np.broadcast_to(np.asarray(C, np.float64), (nv, 3)))
        k = np.ascontiguousarray(key, dtype=np.int32)
        if self._lib.orc_set_block(self._h, _p(k), int(level), *[_p(x) for x in a], _p(c)) != 0:
            raise ValueError("invalid level")

    def count(self):
        nv = ctypes.c_int64()
        nb = self._lib.orc_count_blocks(self._h, ctypes.byref(nv))
        return nb, nv.value

    def extract(self) -> dict:
        """All blocks sorted by key: keys (n,3) int32, levels (n,) uint8, offsets (n+1,) int64, D/W/S2 (V,) float64,
        C (V,3) float64. Voxel i of a block of side n is at x + n (y + n z)."""
        nb, nv = self.count()
        color = bool(self.params.has_color)
        out = dict(keys=np.zeros((nb, 3), np.int32), levels=np.zeros(nb, np.uint8), offsets=np.zeros(nb + 1, np.int64),
                   D=np.empty(nv), W=np.empty(nv), S2=np.empty(nv), C=np.empty((nv, 3)) if color else None)
        self._lib.orc_extract(self._h, _p(out["keys"]), _p(out["levels"]), _p(out["offsets"]), _p(out["D"]),
                              _p(out["W"]), _p(out["S2"]), _p(out["C"]))
        if not color:  # a map without colour: zeros, without the memory
            out["C"] = np.broadcast_to(np.zeros(1), (nv, 3))
        return out

    def resample_block(self, level: int, direction: int, D, W, S2, C=None) -> dict:
        """Apply the merge (direction +1) or split (direction -1) payload rule to one block of ``level``."""
        n_in = len(W)
        n_out = n_in // 8 if direction > 0 else n_in * 8
        a = [np.ascontiguousarray(x, dtype=np.float64) for x in (D, W, S2)]
        c = np.ascontiguousarray(np.zeros((n_in, 3)) if C is None else C, dtype=np.float64)
        out = dict(D=np.zeros(n_out), W=np.zeros(n_out), S2=np.zeros(n_out), C=np.zeros((n_out, 3)))
        rc = self._lib.orc_resample_block(self._h, level, direction, *[_p(x) for x in a], _p(c), _p(out["D"]),
                                          _p(out["W"]), _p(out["S2"]), _p(out["C"]))
        if rc != 0:
            raise ValueError("invalid level/direction")
        return out

    def set_predictor(self, w_bf16: np.ndarray | None):
        """Learned level predictor for later depth frames: MLP_PARAMS BF16 bit patterns (uint16), or None."""
        if w_bf16 is None:
            self._lib.orc_set_predictor(self._h, None, 0)
            return
        w = np.ascontiguousarray(w_bf16, dtype=np.uint16)
        if w.size != MLP_PARAMS:
            raise ValueError("predictor needs %d weights" % MLP_PARAMS)
        self._lib.orc_set_predictor(self._h, _p(w), w.size)

    def set_capture(self, on: bool):
        """Record (key, 16 features) of every new block of later depth frames; clears earlier records."""
        self._lib.orc_set_capture(self._h, int(bool(on)))

    def features(self):
        """Captured records sorted by key: keys (n, 3) int32, features (n, 16) float32."""
        n = self._lib.orc_get_features(self._h, None, None, 0)
        keys = np.zeros((n, 3), np.int32)
        feats = np.zeros((n, MLP_IN), np.float32)
        self._lib.orc_get_features(self._h, _p(keys), _p(feats), n)
        order = np.lexsort((keys[:, 2], keys[:, 1], keys[:, 0]))
        return keys[order], feats[order]

    def block_stats(self) -> dict:
        """Per block (sorted by key): level, mean variance over observed voxels (double), observed count, weight sum."""
        nb, _ = self.count()
        out = dict(keys=np.zeros((nb, 3), np.int32), levels=np.zeros(nb, np.uint8), vbar=np.zeros(nb),
                   n_obs=np.zeros(nb, np.int64), sum_w=np.zeros(nb, np.int64))
        self._lib.orc_block_stats(self._h, _p(out["keys"]), _p(out["levels"]), _p(out["vbar"]), _p(out["n_obs"]),
                                  _p(out["sum_w"]))
        return out


def weld_mesh(tris, delta: float):
    """Vertex collapse of a triangle soup (n, 3, 3) on a grid of spacing delta: vertices (nv, 3) float32 (each the
    smallest member of its cluster, clusters in ascending order) and faces (nf, 3) int32 (degenerate ones dropped)."""
    lib = _load()
    t = np.ascontiguousarray(tris, dtype=np.float32).reshape(-1, 9)
    nf = ctypes.c_int64()
    nv = lib.orc_weld_mesh(_p(t), t.shape[0], delta, None, 0, None, 0, ctypes.byref(nf))
    verts = np.zeros((nv, 3), np.float32)
    faces = np.zeros((nf.value, 3), np.int32)
    lib.orc_weld_mesh(_p(t), t.shape[0], delta, _p(verts), nv, _p(faces), nf.value, ctypes.byref(nf))
    return verts, faces


def qt_contrast(rgb: np.ndarray, x0: int, y0: int, w: int, h: int) -> float:
    """Contrast (Eq. 10) of the rectangle of an (H, W, 3) uint8 image, RGB in byte units."""
    img = np.ascontiguousarray(rgb, dtype=np.uint8)
    return _load().orc_qt_contrast(_p(img), img.shape[1], x0, y0, w, h)


def quadtree(rgb: np.ndarray, threshold: float = 0.1, min_size: int = 1) -> np.ndarray:
    """Leaves (n, 4) int32 (x, y, w, h) of the image's contrast quadtree (Sec. 3.5, Algorithm 1), depth first."""
    img = np.ascontiguousarray(rgb, dtype=np.uint8)
    lib = _load()
    n = lib.orc_quadtree(_p(img), img.shape[1], img.shape[0], threshold, min_size, None, 0)
    out = np.zeros((n, 4), np.int32)
    lib.orc_quadtree(_p(img), img.shape[1], img.shape[0], threshold, min_size, _p(out), n)
    return out


def _k6(K) -> np.ndarray:
    return np.array([K.fx, K.fy, K.cx, K.cy, K.min_depth, K.max_depth], np.float32)


def splat_project(mean, cov, K, T):
    """Eq. 7 for one Gaussian: None when it is not drawn, else a dict with z, mu (u, v), cov (Sigma_I uu, uv, vv) and
    conic (its inverse), all float32. mean (3,), cov (6,) = Sigma_W xx, xy, xz, yy, yz, zz; K a Pinhole (fx, fy, cx,
    cy, min_depth, max_depth are used); T the camera-to-world pose."""
    mean = np.ascontiguousarray(mean, np.float32)
    cov = np.ascontiguousarray(cov, np.float32)
    Tm = np.ascontiguousarray(T, np.float64)
    out = np.zeros(9, np.float32)
    k6 = _k6(K)
    if not _load().orc_splat_project(_p(mean), _p(cov), _p(k6), _p(Tm), _p(out)):
        return None
    return {"z": out[0], "mu": out[1:3].copy(), "cov": out[3:6].copy(), "conic": out[6:9].copy()}


def splat_render(means, covs, opacity, colors, K, T):
    """Eqs. 7-9: colour (H, W, 3) and transmittance (H, W), float64, of n Gaussians (means (n, 3), covs (n, 6),
    opacity (n,), colors (n, 3), float32) seen by the pinhole K (a Pinhole) at camera-to-world pose T; also returns the
    number of Gaussians drawn."""
    means = np.ascontiguousarray(means, np.float32).reshape(-1, 3)
    n = means.shape[0]
    covs = np.ascontiguousarray(covs, np.float32).reshape(n, 6)
    opacity = np.ascontiguousarray(opacity, np.float32).reshape(n)
    colors = np.ascontiguousarray(colors, np.float32).reshape(n, 3)
    Tm = np.ascontiguousarray(T, np.float64)
    rgb = np.zeros((K.height, K.width, 3), np.float64)
    tr = np.zeros((K.height, K.width), np.float64)
    k6 = _k6(K)
    drawn = _load().orc_splat_render(n, _p(means), _p(covs), _p(opacity), _p(colors), _p(k6), _p(Tm), K.width,
                                     K.height, _p(rgb), _p(tr))
    return rgb, tr, int(drawn)


def splat_pixels(means, covs, opacity, colors, K, T, uv):
    """splat_render at the listed pixels only: uv (k, 2) int (u, v); returns rgb (k, 3), trans (k,) float64."""
    means = np.ascontiguousarray(means, np.float32).reshape(-1, 3)
    n = means.shape[0]
    covs = np.ascontiguousarray(covs, np.float32).reshape(n, 6)
    opacity = np.ascontiguousarray(opacity, np.float32).reshape(n)
    colors = np.ascontiguousarray(colors, np.float32).reshape(n, 3)
    uv = np.ascontiguousarray(uv, np.int32).reshape(-1, 2)
    Tm = np.ascontiguousarray(T, np.float64)
    rgb = np.zeros((uv.shape[0], 3), np.float64)
    tr = np.zeros(uv.shape[0], np.float64)
    k6 = _k6(K)
    _load().orc_splat_pixels(n, _p(means), _p(covs), _p(opacity), _p(colors), _p(k6), _p(Tm), uv.shape[0], _p(uv),
                             _p(rgb), _p(tr))
    return rgb, tr


def mc_table():
    """The oracle's Marching Cubes case table: triangles per case (256,), edge triples (256, 12, 3) (-1 unused),
    edge end corners (12, 2)."""
    lib = _load()
    nt = np.zeros(256, np.int32)
    ed = np.zeros((256, 36), np.int8)
    ec = np.zeros((12, 2), np.int8)
    lib.orc_mc_table(_p(nt), _p(ed), _p(ec))
    tri = ed.reshape(256, 12, 3).astype(np.int32)
    for c in range(256):
        tri[c, nt[c]:] = -1
    return nt, tri, ec.astype(np.int32)


def segment_cells(A, B, unit: int, mode: str = "bruteforce") -> np.ndarray:
    """Cells (edge ``unit``) met by the closed fixed-point segment A -> B. mode "bruteforce" or "walk"."""
    lib = _load()
    a = np.ascontiguousarray(A, dtype=np.int64)
    b = np.ascontiguousarray(B, dtype=np.int64)
    cap = 1 << 16
    out = np.zeros((cap, 3), np.int64)
    n = lib.orc_segment_cells(_p(a), _p(b), unit, 0 if mode == "bruteforce" else 1, _p(out), cap)
    return out[:min(n, cap)].copy()


def half_round(x: float) -> float:
    return _load().orc_half_round(x)


BLOCK_UNIT = 1 << 16      # fixed-point units per block edge
VOXEL_UNIT = BLOCK_UNIT // 8


# ---- learned level predictor (level_predictor.cpp): float restatement used for bit-exact level parity
MLP_IN, MLP_HIDDEN, MLP_LEVELS = 16, 64, 3
MLP_PARAMS = MLP_IN * MLP_HIDDEN + MLP_HIDDEN + MLP_HIDDEN * MLP_HIDDEN + MLP_HIDDEN + MLP_HIDDEN * MLP_LEVELS + \
    MLP_LEVELS


def bf16_round(x: float) -> float:
    return _load().orc_bf16_round(x)


def exp_cw(x: float) -> float:
    return _load().orc_exp_cw(x)


def erf_as(x: float) -> float:
    return _load().orc_erf_as(x)


def gelu(x: float) -> float:
    return _load().orc_gelu(x)


def mlp_forward(w_bf16: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Logits (n, 3) float32 of the network with BF16 weights (bit patterns) on features x (n, 16)."""
    w = np.ascontiguousarray(w_bf16, dtype=np.uint16)
    xs = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, MLP_IN)
    out = np.zeros((xs.shape[0], MLP_LEVELS), np.float32)
    _load().orc_mlp_forward(_p(w), _p(xs), xs.shape[0], _p(out))
    return out


def block_features(K: Pinhole, R: np.ndarray, t: np.ndarray, rho: np.ndarray, E: float, tau: float, key,
                   w_bf16: np.ndarray | None = None, n_levels: int = 3):
    """Features (16,) float32 of block ``key`` from a range image (h, w) (< 0 invalid), with float pose R (3x3,
    world <- camera) and t; and the predicted level when weights are given. None when the block is not visible."""
    Rf = np.ascontiguousarray(R, dtype=np.float32).reshape(9)
    tf = np.ascontiguousarray(t, dtype=np.float32).reshape(3)
    r = np.ascontiguousarray(rho, dtype=np.float32)
    f = np.zeros(MLP_IN, np.float32)
    lvl = ctypes.c_int(-1)
    w = None if w_bf16 is None else np.ascontiguousarray(w_bf16, dtype=np.uint16)
    ok = _load().orc_block_features(ctypes.byref(K), _p(Rf), _p(tf), _p(r), E, tau, int(key[0]), int(key[1]),
                                    int(key[2]), _p(w), n_levels, _p(f), ctypes.byref(lvl))
    if not ok:
        return None
    return (f, lvl.value) if w is not None else f


def lidar_block_features(moments, T_ws: np.ndarray, E: float, tau: float, key, w_bf16: np.ndarray | None = None,
                         n_levels: int = 3):
    """Features (16,) float32 of a new block of a LiDAR scan from its 10 end-point moments (n, sums of q_x, q_y,
    q_z, of q_x^2, q_y^2, q_z^2, of q_x q_y, q_x q_z, q_y q_z; q = position in the block in units of E / 1024) and the
    scan pose T_ws (4x4, double); and the predicted level when weights are given."""
    mom = np.ascontiguousarray(moments, dtype=np.uint64).reshape(10)
    T = np.ascontiguousarray(T_ws, dtype=np.float64).reshape(16)
    f = np.zeros(MLP_IN, np.float32)
    lvl = ctypes.c_int(-1)
    w = None if w_bf16 is None else np.ascontiguousarray(w_bf16, dtype=np.uint16)
    _load().orc_lidar_block_features(_p(mom), _p(T), E, tau, int(key[0]), int(key[1]), int(key[2]), _p(w),
                                     n_levels, _p(f), ctypes.byref(lvl))
    return (f, lvl.value) if w is not None else f
