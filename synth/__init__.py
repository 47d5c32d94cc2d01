"""Seeded synthetic inputs shared by the CPU oracle and the CUDA library.

This package renders analytic scenes (boxes, spheres, planes) into pinhole depth + RGB frames and spinning-LiDAR scans,
with seeded noise, and holds the workload tables (sensor, scene and map parameters as plain numbers). It contains none
of the fusion method's arithmetic: it only produces inputs. The paper evaluates on ScanNet, Replica, Newer College and
Oxford-Spires (Sec. 4.1.1 "Datasets"); these seeded scenes stand in for them.

The renderer is plain C (``synth.c``), compiled on first use into ``libsynth.so`` next to this file.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libsynth.so")
_SRC = os.path.join(_HERE, "synth.c")
_lib = None

PRIM_ROOM, PRIM_BOX, PRIM_SPHERE, PRIM_GROUND = 0, 1, 2, 3
PRIM_STRIDE = 14


def build(force: bool = False) -> str:
    """Compile libsynth.so (gcc, -O2, pthreads) if missing or older than its source."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp, fp, u8p = (ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float),
                       ctypes.POINTER(ctypes.c_uint8))
        lib.synth_render_depth.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64, fp, u8p, ctypes.c_int]
        lib.synth_render_lidar.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_double, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_uint64, ctypes.c_uint64, fp, ctypes.c_int]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct)) if a is not None else None


def _threads() -> int:
    return max(1, min(64, os.cpu_count() or 1))


# ----------------------------------------------------------------------------------------------------- scenes

def _prim(kind, p6, col_a, col_b=None, period=0.0):
    row = np.zeros(PRIM_STRIDE)
    row[0] = kind
    row[1:7] = p6
    row[7:10] = col_a
    row[10:13] = col_a if col_b is None else col_b
    row[13] = period
    return row


def tiny_scene() -> np.ndarray:
    """Sphere of radius 0.5 m centred at (0, 0, 1.5) inside the room [-1.5, 1.5]^2 x [0, 3] (camera frame = world)."""
    return np.stack([
        _prim(PRIM_ROOM, [-1.5, -1.5, 0.0, 1.5, 1.5, 3.0], [200, 180, 160], [90, 80, 70], 0.1),
        _prim(PRIM_SPHERE, [0.0, 0.0, 1.5, 0.5, 0.0, 0.0], [220, 60, 40], [40, 60, 220], 0.1),
    ])


def rgbd_scene(seed: int, n_boxes: int = 20, n_spheres: int = 10) -> np.ndarray:
    """Room [-4, 4]^2 x [0, 3] (z up) with seeded boxes resting on the floor and floating spheres.

    Box edges ~ U(0.2, 1.0) per axis, centres |x|, |y| <= 1.4. Sphere radii ~ U(0.1, 0.4), centres |x|, |y| <= 1.4,
    z in [r, 1.5]. Primitives that reach within 0.3 m of the camera circle (radius 2 m) are redrawn so that the
    trajectory stays in free space. Every primitive carries a 10 cm checker of two seeded colours.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    prims = [_prim(PRIM_ROOM, [-4.0, -4.0, 0.0, 4.0, 4.0, 3.0], rng.integers(40, 256, 3), rng.integers(40, 256, 3),
                   0.1)]
    made = 0
    while made < n_boxes:
        e = rng.uniform(0.2, 1.0, 3)
        c = rng.uniform(-1.4, 1.4, 2)
        lo = np.array([c[0] - e[0] / 2, c[1] - e[1] / 2, 0.0])
        hi = np.array([c[0] + e[0] / 2, c[1] + e[1] / 2, e[2]])
        corners = np.array([[x, y] for x in (lo[0], hi[0]) for y in (lo[1], hi[1])])
        if np.max(np.hypot(corners[:, 0], corners[:, 1])) > 1.7:
            continue
        prims.append(_prim(PRIM_BOX, [*lo, *hi], rng.integers(40, 256, 3), rng.integers(40, 256, 3), 0.1))
        made += 1
    made = 0
    while made < n_spheres:
        r = rng.uniform(0.1, 0.4)
        c = rng.uniform(-1.4, 1.4, 2)
        z = rng.uniform(r, 1.5)
        if math.hypot(c[0], c[1]) + r > 1.7:
            continue
        prims.append(_prim(PRIM_SPHERE, [c[0], c[1], z, r, 0, 0], rng.integers(40, 256, 3), rng.integers(40, 256, 3),
                           0.1))
        made += 1
    return np.stack(prims)


def lidar_scene(seed: int, x_min: float = -100.0, x_max: float = 600.0) -> np.ndarray:
    """Street along +x: ground plane z = 0, box buildings on both sides, poles at |y| = 6 m.

    Buildings: length U(10, 40) m, gap U(2, 10) m, front U(8, 12) m from the street axis, back at 30 m,
    height U(5, 25) m. Poles: 0.2 x 0.2 x 6 m, spaced U(10, 20) m.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    prims = [_prim(PRIM_GROUND, [0, 0, 0, 0, 0, 0], [120, 120, 120])]
    for side in (+1.0, -1.0):
        x = x_min
        while x < x_max:
            length = rng.uniform(10.0, 40.0)
            front = rng.uniform(8.0, 12.0)
            height = rng.uniform(5.0, 25.0)
            y0, y1 = (front, 30.0) if side > 0 else (-30.0, -front)
            prims.append(_prim(PRIM_BOX, [x, y0, 0.0, x + length, y1, height], rng.integers(40, 256, 3)))
            x += length + rng.uniform(2.0, 10.0)
        x = x_min
        while x < x_max:
            x += rng.uniform(10.0, 20.0)
            y = 6.0 * side
            prims.append(_prim(PRIM_BOX, [x - 0.1, y - 0.1, 0.0, x + 0.1, y + 0.1, 6.0], [200, 200, 40]))
    return np.stack(prims)


# ----------------------------------------------------------------------------------------------------- poses

def look_at(position, target, up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """World <- camera 4x4 pose for an OpenCV camera (x right, y down, z forward) at ``position`` facing ``target``."""
    p = np.asarray(position, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - p
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, dtype=np.float64))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    T = np.eye(4)
    T[:3, 0], T[:3, 1], T[:3, 2], T[:3, 3] = r, d, f, p
    return T


def rgbd_pose(k: int, n_frames: int = 300, radius: float = 2.0, height: float = 1.2) -> np.ndarray:
    """Camera k on the circle of the given radius at the given height, looking at (0, 0, 0.5)."""
    phi = 2.0 * math.pi * k / n_frames
    return look_at((radius * math.cos(phi), radius * math.sin(phi), height), (0.0, 0.0, 0.5))


def lidar_pose(k: int, step: float = 1.0, height: float = 1.8) -> np.ndarray:
    """Sensor k at x = k * step metres, heading +x (sensor frame: x forward, y left, z up)."""
    T = np.eye(4)
    T[0, 3] = k * step
    T[2, 3] = height
    return T


# ----------------------------------------------------------------------------------------------------- workloads

@dataclass
class Workload:
    """A sensor + scene + map configuration (plain numbers; each side builds its own parameter struct from it)."""
    name: str
    sensor: str                      # "camera" or "lidar"
    seed: int
    n_frames: int
    # map
    base_voxel: float                # coarsest-level voxel edge [m]
    n_levels: int
    truncation: float                # tau [m]
    var_threshold: tuple             # theta_l for merge l -> l+1 [m^2]
    split_hysteresis: float = 4.0    # h; 0 disables split
    min_obs: int = 4                 # k_min
    hash_log2: int = 16
    max_blocks: tuple = (1 << 16, 1 << 16, 1 << 16)
    max_touched: int = 1 << 18
    fp16: bool = False
    has_color: bool = True
    # camera
    width: int = 0
    height: int = 0
    fx: float = 0.0
    fy: float = 0.0
    cx: float = 0.0
    cy: float = 0.0
    min_depth: float = 0.1
    max_depth: float = 10.0
    noise_coef: float = 0.0
    dropout: float = 0.0
    # lidar
    n_beams: int = 0
    n_azimuth: int = 0
    elev_deg: tuple = (-22.5, 22.5)
    range_noise: float = 0.0
    r_min: float = 0.5
    r_max: float = 80.0
    extra: dict = field(default_factory=dict)

    @property
    def voxel0(self) -> float:
        return self.base_voxel / (1 << (self.n_levels - 1))

    def scene(self) -> np.ndarray:
        kind = self.extra.get("scene", self.name)
        if kind == "tiny":
            return tiny_scene()
        if kind == "lidar":
            return lidar_scene(self.seed)
        return rgbd_scene(self.seed)

    def pose(self, k: int) -> np.ndarray:
        kind = self.extra.get("scene", self.name)
        if kind == "tiny":
            return np.eye(4)
        if kind == "lidar":
            return lidar_pose(k)
        return rgbd_pose(k % self.extra.get("orbit_frames", 300), self.extra.get("orbit_frames", 300))


def tiny(noise: bool = True) -> Workload:
    """One 160x120 frame (fx = fy = 120) of a 0.5 m sphere 1.5 m ahead in a 3 m room; 2 levels 1/2 cm; tau = 8 cm."""
    return Workload(name="tiny", sensor="camera", seed=0, n_frames=1, base_voxel=0.02, n_levels=2,
                    truncation=0.08, var_threshold=(1e-6,), hash_log2=16, max_blocks=(1 << 15, 1 << 15, 1 << 10),
                    max_touched=1 << 15, width=160, height=120, fx=120.0, fy=120.0, cx=80.0, cy=60.0,
                    min_depth=0.1, max_depth=5.0, noise_coef=1e-3 if noise else 0.0)


def rgbd(seed: int = 1, n_frames: int = 300, fp16: bool = False) -> Workload:
    """300 frames of 640x480 (fx = fy = 525) on a 2 m circle; 3 levels 1/2/4 cm; tau = 3 x 4 cm."""
    return Workload(name="rgbd", sensor="camera", seed=seed, n_frames=n_frames, base_voxel=0.04, n_levels=3,
                    truncation=0.12, var_threshold=(2e-5, 8e-5), hash_log2=20,
                    max_blocks=(1 << 19, 1 << 19, 1 << 19), max_touched=1 << 18, fp16=fp16, width=640, height=480,
                    fx=525.0, fy=525.0, cx=320.0, cy=240.0, min_depth=0.1, max_depth=10.0, noise_coef=1.5e-3,
                    dropout=0.01)


def lidar(seed: int = 2, n_frames: int = 500) -> Workload:
    """500 scans of 128 x 2048 points; 3 levels 5/10/20 cm; tau = 3 x 20 cm; FP16 TSDF storage, no colour."""
    return Workload(name="lidar", sensor="lidar", seed=seed, n_frames=n_frames, base_voxel=0.20, n_levels=3,
                    truncation=0.60, var_threshold=(4e-4, 1.6e-3), hash_log2=22,
                    max_blocks=(1 << 21, 1 << 20, 1 << 20), max_touched=1 << 19, fp16=True, has_color=False,
                    n_beams=128, n_azimuth=2048, range_noise=0.02, r_min=0.5, r_max=80.0)


def batched_sizes(seed: int = 3, n_maps: int = 16):
    """Per-map frame size drawn uniformly from {320x240, 640x480, 848x480, 1280x720}."""
    sizes = [(320, 240), (640, 480), (848, 480), (1280, 720)]
    rng = np.random.Generator(np.random.PCG64(seed))
    return [sizes[i] for i in rng.integers(0, 4, n_maps)]


def batched(n_maps: int = 16, n_frames: int = 100):
    """16 RGB-D-style maps (scene seeds 100..115) with uneven frame sizes; fx = fy = 525 * W / 640; FP16 storage."""
    out = []
    for m, (w, h) in enumerate(batched_sizes(3, n_maps)):
        wl = rgbd(seed=100 + m, n_frames=n_frames, fp16=True)
        wl.name = f"batched{m}"
        wl.extra = {"scene": "rgbd", "orbit_frames": n_frames}
        wl.width, wl.height = w, h
        wl.fx = wl.fy = 525.0 * w / 640.0
        wl.cx, wl.cy = w / 2.0, h / 2.0
        wl.max_blocks = (1 << 18, 1 << 18, 1 << 18)
        out.append(wl)
    return out


# ----------------------------------------------------------------------------------------------------- rendering

def render_depth(wl: Workload, frame: int, scene: np.ndarray | None = None, pose: np.ndarray | None = None,
                 seed: int | None = None):
    """Render frame ``frame`` of a camera workload. Returns (depth float32 HxW, rgb uint8 HxWx3, T_wc float64 4x4)."""
    lib = _load()
    sc = np.ascontiguousarray(wl.scene() if scene is None else scene, dtype=np.float64)
    T = np.ascontiguousarray(wl.pose(frame) if pose is None else pose, dtype=np.float64)
    depth = np.empty((wl.height, wl.width), dtype=np.float32)
    rgb = np.empty((wl.height, wl.width, 3), dtype=np.uint8)
    lib.synth_render_depth(_ptr(sc, ctypes.c_double), sc.shape[0], wl.width, wl.height, wl.fx, wl.fy, wl.cx, wl.cy,
                           _ptr(T, ctypes.c_double), wl.noise_coef, wl.dropout, wl.seed if seed is None else seed,
                           frame, _ptr(depth, ctypes.c_float), _ptr(rgb, ctypes.c_uint8), _threads())
    return depth, rgb, T


def render_lidar(wl: Workload, frame: int, scene: np.ndarray | None = None, pose: np.ndarray | None = None):
    """Render scan ``frame`` of a LiDAR workload. Returns (xyz float32 Nx3 in the sensor frame, NaN = no return,
    T_ws float64 4x4)."""
    lib = _load()
    sc = np.ascontiguousarray(wl.scene() if scene is None else scene, dtype=np.float64)
    T = np.ascontiguousarray(wl.pose(frame) if pose is None else pose, dtype=np.float64)
    xyz = np.empty((wl.n_beams * wl.n_azimuth, 3), dtype=np.float32)
    lib.synth_render_lidar(_ptr(sc, ctypes.c_double), sc.shape[0], wl.n_beams, wl.n_azimuth, wl.elev_deg[0],
                           wl.elev_deg[1], _ptr(T, ctypes.c_double), wl.range_noise, wl.r_min, wl.r_max, wl.seed,
                           frame, _ptr(xyz, ctypes.c_float), _threads())
    return xyz, T


def gaussians(wl: Workload, n: int, frames=(0, 40, 80, 120, 160, 200, 240, 280), seed: int = 7,
              footprint_px=(1.5, 6.0)) -> dict:
    """Seeded 3D Gaussians on the scene's surfaces, depth-seeded like the splats of the rendering branch: n pixels
    drawn at random from noise-free depth renders of camera workload ``wl`` at ``frames`` are back-projected to
    world points (the means), coloured by their pixel (RGB / 255), given a random orientation and per-axis standard
    deviations of U(footprint_px) pixels at their depth times U(0.3, 1) anisotropy, and an opacity of U(0.3, 0.95).
    Returns means (n, 3), covs (n, 6: xx, xy, xz, yy, yz, zz), opacity (n,), colors (n, 3), all float32."""
    import dataclasses
    rng = np.random.default_rng(seed)
    clean = dataclasses.replace(wl, noise_coef=0.0, dropout=0.0)
    sc = wl.scene()
    per = [n // len(frames) + (1 if i < n % len(frames) else 0) for i in range(len(frames))]
    means, cols, dist = [], [], []
    for k, cnt in zip(frames, per):
        depth, rgb, T = render_depth(clean, k, scene=sc)
        vv, uu = np.nonzero(depth > 0)
        pick = rng.choice(vv.size, size=cnt, replace=vv.size < cnt)
        u, v = uu[pick].astype(np.float64), vv[pick].astype(np.float64)
        z = depth[vv[pick], uu[pick]].astype(np.float64)
        pc = np.stack([(u - wl.cx) / wl.fx * z, (v - wl.cy) / wl.fy * z, z], 1)
        means.append(pc @ T[:3, :3].T + T[:3, 3])
        cols.append(rgb[vv[pick], uu[pick]].astype(np.float64) / 255.0)
        dist.append(np.linalg.norm(pc, axis=1))  # distance from the camera that saw the point
    mu = np.concatenate(means)
    col = np.concatenate(cols)
    dist = np.concatenate(dist)
    # standard deviations: a footprint in pixels at that distance
    s = (dist / wl.fx)[:, None] * rng.uniform(*footprint_px, size=(n, 1)) * rng.uniform(0.3, 1.0, size=(n, 3))
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, zq = q.T
    Rm = np.stack([1 - 2 * (y * y + zq * zq), 2 * (x * y - w * zq), 2 * (x * zq + w * y),
                   2 * (x * y + w * zq), 1 - 2 * (x * x + zq * zq), 2 * (y * zq - w * x),
                   2 * (x * zq - w * y), 2 * (y * zq + w * x), 1 - 2 * (x * x + y * y)], 1).reshape(n, 3, 3)
    S = np.einsum("nij,nj,nkj->nik", Rm, s * s, Rm)
    covs = np.stack([S[:, 0, 0], S[:, 0, 1], S[:, 0, 2], S[:, 1, 1], S[:, 1, 2], S[:, 2, 2]], 1)
    return {"means": mu.astype(np.float32), "covs": covs.astype(np.float32),
            "opacity": rng.uniform(0.3, 0.95, n).astype(np.float32), "colors": col.astype(np.float32)}
