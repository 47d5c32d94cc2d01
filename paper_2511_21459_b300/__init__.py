"""B300 (sm_103a) variance-adaptive hashed TSDF map: thin Python binding of libmrhash's C ABI (include/mrhash.h).

Every step of the per-frame path runs in the library's CUDA kernels; this module only marshals arguments. PyTorch is
used for device buffers and streams. There is no CPU fallback: if ``libmrhash.so`` is missing or cannot be loaded,
importing the binding's entry points raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmrhash.so")
_lib = None

MRH_STORAGE_FP32, MRH_STORAGE_FP16 = 0, 1
STATUS = {0: "ok", 1: "invalid argument", 2: "out of device memory", 3: "hash table probe limit reached",
          4: "block heap empty", 5: "per-frame list full", 6: "CUDA error", 7: "output buffer too small",
          8: "more blocks than the no-allocation extract's fixed scratch holds",
          9: "hash table and block heaps disagree on the number of blocks"}


class MrhError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {STATUS.get(code, 'unknown')} ({code})")


class Params(ctypes.Structure):
    """mrh_map_params"""
    _fields_ = [("base_voxel_size", ctypes.c_float), ("n_levels", ctypes.c_int32), ("truncation", ctypes.c_float),
                ("var_threshold", ctypes.c_double * 2), ("split_hysteresis", ctypes.c_double),
                ("min_obs", ctypes.c_int32), ("hash_slots_log2", ctypes.c_uint32),
                ("max_blocks", ctypes.c_uint32 * 3), ("max_touched", ctypes.c_uint32),
                ("max_observations", ctypes.c_uint32), ("storage", ctypes.c_int32), ("has_color", ctypes.c_int32),
                ("min_range", ctypes.c_float), ("max_range", ctypes.c_float)]


class Pinhole(ctypes.Structure):
    """mrh_pinhole"""
    _fields_ = [("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("min_depth", ctypes.c_float),
                ("max_depth", ctypes.c_float)]


class Stats(ctypes.Structure):
    """mrh_stats"""
    _fields_ = [("frame", ctypes.c_uint64), ("valid_rays", ctypes.c_uint64), ("touched", ctypes.c_uint64),
                ("new_blocks", ctypes.c_uint64), ("merged", ctypes.c_uint64), ("split", ctypes.c_uint64),
                ("fp64_rechecks", ctypes.c_uint64), ("live_blocks", ctypes.c_uint64 * 3),
                ("touched_level", ctypes.c_uint64 * 3), ("observations", ctypes.c_uint64),
                ("updated_voxels", ctypes.c_uint64), ("lidar_restaged", ctypes.c_uint64), ("evicted", ctypes.c_uint64),
                ("restored", ctypes.c_uint64), ("archived", ctypes.c_uint64),
                ("lidar_max_voxel_obs", ctypes.c_uint64), ("status", ctypes.c_uint32)]

    def as_dict(self):
        d = {n: getattr(self, n) for n, _ in self._fields_ if n not in ("live_blocks", "touched_level")}
        d["live_blocks"] = list(self.live_blocks)
        d["touched_level"] = list(self.touched_level)
        return d


KERNEL_GROUPS = ["begin", "alloc", "bin", "lidar_obs", "fuse", "release", "raycast", "mesh", "stream"]

MRH_BATCH_GRAPH, MRH_BATCH_AUTOTUNE = 1, 2


class BatchFrame(ctypes.Structure):
    """mrh_batch_frame"""
    _fields_ = [("K", Pinhole), ("T_wc", ctypes.c_double * 16), ("depth_dev", ctypes.c_void_p),
                ("rgb_dev", ctypes.c_void_p), ("raycast_dev", ctypes.c_void_p)]


EXPORTS = ["mrh_map_create", "mrh_map_destroy", "mrh_integrate_depth", "mrh_integrate_points", "mrh_raycast",
           "mrh_count_blocks", "mrh_extract_blocks", "mrh_extract_blocks_noalloc", "mrh_get_stats", "mrh_sync",
           "mrh_clear_status", "mrh_set_profiling", "mrh_get_profile", "mrh_batch_create", "mrh_batch_integrate",
           "mrh_batch_config", "mrh_batch_last_step_ms", "mrh_batch_destroy", "mrh_set_predictor",
           "mrh_set_feature_capture",
           "mrh_get_features", "mrh_mlp_create", "mrh_mlp_destroy", "mrh_mlp_train_step", "mrh_mlp_loss_grad",
           "mrh_mlp_predict", "mrh_mlp_get_weights", "mrh_hash_slot", "mrh_status_string", "mrh_last_cuda_error",
           "mrh_version", "mrh_extract_mesh", "mrh_mesh_case_table", "mrh_weld_mesh", "mrh_quadtree",
           "mrh_set_streaming", "mrh_save_map", "mrh_load_map", "mrh_splat_render"]

MLP_IN, MLP_HIDDEN, MLP_LEVELS = 16, 64, 3
MLP_PARAMS = MLP_IN * MLP_HIDDEN + MLP_HIDDEN + MLP_HIDDEN * MLP_HIDDEN + MLP_HIDDEN + MLP_HIDDEN * MLP_LEVELS + \
    MLP_LEVELS


def lib():
    """Load libmrhash.so (fails loudly when it is missing: there is no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libmrhash.so not built ({LIB_PATH}); run `python -m paper_2511_21459_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        vp, u64, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
        L.mrh_map_create.argtypes = [ctypes.POINTER(Params), i32, ctypes.POINTER(vp)]
        L.mrh_map_destroy.argtypes = [vp]
        L.mrh_integrate_depth.argtypes = [vp, ctypes.POINTER(Pinhole), vp, vp, vp, vp]
        L.mrh_integrate_points.argtypes = [vp, vp, vp, u64, vp]
        L.mrh_raycast.argtypes = [vp, ctypes.POINTER(Pinhole), vp, vp, vp, vp, vp]
        L.mrh_count_blocks.argtypes = [vp, ctypes.POINTER(u64), ctypes.POINTER(u64), vp]
        L.mrh_extract_mesh.argtypes = [vp, vp, u64, ctypes.POINTER(u64), vp]
        L.mrh_mesh_case_table.argtypes = [vp, vp, vp]
        L.mrh_mesh_case_table.restype = None
        L.mrh_set_streaming.argtypes = [vp, ctypes.c_float, ctypes.c_float, ctypes.c_uint32]
        L.mrh_save_map.argtypes = [vp, ctypes.c_char_p, vp]
        L.mrh_splat_render.argtypes = [vp, vp, vp, vp, ctypes.c_uint64, ctypes.POINTER(Pinhole), vp, vp, vp,
                                       ctypes.POINTER(ctypes.c_uint64), ctypes.c_int, vp]
        L.mrh_load_map.argtypes = [ctypes.c_char_p, ctypes.c_int, ctypes.POINTER(vp)]
        L.mrh_quadtree.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, vp, u64,
                                   ctypes.POINTER(u64), ctypes.c_int, vp]
        L.mrh_weld_mesh.argtypes = [vp, vp, u64, ctypes.c_float, vp, u64, vp, u64, ctypes.POINTER(u64),
                                    ctypes.POINTER(u64), vp]
        L.mrh_extract_blocks.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, u64, u64, ctypes.POINTER(u64),
                                         ctypes.POINTER(u64), vp]
        L.mrh_extract_blocks_noalloc.argtypes = L.mrh_extract_blocks.argtypes
        L.mrh_get_stats.argtypes = [vp, ctypes.POINTER(Stats), vp]
        L.mrh_sync.argtypes = [vp, vp]
        L.mrh_clear_status.argtypes = [vp, vp]
        L.mrh_set_profiling.argtypes = [vp, i32]
        L.mrh_get_profile.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(u64), i32, i32, vp]
        L.mrh_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Pinhole), i32, i32, ctypes.POINTER(vp)]
        L.mrh_batch_integrate.argtypes = [vp, ctypes.POINTER(BatchFrame), vp]
        L.mrh_batch_config.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
        L.mrh_batch_last_step_ms.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
        L.mrh_batch_destroy.argtypes = [vp]
        L.mrh_set_predictor.argtypes = [vp, vp, u64]
        L.mrh_set_feature_capture.argtypes = [vp, ctypes.c_uint32]
        L.mrh_get_features.argtypes = [vp, vp, vp, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32),
                                       ctypes.POINTER(u64), i32, vp]
        L.mrh_mlp_create.argtypes = [vp, i32, ctypes.POINTER(vp)]
        L.mrh_mlp_destroy.argtypes = [vp]
        L.mrh_mlp_train_step.argtypes = [vp, vp, vp, ctypes.c_uint32, ctypes.c_float, vp, vp]
        L.mrh_mlp_loss_grad.argtypes = [vp, vp, vp, ctypes.c_uint32, vp, vp, vp]
        L.mrh_mlp_predict.argtypes = [vp, vp, ctypes.c_uint32, vp, vp]
        L.mrh_mlp_get_weights.argtypes = [vp, vp, vp, vp]
        L.mrh_hash_slot.restype = ctypes.c_uint32
        L.mrh_hash_slot.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint32]
        L.mrh_status_string.restype = ctypes.c_char_p
        L.mrh_last_cuda_error.restype = ctypes.c_char_p
        L.mrh_version.restype = ctypes.c_char_p
        for name in ("mrh_map_create", "mrh_map_destroy", "mrh_integrate_depth", "mrh_integrate_points",
                     "mrh_raycast", "mrh_count_blocks", "mrh_extract_blocks", "mrh_extract_blocks_noalloc",
                     "mrh_get_stats", "mrh_sync",
                     "mrh_clear_status", "mrh_set_profiling", "mrh_get_profile", "mrh_batch_create",
                     "mrh_batch_integrate", "mrh_batch_config", "mrh_batch_last_step_ms", "mrh_batch_destroy",
                     "mrh_set_predictor",
                     "mrh_set_feature_capture", "mrh_get_features", "mrh_mlp_create", "mrh_mlp_destroy",
                     "mrh_mlp_train_step", "mrh_mlp_loss_grad", "mrh_mlp_predict", "mrh_mlp_get_weights"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


DEVICE_CAPACITY_CODES = (3, 4, 5)  # sticky device statuses: the map stays valid, reported by stats() / sync()


def _check(code: int, what: str, allow=()):
    if code != 0 and code not in allow:
        err = lib().mrh_last_cuda_error().decode()
        raise MrhError(code, what + (f" [{err}]" if code == 6 and err else ""))


def quadtree(rgb, threshold: float = 0.1, min_size: int = 1, stream=None):
    """Contrast quadtree (Sec. 3.5) of an (H, W, 3) uint8 CUDA tensor: leaves (n, 4) int32 CUDA tensor (x, y, w, h),
    in no particular order (see mrh_quadtree)."""
    import torch
    img = rgb.contiguous()
    h, w = int(img.shape[0]), int(img.shape[1])
    dev = img.device.index if img.device.index is not None else torch.cuda.current_device()
    n = ctypes.c_uint64()
    cap = w * h
    out = torch.empty((cap, 4), dtype=torch.int32, device=img.device)
    _check(lib().mrh_quadtree(_ptr(img), w, h, float(threshold), int(min_size), _ptr(out), cap, ctypes.byref(n), dev,
                              _stream(stream)), "mrh_quadtree")
    return out[:n.value]


def splat_render(means, covs, opacity, colors, K: Pinhole, T_wc, out=None, trans=None, stream=None):
    """Gaussian-splat rendering (see mrh_splat_render): means (n, 3), covs (n, 6), opacity (n,), colors (n, 3)
    float32 CUDA tensors on one device; returns (rgb (h, w, 3), transmittance (h, w), pairs). ``out`` / ``trans``:
    optional CUDA tensors to write into; trans=False skips the transmittance."""
    import torch
    dev = means.device
    n = int(means.shape[0])
    for t, shape in ((means, (n, 3)), (covs, (n, 6)), (opacity, (n,)), (colors, (n, 3))):
        if t.device != dev or t.dtype != torch.float32 or tuple(t.shape) != shape or not t.is_contiguous():
            raise ValueError(f"expected a contiguous float32 {shape} tensor on {dev}")
    if out is None:
        out = torch.empty((K.height, K.width, 3), dtype=torch.float32, device=dev)
    if trans is None:
        trans = torch.empty((K.height, K.width), dtype=torch.float32, device=dev)
    tr = trans if trans is not False else None
    T = _pose(T_wc)
    pairs = ctypes.c_uint64()
    _check(lib().mrh_splat_render(_ptr(means), _ptr(covs), _ptr(opacity), _ptr(colors), n, ctypes.byref(K),
                                  ctypes.c_void_p(T.ctypes.data), _ptr(out), _ptr(tr), ctypes.byref(pairs),
                                  dev.index if dev.index is not None else torch.cuda.current_device(),
                                  _stream(stream)), "mrh_splat_render")
    return out, tr, pairs.value


def mesh_case_table():
    """The library's Marching Cubes case table (host, no GPU needed): triangles per case (256,), edge triples
    (256, 5, 3) (-1 unused), edge end corners (12, 2)."""
    import numpy as np
    nt = np.zeros(256, np.uint8)
    tri = np.zeros((256, 15), np.int8)
    ec = np.zeros((12, 2), np.int8)
    lib().mrh_mesh_case_table(ctypes.c_void_p(nt.ctypes.data), ctypes.c_void_p(tri.ctypes.data),
                              ctypes.c_void_p(ec.ctypes.data))
    return nt.astype(np.int32), tri.reshape(256, 5, 3).astype(np.int32), ec.astype(np.int32)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _pose(T) -> np.ndarray:
    T = np.ascontiguousarray(np.asarray(T, dtype=np.float64).reshape(4, 4))
    return T


def hash_slot(x: int, y: int, z: int, log2_slots: int) -> int:
    """Eq. 4 slot of block key (x, y, z) (host helper, no GPU needed)."""
    return int(lib().mrh_hash_slot(x, y, z, log2_slots))


def params_from(wl, storage: int | None = None, max_observations: int | None = None) -> Params:
    """Map parameters for a workload description (``synth.Workload``)."""
    p = Params()
    p.base_voxel_size = wl.base_voxel
    p.n_levels = wl.n_levels
    p.truncation = wl.truncation
    th = list(wl.var_threshold) + [0.0, 0.0]
    p.var_threshold[0], p.var_threshold[1] = th[0], th[1]
    p.split_hysteresis = wl.split_hysteresis
    p.min_obs = wl.min_obs
    p.hash_slots_log2 = wl.hash_log2
    mb = list(wl.max_blocks) + [1, 1, 1]
    for l in range(3):
        p.max_blocks[l] = mb[l]
    p.max_touched = wl.max_touched
    if max_observations is None:
        max_observations = (1 << 25) if wl.sensor == "lidar" else 0
    p.max_observations = max_observations
    p.storage = (MRH_STORAGE_FP16 if wl.fp16 else MRH_STORAGE_FP32) if storage is None else storage
    p.has_color = int(wl.has_color)
    p.min_range, p.max_range = wl.r_min, wl.r_max
    return p


def pinhole_from(wl) -> Pinhole:
    k = Pinhole()
    k.fx, k.fy, k.cx, k.cy = wl.fx, wl.fy, wl.cx, wl.cy
    k.width, k.height = wl.width, wl.height
    k.min_depth, k.max_depth = wl.min_depth, wl.max_depth
    return k


class Map:
    """A map on one CUDA device. Inputs are CUDA tensors on that device; poses are 4x4 (or 16) float64 host arrays."""

    def __init__(self, params: Params, device: int = 0):
        self._lib = lib()
        self.params = params
        self.device = device
        h = ctypes.c_void_p()
        _check(self._lib.mrh_map_create(ctypes.byref(params), device, ctypes.byref(h)), "mrh_map_create")
        self._h = h

    @classmethod
    def load(cls, path: str, device: int = 0) -> "Map":
        """A map on ``device`` from a file written by ``Map.save`` (see mrh_load_map)."""
        self = cls.__new__(cls)
        self._lib = lib()
        self.device = device
        h = ctypes.c_void_p()
        _check(self._lib.mrh_load_map(os.fsencode(path), device, ctypes.byref(h)), "mrh_load_map")
        self._h = h
        with open(path, "rb") as f:  # the creation parameters follow the magic, version and size words
            f.seek(16)
            self.params = Params.from_buffer_copy(f.read(ctypes.sizeof(Params)))
        return self

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mrh_map_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def integrate_depth(self, K: Pinhole, T_wc, depth, rgb=None, stream=None):
        T = _pose(T_wc)
        _check(self._lib.mrh_integrate_depth(self._h, ctypes.byref(K), ctypes.c_void_p(T.ctypes.data), _ptr(depth),
                                             _ptr(rgb), _stream(stream)), "mrh_integrate_depth")

    def integrate_points(self, T_ws, xyz, stream=None):
        T = _pose(T_ws)
        _check(self._lib.mrh_integrate_points(self._h, ctypes.c_void_p(T.ctypes.data), _ptr(xyz), xyz.shape[0],
                                              _stream(stream)), "mrh_integrate_points")

    def raycast(self, K: Pinhole, T_wc, out=None, stream=None, normals=None, rgb=None):
        """z-depth (h, w) float32 CUDA tensor (written into ``out`` when given). ``normals`` / ``rgb``: True (allocate)
        or a CUDA tensor (h, w, 3) float32 / uint8 to receive the unit normal / colour at the hit as well; then the
        result is a tuple (depth, [normals], [rgb])."""
        import torch
        T = _pose(T_wc)
        dev = f"cuda:{self.device}"
        if out is None:
            out = torch.empty((K.height, K.width), dtype=torch.float32, device=dev)
        if normals is True:
            normals = torch.empty((K.height, K.width, 3), dtype=torch.float32, device=dev)
        if rgb is True:
            rgb = torch.empty((K.height, K.width, 3), dtype=torch.uint8, device=dev)
        nrm = normals if normals is not None and normals is not False else None
        col = rgb if rgb is not None and rgb is not False else None
        _check(self._lib.mrh_raycast(self._h, ctypes.byref(K), ctypes.c_void_p(T.ctypes.data), _ptr(out), _ptr(nrm),
                                     _ptr(col), _stream(stream)), "mrh_raycast")
        if nrm is None and col is None:
            return out
        return (out,) + ((nrm,) if nrm is not None else ()) + ((col,) if col is not None else ())

    def extract_mesh(self, capacity=None, stream=None):
        """Multi-resolution Marching Cubes triangles (n, 3, 3) float32 CUDA tensor (vertices in metres, counter-clockwise
        seen from positive distance, in no particular order). With capacity None the call counts first, then
        allocates exactly; otherwise MrhError (capacity) when the mesh has more triangles."""
        import torch
        n = ctypes.c_uint64()
        if capacity is None:
            _check(self._lib.mrh_extract_mesh(self._h, None, 0, ctypes.byref(n), _stream(stream)), "mrh_extract_mesh",
                   allow=(7,))
            capacity = n.value
        out = torch.empty((max(int(capacity), 1), 3, 3), dtype=torch.float32, device=f"cuda:{self.device}")
        _check(self._lib.mrh_extract_mesh(self._h, ctypes.c_void_p(out.data_ptr()), int(capacity), ctypes.byref(n),
                                          _stream(stream)), "mrh_extract_mesh")
        return out[:n.value]

    def set_streaming(self, fraction: float, radius: float = 0.0, archive_blocks: int = 1 << 16):
        """Capacity-driven streaming (see mrh_set_streaming): fraction of a level's pool that triggers eviction, the
        LiDAR radius [m], and the archive's capacity in blocks."""
        _check(self._lib.mrh_set_streaming(self._h, float(fraction), float(radius), int(archive_blocks)),
               "mrh_set_streaming")

    def save(self, path: str, stream=None):
        """Write the map (resident and archived blocks) to a file (see mrh_save_map)."""
        _check(self._lib.mrh_save_map(self._h, os.fsencode(path), _stream(stream)), "mrh_save_map")

    def weld_mesh(self, tris, delta: float, stream=None):
        """Vertex collapse of a triangle soup (n, 3, 3) float32 CUDA tensor on a grid of spacing delta [m]:
        vertices (nv, 3) float32 and faces (nf, 3) int32 CUDA tensors (see mrh_weld_mesh)."""
        import torch
        t = tris.contiguous()
        nv, nf = ctypes.c_uint64(), ctypes.c_uint64()
        _check(self._lib.mrh_weld_mesh(self._h, _ptr(t), t.shape[0], float(delta), None, 0, None, 0,
                                       ctypes.byref(nv), ctypes.byref(nf), _stream(stream)), "mrh_weld_mesh",
               allow=(7,))
        dev = f"cuda:{self.device}"
        verts = torch.empty((max(nv.value, 1), 3), dtype=torch.float32, device=dev)
        faces = torch.empty((max(nf.value, 1), 3), dtype=torch.int32, device=dev)
        _check(self._lib.mrh_weld_mesh(self._h, _ptr(t), t.shape[0], float(delta), _ptr(verts), nv.value,
                                       _ptr(faces), nf.value, ctypes.byref(nv), ctypes.byref(nf), _stream(stream)),
               "mrh_weld_mesh")
        return verts[:nv.value], faces[:nf.value]

    def count(self, stream=None):
        nb, nv = ctypes.c_uint64(), ctypes.c_uint64()
        _check(self._lib.mrh_count_blocks(self._h, ctypes.byref(nb), ctypes.byref(nv), _stream(stream)),
               "mrh_count_blocks", allow=DEVICE_CAPACITY_CODES)
        return nb.value, nv.value

    def extract(self, stream=None) -> dict:
        """All blocks sorted by key: keys (n,3) int32, levels (n,) uint8, offsets (n+1,) int64, D/W/S2 (V,) float32,
        C (V,3) float32 (CUDA tensors)."""
        import torch
        nb, nv = self.count(stream)
        dev = f"cuda:{self.device}"
        out = dict(keys=torch.empty((max(nb, 1), 3), dtype=torch.int32, device=dev),
                   levels=torch.empty(max(nb, 1), dtype=torch.uint8, device=dev),
                   offsets=torch.zeros(nb + 1, dtype=torch.int64, device=dev),
                   D=torch.empty(max(nv, 1), dtype=torch.float32, device=dev),
                   W=torch.empty(max(nv, 1), dtype=torch.float32, device=dev),
                   S2=torch.empty(max(nv, 1), dtype=torch.float32, device=dev),
                   C=torch.empty((max(nv, 1), 3), dtype=torch.float32, device=dev))
        wb, wv = ctypes.c_uint64(), ctypes.c_uint64()
        code = self._lib.mrh_extract_blocks(self._h, _ptr(out["keys"]), _ptr(out["levels"]), _ptr(out["offsets"]),
                                            _ptr(out["D"]), _ptr(out["W"]), _ptr(out["S2"]), _ptr(out["C"]),
                                            max(nb, 1), max(nv, 1), ctypes.byref(wb), ctypes.byref(wv),
                                            _stream(stream))
        _check(code, "mrh_extract_blocks", allow=DEVICE_CAPACITY_CODES)
        n, v = wb.value, wv.value
        return dict(keys=out["keys"][:n], levels=out["levels"][:n], offsets=out["offsets"], D=out["D"][:v],
                    W=out["W"][:v], S2=out["S2"][:v], C=out["C"][:v])

    def stats(self, stream=None) -> dict:
        s = Stats()
        code = self._lib.mrh_get_stats(self._h, ctypes.byref(s), _stream(stream))
        d = s.as_dict()
        d["status_code"] = code
        return d

    def sync(self, stream=None):
        _check(self._lib.mrh_sync(self._h, _stream(stream)), "mrh_sync")

    def set_profiling(self, enable: bool):
        _check(self._lib.mrh_set_profiling(self._h, int(enable)), "mrh_set_profiling")

    def profile(self, reset: bool = False, stream=None) -> dict:
        """{group: (device ms, launches)} accumulated since the last reset."""
        n = len(KERNEL_GROUPS)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_uint64 * n)()
        _check(self._lib.mrh_get_profile(self._h, ms, cnt, n, int(reset), _stream(stream)), "mrh_get_profile")
        return {g: (ms[i], cnt[i]) for i, g in enumerate(KERNEL_GROUPS)}

    def clear_status(self, stream=None):
        _check(self._lib.mrh_clear_status(self._h, _stream(stream)), "mrh_clear_status")

    def set_predictor(self, w_bf16):
        """Learned level predictor for later depth frames: MLP_PARAMS BF16 bit patterns (numpy uint16), or None."""
        if w_bf16 is None:
            _check(self._lib.mrh_set_predictor(self._h, None, 0), "mrh_set_predictor")
            return
        w = np.ascontiguousarray(w_bf16, dtype=np.uint16)
        _check(self._lib.mrh_set_predictor(self._h, ctypes.c_void_p(w.ctypes.data), w.size), "mrh_set_predictor")

    def set_feature_capture(self, capacity: int):
        """Record (key, features) of up to ``capacity`` new blocks of later depth frames; 0 turns it off."""
        _check(self._lib.mrh_set_feature_capture(self._h, int(capacity)), "mrh_set_feature_capture")

    def features(self, reset: bool = False, stream=None):
        """Recorded new-block features: (keys (n,3) int32, features (n,16) float32) CUDA tensors in record order,
        and the number of records offered (more than n when the capacity was exceeded)."""
        import torch
        n, seen = ctypes.c_uint32(), ctypes.c_uint64()
        _check(self._lib.mrh_get_features(self._h, None, None, 0, ctypes.byref(n), ctypes.byref(seen), 0,
                                          _stream(stream)), "mrh_get_features", allow=(7,))
        dev = f"cuda:{self.device}"
        keys = torch.empty((max(n.value, 1), 3), dtype=torch.int32, device=dev)
        feats = torch.empty((max(n.value, 1), MLP_IN), dtype=torch.float32, device=dev)
        _check(self._lib.mrh_get_features(self._h, _ptr(keys), _ptr(feats), max(n.value, 1), ctypes.byref(n),
                                          ctypes.byref(seen), int(reset), _stream(stream)), "mrh_get_features")
        return keys[:n.value], feats[:n.value], seen.value


class Mlp:
    """GPU trainer of the level predictor (mrh_mlp_*): FP32 master weights, BF16 forward / backward, Adam."""

    def __init__(self, init_weights, device: int = 0):
        self._lib = lib()
        self.device = device
        w = np.ascontiguousarray(init_weights, dtype=np.float32)
        if w.size != MLP_PARAMS:
            raise ValueError(f"need {MLP_PARAMS} weights")
        h = ctypes.c_void_p()
        _check(self._lib.mrh_mlp_create(ctypes.c_void_p(w.ctypes.data), device, ctypes.byref(h)), "mrh_mlp_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mrh_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def train_step(self, x, labels, lr: float, loss_out, stream=None):
        """One Adam step on (x (n,16) float32, labels (n,) int32) CUDA tensors; loss_out: 1-element CUDA tensor."""
        _check(self._lib.mrh_mlp_train_step(self._h, _ptr(x), _ptr(labels), x.shape[0], float(lr), _ptr(loss_out),
                                            _stream(stream)), "mrh_mlp_train_step")

    def loss_grad(self, x, labels, stream=None):
        """(loss (1,), grad (MLP_PARAMS,)) CUDA tensors for the current BF16 weights."""
        import torch
        dev = f"cuda:{self.device}"
        loss = torch.empty(1, dtype=torch.float32, device=dev)
        grad = torch.empty(MLP_PARAMS, dtype=torch.float32, device=dev)
        _check(self._lib.mrh_mlp_loss_grad(self._h, _ptr(x), _ptr(labels), x.shape[0], _ptr(loss), _ptr(grad),
                                           _stream(stream)), "mrh_mlp_loss_grad")
        return loss, grad

    def predict(self, x, stream=None):
        import torch
        out = torch.empty((x.shape[0], MLP_LEVELS), dtype=torch.float32, device=f"cuda:{self.device}")
        _check(self._lib.mrh_mlp_predict(self._h, _ptr(x), x.shape[0], _ptr(out), _stream(stream)),
               "mrh_mlp_predict")
        return out

    def weights(self, stream=None):
        """(FP32 master weights, BF16 bit patterns) as numpy arrays."""
        master = np.zeros(MLP_PARAMS, np.float32)
        bf = np.zeros(MLP_PARAMS, np.uint16)
        _check(self._lib.mrh_mlp_get_weights(self._h, ctypes.c_void_p(master.ctypes.data),
                                             ctypes.c_void_p(bf.ctypes.data), _stream(stream)),
               "mrh_mlp_get_weights")
        return master, bf


class Batch:
    """Several maps integrated together, one launch per phase (mrh_batch_*). ``maps`` must outlive the batch."""

    def __init__(self, maps, cams, flags: int = MRH_BATCH_GRAPH | MRH_BATCH_AUTOTUNE):
        self._lib = lib()
        self.maps = list(maps)
        self.cams = list(cams)
        n = len(self.maps)
        hs = (ctypes.c_void_p * n)(*[m._h.value for m in self.maps])
        ks = (Pinhole * n)(*self.cams)
        h = ctypes.c_void_p()
        _check(self._lib.mrh_batch_create(hs, ks, n, flags, ctypes.byref(h)), "mrh_batch_create")
        self._h = h

    def integrate(self, frames, stream=None):
        """frames: per map (T_wc 4x4, depth CUDA tensor, rgb CUDA tensor or None, raycast out CUDA tensor or None)."""
        n = len(self.maps)
        arr = (BatchFrame * n)()
        for i, (T, depth, rgb, out) in enumerate(frames):
            arr[i].K = self.cams[i]
            Tf = _pose(T).ravel()
            for k in range(16):
                arr[i].T_wc[k] = float(Tf[k])
            arr[i].depth_dev = depth.data_ptr()
            arr[i].rgb_dev = rgb.data_ptr() if rgb is not None else None
            arr[i].raycast_dev = out.data_ptr() if out is not None else None
        _check(self._lib.mrh_batch_integrate(self._h, arr, _stream(stream)), "mrh_batch_integrate")

    def config(self) -> dict:
        c = (ctypes.c_int * 8)()
        _check(self._lib.mrh_batch_config(self._h, c), "mrh_batch_config")
        return dict(alloc_tile=(c[0], c[1]), probe_width=c[2], fuse_warps=c[3], fuse_ctas_per_sm=c[4],
                    raycast_warp_tile="16x2" if c[5] else "8x4", tuned=bool(c[6]), graph=bool(c[7]))

    def last_step_ms(self) -> dict:
        """Device time of the last step's phases (waits for it): allocation, binning, fusion, release + raycast."""
        c = (ctypes.c_float * 4)()
        _check(self._lib.mrh_batch_last_step_ms(self._h, c), "mrh_batch_last_step_ms")
        return dict(alloc=c[0], bin=c[1], fuse=c[2], raycast=c[3])

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mrh_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
