#!/usr/bin/env python
"""Benchmark of the per-frame hot path: integrated points/s and frames/s on the RGB-D sequence (640x480, 3 levels
1/2/4 cm, tau 12 cm, 2^20-slot hash, colour, FP32 storage; a 640x480 raycast of depth, normal and colour every
frame), with a LiDAR line
(128 x 2048 = 262,144 points per scan, FP16 storage) and the HBM roofline of the fusion kernel.

A step is one frame: allocation, fusion + block variance + re-levelling, heap release, and the raycast (depth, normal
and colour) of that frame's view. Inputs are seeded synthetic frames (the paper's RGB-D and LiDAR datasets are not available), generated before
timing and resident in HBM. Every step is timed with CUDA events on the launching stream; L2 is flushed (a 256 MiB
write) between steps, outside the timed events.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With --gpus N > 1 (launched by torch.distributed.run) each rank integrates its own replica of the sequence on its own
GPU (no data exchange): weak scaling, value = all ranks' points / slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "integrated points/s & frames/s (RGB-D 640x480, LiDAR 262k pts) vs HBM roofline"
RGBD_WORKLOAD = ("rgbd-640x480-seq300 (3 levels 1/2/4 cm, tau 12 cm, 2^20 hash, colour, FP32 storage) + 640x480 "
                 "raycast (depth, normal, colour) per frame")
FALLBACK_HBM_GBS = 6400.0
L2_FLUSH_BYTES = 256 << 20


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=290)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--lidar-steps", type=int, default=40)
    ap.add_argument("--batched-steps", type=int, default=20)
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-lidar", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--learned-epochs", type=int, default=12)
    ap.add_argument("--no-feature-study", action="store_true",
                    help="skip the comparison of range-image and TSDF-statistics features for the learned level")
    ap.add_argument("--learned-repeats", type=int, default=5, help="interleaved timed runs of plain and learned")
    ap.add_argument("--learned-lidar-train-scans", type=int, default=500)
    ap.add_argument("--learned-lidar-scans", type=int, default=500)
    ap.add_argument("--no-mesh", action="store_true")
    ap.add_argument("--no-quadtree", action="store_true")
    ap.add_argument("--no-streaming", action="store_true")
    ap.add_argument("--no-splat", action="store_true")
    ap.add_argument("--ablation", action="store_true",
                    help="only the variance-threshold sweep (Sec. 5.1 analogue): one JSON line, then exit")
    ap.add_argument("--cpu-budget-s", type=float, default=20.0)
    ap.add_argument("--cpu-replicas", type=int, default=32, help="oracle replicas on the host cores (1 = none)")
    ap.add_argument("--profile-case", choices=["rgbd", "rgbd-grown", "lidar", "batched", "learned", "mesh", "quadtree",
                                               "stream", "splat"],
                    default=None, help="small case for profiler captures (reduced heap capacity)")
    return ap.parse_args()


def profile_case(kind: str) -> int:
    """A few frames of the benchmark sequence on a map with reduced heap capacity (a few hundred MB on the device),
    so that profiler captures of single launches stay small."""
    import torch
    import paper_2511_21459_b300 as mrh
    from paper_2511_21459_b300 import build
    build.build()
    if kind == "rgbd":
        wl = synth.rgbd()
        wl.max_blocks = (1 << 15, 1 << 14, 1 << 14)
        m = mrh.Map(mrh.params_from(wl))
        K = mrh.pinhole_from(wl)
        out = torch.empty((wl.height, wl.width), device="cuda")
        nrm = torch.empty((wl.height, wl.width, 3), device="cuda")
        col = torch.empty((wl.height, wl.width, 3), dtype=torch.uint8, device="cuda")
        for k, (d, c, T) in enumerate(camera_frames(wl, 0, 6)):
            m.integrate_depth(K, T, torch.from_numpy(d).cuda(), torch.from_numpy(c).cuda())
            m.raycast(K, T, out, normals=nrm, rgb=col)
            st = m.stats()
            print(json.dumps({"frame": k, "touched_level": st["touched_level"], "new_blocks": st["new_blocks"],
                              "fuse_algorithmic_bytes": fuse_bytes_camera(st, wl, voxel_bytes(wl))}))
    elif kind == "rgbd-grown":
        # the whole 300-frame orbit integrated (heaps reduced to about 2 GB), then three raycasts with normals and
        # colour from poses spread over the orbit: the map the timed frames of the benchmark see late in the sequence
        wl = synth.rgbd()
        wl.max_blocks = (1 << 17, 1 << 15, 1 << 15)
        m = mrh.Map(mrh.params_from(wl))
        K = mrh.pinhole_from(wl)
        for k, (d, c, T) in enumerate(camera_frames(wl, 0, wl.n_frames)):
            m.integrate_depth(K, T, torch.from_numpy(d).cuda(), torch.from_numpy(c).cuda())
            if k >= wl.n_frames - 3:
                st = m.stats()
                print(json.dumps({"frame": k, "touched_level": st["touched_level"],
                                  "fuse_algorithmic_bytes": fuse_bytes_camera(st, wl, voxel_bytes(wl))}))
        out = torch.empty((wl.height, wl.width), device="cuda")
        nrm = torch.empty((wl.height, wl.width, 3), device="cuda")
        col = torch.empty((wl.height, wl.width, 3), dtype=torch.uint8, device="cuda")
        for k in (40, 150, 299):
            m.raycast(K, wl.pose(k), out, normals=nrm, rgb=col)
        st = m.stats()
        print(json.dumps({"live_blocks": st["live_blocks"], "touched_level_last": st["touched_level"],
                          "fuse_algorithmic_bytes_last": fuse_bytes_camera(st, wl, voxel_bytes(wl))}))
    elif kind == "mesh":
        wl = synth.rgbd()
        wl.max_blocks = (1 << 16, 1 << 14, 1 << 14)
        m = mrh.Map(mrh.params_from(wl))
        K = mrh.pinhole_from(wl)
        for d, c, T in camera_frames(wl, 0, 30)[::5]:
            m.integrate_depth(K, T, torch.from_numpy(d).cuda(), torch.from_numpy(c).cuda())
        for _ in range(3):
            t = m.extract_mesh()
        st = m.stats()
        print(json.dumps({"triangles": int(t.shape[0]), "live_blocks": st["live_blocks"],
                          "mesh_algorithmic_bytes": mesh_bytes(st, wl, int(t.shape[0]))}))
    elif kind == "quadtree":
        wl = synth.rgbd()
        imgs = [torch.from_numpy(c).cuda() for _, c, _ in camera_frames(wl, 0, 4)]
        leaves = 0
        for _ in range(3):
            for im in imgs:
                leaves = int(mrh.quadtree(im, 0.1, 1).shape[0])
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": kind, "leaves_last": leaves}))
        return 0
    elif kind == "splat":
        wl = synth.rgbd()
        g = {k: torch.from_numpy(v).cuda() for k, v in synth.gaussians(wl, 1_000_000).items()}
        K = mrh.pinhole_from(wl)
        pairs = 0
        for k in range(3):
            _, _, pairs = mrh.splat_render(g["means"], g["covs"], g["opacity"], g["colors"], K, wl.pose(10 * k))
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": kind, "pairs_last": pairs}))
        return 0
    elif kind == "stream":
        # the streaming leg's LiDAR street, its pools and settings, 80 scans (eviction starts part way)
        import dataclasses
        wl = dataclasses.replace(synth.lidar(), max_blocks=(1 << 18, 1 << 16, 1 << 16))
        m = mrh.Map(mrh.params_from(wl))
        m.set_streaming(0.5, 80.0, 1 << 19)
        scene = wl.scene()
        ev = rs = 0
        for k in range(80):
            xyz, T = synth.render_lidar(wl, k, scene=scene)
            m.integrate_points(T, torch.from_numpy(xyz).cuda())
            st = m.stats()
            ev += st["evicted"]
            rs += st["restored"]
        print(json.dumps({"evicted": ev, "restored": rs, "archived": st["archived"]}))
    elif kind == "lidar":
        wl = synth.lidar()
        wl.max_blocks = (1 << 18, 1 << 16, 1 << 16)
        m = mrh.Map(mrh.params_from(wl, max_observations=1 << 24))
        scene = wl.scene()
        for k in range(4):
            xyz, T = synth.render_lidar(wl, k, scene=scene)
            m.integrate_points(T, torch.from_numpy(xyz).cuda())
            st = m.stats()
            print(json.dumps({"scan": k, "fuse_algorithmic_bytes":
                              fuse_bytes_lidar(st, wl.n_beams * wl.n_azimuth, voxel_bytes(wl))}))
    elif kind == "batched":
        # the first 8 of the 16 batched maps, 4 steps, reduced heaps (about 2 GB on the device)
        wls = synth.batched()[:8]
        for w in wls:
            w.max_blocks = (1 << 15, 1 << 13, 1 << 13)
        maps = [mrh.Map(mrh.params_from(w)) for w in wls]
        batch = mrh.Batch(maps, [mrh.pinhole_from(w) for w in wls])
        outs = [torch.empty((w.height, w.width), device="cuda") for w in wls]
        scenes = [w.scene() for w in wls]
        for k in range(4):
            fr = [synth.render_depth(w, k, scene=sc) for w, sc in zip(wls, scenes)]
            batch.integrate([(T, torch.from_numpy(d).cuda(), torch.from_numpy(c).cuda(), o)
                             for (d, c, T), o in zip(fr, outs)])
            print(json.dumps({"step": k, "fuse_algorithmic_bytes":
                              sum(fuse_bytes_camera(mm.stats(), w, voxel_bytes(w)) for mm, w in zip(maps, wls))}))
        torch.cuda.synchronize()
        batch.close()
        m = maps[0]
    else:
        # the learned level predictor: a short GPU training run on the features of 3 plain frames, then 3 frames with
        # the predictor set (reduced heaps)
        from paper_2511_21459_b300 import predictor
        wl = synth.rgbd()
        wl.max_blocks = (1 << 15, 1 << 14, 1 << 14)
        K = mrh.pinhole_from(wl)
        frames = camera_frames(wl, 0, 6)
        m0 = mrh.Map(mrh.params_from(wl))
        m0.set_feature_capture(1 << 16)
        for d, c, T in frames[:3]:
            m0.integrate_depth(K, T, torch.from_numpy(d).cuda(), torch.from_numpy(c).cuda())
        keys, feats, _ = m0.features()
        ex = m0.extract()
        y = predictor.level_labels(keys.cpu().numpy(), ex["keys"].cpu().numpy(), ex["levels"].cpu().numpy())
        ok = y >= 0
        net, _ = predictor.train(feats[torch.from_numpy(ok).cuda()].contiguous(), torch.from_numpy(y[ok]).cuda(),
                                 epochs=4, batch=4096)
        m0.close()
        m = mrh.Map(mrh.params_from(wl))
        m.set_predictor(net.weights()[1])
        for d, c, T in frames[3:]:
            m.integrate_depth(K, T, torch.from_numpy(d).cuda(), torch.from_numpy(c).cuda())
    torch.cuda.synchronize()
    st = m.stats()
    print(json.dumps({"profile_case": kind, "status": st["status_code"], "touched_last": st["touched"]}))
    return 0 if st["status_code"] == 0 else 1


def host_cpu() -> dict:
    """CPU model and logical core count of the host the oracle runs on."""
    model = "unknown"
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"cpu_model": model, "nproc": os.cpu_count()}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


# ----------------------------------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.gpu = gpu_index
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu=timestamp,{self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 10:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        smax = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[6:10]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------------------------------- helpers

def dist_setup(n_gpus):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    else:
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce_over_ranks(x: float, world: int, op: str) -> float:
    """All-reduce of one number over the ranks (a device tensor under NCCL, a host tensor under gloo)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def max_over_ranks(x: float, world: int) -> float:
    return _reduce_over_ranks(x, world, "max")


def sum_over_ranks(x: float, world: int) -> float:
    return _reduce_over_ranks(x, world, "sum")


def whole_job_rate(units: float, ms: float, world: int) -> float:
    """Units per second of the whole job: every rank's units over the slowest rank's time (weak scaling)."""
    return sum_over_ranks(units, world) / (max_over_ranks(ms, world) / 1000.0)


def camera_frames(wl, start, count):
    scene = wl.scene()
    return [synth.render_depth(wl, start + k, scene=scene) for k in range(count)]


def fuse_bytes_camera(stats, wl, s_v):
    """Algorithmic bytes of one camera fusion launch: the depth (+ colour) image once, every touched block's payload
    read and written once, its 16-byte hash entry read, and the entry of every new block written."""
    img = wl.width * wl.height * (4 + (3 if wl.has_color else 0))
    payload = sum(2 * ((8 >> l) ** 3) * s_v * n for l, n in enumerate(stats["touched_level"]))
    return img + payload + 16 * stats["touched"] + 16 * stats["new_blocks"]


def fuse_bytes_lidar(stats, n_points, s_v):
    """Algorithmic bytes of one LiDAR fusion launch: the scan's points once, every voxel the rays cross read and
    written once, and the touched blocks' 16-byte hash entries."""
    return 12 * n_points + 2 * s_v * stats["updated_voxels"] + 16 * stats["touched"]


def source_sha256(files=("mrh_fuse.cu", "mrh_fuse.cuh", "mrh_internal.cuh"), with_build=False) -> str:
    """Hash of the sources a kernel is compiled from, and optionally of the build script that holds the compiler
    flags (a stored ncu capture is used only while it matches)."""
    import hashlib
    h = hashlib.sha256()
    paths = [os.path.join(ROOT, "paper_2511_21459_b300", "csrc", f) for f in files]
    if with_build:
        paths.append(os.path.join(ROOT, "paper_2511_21459_b300", "build.py"))
    for path in paths:
        with open(path, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def fusion_source_sha256() -> str:
    return source_sha256()


LIDAR_FUSION_SOURCES = ("mrh_fuse.cu", "mrh_fuse.cuh", "mrh_internal.cuh")
BATCH_FUSE_SOURCES = ("mrh_batch.cu", "mrh_fuse.cuh", "mrh_internal.cuh")


def stored_traffic(name, files, algorithmic_bytes_per_launch):
    """DRAM bytes per launch from a stored ncu capture (profiles/<name>.json: DRAM bytes per algorithmic byte of the
    captured launches), scaled to this run's algorithmic bytes per launch; None unless the capture was taken from the
    same kernel sources."""
    path = os.path.join(ROOT, "profiles", name + ".json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        tr = json.load(f)
    if tr.get("source_sha256") != source_sha256(files):
        return None
    return int(tr["dram_bytes_per_algorithmic_byte"] * algorithmic_bytes_per_launch)


RAYCAST_SOURCES = ("mrh_raycast.cu", "mrh_raycast.cuh", "mrh_internal.cuh")


def raycast_roofline(ray_ms_avg, rays_per_launch, clk, n_sms):
    """The raycast against the instruction-issue roofline: it is bound by issue and dependent latency (0.5 % of
    HBM). achieved = warp instructions per launch / launch time, the instructions per ray taken from one ncu capture
    of the same kernel on a view of the grown map (profiles/raycast_rgbd.json) times this run's rays per launch;
    peak = SMs x 4 schedulers x one warp instruction per cycle at the highest SM clock sampled under load."""
    path = os.path.join(ROOT, "profiles", "raycast_rgbd.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        pr = json.load(f)
    if pr.get("source_sha256") != source_sha256(RAYCAST_SOURCES, with_build=True):
        return None
    mhz = float((clk or {}).get("sm_max_mhz") or pr["sm_mhz"])
    peak = n_sms * 4 * mhz * 1e6 / 1e9  # G warp instructions / s
    instr = pr["warp_instructions_per_ray"] * rays_per_launch
    ach = instr / (ray_ms_avg / 1000.0) / 1e9
    return {"kernel": "k_raycast (depth, normal, colour)", "bound": "alu", "achieved": round(ach, 1),
            "peak": round(peak, 1), "unit": "G warp instructions/s", "frac": round(ach / peak, 4),
            "peak_kind": "derived: SMs x 4 schedulers x SM clock", "traffic": None,
            "warp_instructions_per_launch": int(instr), "active_threads_per_instruction": pr["active_threads"],
            "launch_ms_avg": round(ray_ms_avg, 5)}


def voxel_bytes(wl):
    if wl.fp16:
        return 2 + (6 if wl.has_color else 0) + 8
    return 12 + (12 if wl.has_color else 0)


# ----------------------------------------------------------------------------------------------------- GPU arm

def timed_frames(n_frames, warmup, steps):
    """Indices of the timed frames: `steps` frames spread evenly over the sequence after the warm-up frames (every
    frame is integrated in order; the others untimed), so the timing covers the young and the grown map alike."""
    last = n_frames - 1
    if steps <= 1:
        return [min(warmup, last)]
    idx = sorted({warmup + (i * (last - warmup)) // (steps - 1) for i in range(steps)})
    if len(idx) < steps:  # more steps than frames after the warm-up: consecutive frames
        idx = list(range(warmup, min(warmup + steps, n_frames)))
    return idx


def run_camera_gpu(wl, frames, warmup, timed, flush, predictor=None, keep=False):
    """Integrate frames[0 .. max(timed)] in order; the first `warmup` with a raycast each, untimed; every frame in
    `timed` as one timed step (integrate + raycast of depth, normals and colour between CUDA events on the launching
    stream, L2 flushed before each); the others integrated untimed."""
    import torch
    import paper_2511_21459_b300 as mrh
    K = mrh.pinhole_from(wl)
    m = mrh.Map(mrh.params_from(wl), device=torch.cuda.current_device())
    if predictor is not None:
        m.set_predictor(predictor)
    last = max(timed)
    dev = [(torch.from_numpy(d).cuda(), torch.from_numpy(c).cuda(), T) for d, c, T in frames[:last + 1]]
    out = torch.empty((wl.height, wl.width), dtype=torch.float32, device="cuda")
    nrm = torch.empty((wl.height, wl.width, 3), dtype=torch.float32, device="cuda")
    col = torch.empty((wl.height, wl.width, 3), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for k in range(warmup):
        d, c, T = dev[k]
        m.integrate_depth(K, T, d, c)
        m.raycast(K, T, out, normals=nrm, rgb=col)
    torch.cuda.synchronize()
    tset = set(timed)
    rays, fbytes, obs = 0, 0, 0
    touched = [0, 0, 0]
    ev = []
    prof = {}
    for k in range(warmup, last + 1):
        d, c, T = dev[k]
        if k not in tset:
            m.integrate_depth(K, T, d, c)
            continue
        flush.zero_()
        torch.cuda.synchronize()
        m.set_profiling(True)
        m.profile(reset=True)
        e = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        e[0].record(stream)
        m.integrate_depth(K, T, d, c)
        m.raycast(K, T, out, normals=nrm, rgb=col)
        e[1].record(stream)
        ev.append(e)
        st = m.stats()  # synchronises (outside the timed events)
        for g, v in m.profile().items():
            a = prof.setdefault(g, [0.0, 0])
            a[0] += v[0]
            a[1] += v[1]
        m.set_profiling(False)
        if st["status_code"] != 0:
            raise RuntimeError(f"map status {st['status_code']} at frame {k}")
        rays += st["valid_rays"]
        obs += st["observations"]
        touched = [a + b for a, b in zip(touched, st["touched_level"])]
        fbytes += fuse_bytes_camera(st, wl, voxel_bytes(wl))
    torch.cuda.synchronize()
    times = [a.elapsed_time(b) for a, b in ev]
    final = m.stats()
    out = dict(ms=sum(times), ms_steps=times, rays=rays, fuse_bytes=fbytes, prof={g: tuple(v) for g, v in prof.items()},
               final=final, observations=obs, touched_level=touched)
    if keep:
        out["map"] = m
    else:
        m.close()
    return out


def chamfer_vs_truth(m, wl, views, poses=None):
    """Chamfer-L1 (Sec. 4.1.2) of the map's raycast depth at the given frames (or camera-to-world `poses`) against
    noise-free renders of the same views, both back-projected (every 2nd pixel)."""
    import dataclasses
    import paper_2511_21459_b300 as mrh
    from paper_2511_21459_b300 import metrics
    K = mrh.pinhole_from(wl)
    clean = dataclasses.replace(wl, noise_coef=0.0, dropout=0.0)
    scene = wl.scene()
    rec, gt = [], []
    for i, k in enumerate(views):
        T = wl.pose(k) if poses is None else poses[i]
        d = m.raycast(K, T).cpu().numpy()
        rec.append(metrics.backproject(d, wl.fx, wl.fy, wl.cx, wl.cy, T, stride=2))
        g, _, _ = synth.render_depth(clean, k, scene=scene, pose=T)
        g = np.where((g >= wl.min_depth) & (g <= wl.max_depth), g, 0.0)
        gt.append(metrics.backproject(g, wl.fx, wl.fy, wl.cx, wl.cy, T, stride=2))
    return metrics.chamfer(np.concatenate(rec), np.concatenate(gt))


def spread(xs):
    """Mean, minimum, maximum and relative spread ((max - min) / mean) of repeated timings."""
    xs = [float(x) for x in xs]
    mean = sum(xs) / len(xs)
    return {"mean": round(mean, 5), "min": round(min(xs), 5), "max": round(max(xs), 5),
            "spread": round((max(xs) - min(xs)) / mean, 4), "n": len(xs)}


def lidar_training_data(lw, n_scans):
    """Features and plain-rule labels of every new block of a seeded LiDAR training street (another scene seed):
    features recorded by the library as the scans are integrated, label = the block's level at the end."""
    import torch
    import paper_2511_21459_b300 as mrh
    from paper_2511_21459_b300 import predictor
    scene = lw.scene()
    m = mrh.Map(mrh.params_from(lw), device=torch.cuda.current_device())
    m.set_feature_capture(1 << 22)
    for k in range(n_scans):
        xyz, T = synth.render_lidar(lw, k, scene=scene)
        m.integrate_points(T, torch.from_numpy(xyz).cuda())
    st = m.stats()
    keys, feats, seen = m.features()
    ex = m.extract()
    y = predictor.level_labels(keys.cpu().numpy(), ex["keys"].cpu().numpy(), ex["levels"].cpu().numpy())
    ok = y >= 0
    info = {"scene_seed": lw.seed, "scans": n_scans, "records": int(seen), "live_blocks": st["live_blocks"],
            "status": st["status_code"]}
    m.close()
    return feats[torch.from_numpy(ok).cuda()].contiguous(), torch.from_numpy(y[ok]).cuda(), info


def run_learned_lidar(lw, w_bf16, net, flush, n_scans=500, warmup=3, repeats=5,
                      view_x=(25.0, 125.0, 225.0, 325.0, 425.0)):
    """The learned predictor on a fresh LiDAR street against the plain rule: both maps integrate the same n_scans
    scans (device-resident), each scan after the first `warmup` timed between CUDA events with L2 flushed before it;
    `repeats` interleaved runs of each; Chamfer-L1 of the maps' raycast depth from pinhole views down the street
    against noise-free renders; misclassification of the network against the plain rule's final levels."""
    import dataclasses
    import torch
    import paper_2511_21459_b300 as mrh
    from paper_2511_21459_b300 import predictor
    scene = lw.scene()
    dev = []
    for k in range(n_scans):
        xyz, T = synth.render_lidar(lw, k, scene=scene)
        dev.append((torch.from_numpy(xyz).cuda(), T))
    stream = torch.cuda.current_stream()

    def one(w, keep=False, capture=False):
        m = mrh.Map(mrh.params_from(lw), device=torch.cuda.current_device())
        if w is not None:
            m.set_predictor(w)
        if capture:
            m.set_feature_capture(1 << 22)
        ev, obs, rays = [], 0, 0
        touched = [0, 0, 0]
        for k, (x, T) in enumerate(dev):
            if k < warmup:
                m.integrate_points(T, x)
                continue
            flush.zero_()
            e = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            e[0].record(stream)
            m.integrate_points(T, x)
            e[1].record(stream)
            ev.append(e)
            st = m.stats()
            if st["status_code"] != 0:
                raise RuntimeError(f"LiDAR map status {st['status_code']} at scan {k}")
            obs += st["observations"]
            rays += st["valid_rays"]
            touched = [a + b for a, b in zip(touched, st["touched_level"])]
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / len(ev)
        out = {"ms_per_scan": ms, "observations": obs, "rays": rays, "touched_level": touched,
               "live_blocks": m.stats()["live_blocks"]}
        if keep:
            out["map"] = m
        else:
            m.close()
        return out

    plain_ms, learned_ms = [], []
    for r in range(repeats):
        plain_ms.append(one(None)["ms_per_scan"])
        learned_ms.append(one(w_bf16)["ms_per_scan"])
    p = one(None, keep=True, capture=True)
    q = one(w_bf16, keep=True)
    cam = dataclasses.replace(lw, sensor="camera", width=640, height=480, fx=400.0, fy=400.0, cx=319.5, cy=239.5,
                              min_depth=0.5, max_depth=60.0, extra={"scene": "lidar"})
    poses = [synth.look_at((x, 0.0, 1.8), (x + 10.0, 0.0, 1.5)) for x in view_x]
    # the bound of any predictor: every new block started at one level (constant networks)
    bound = {}
    for lv in range(1, lw.n_levels):
        c = one(predictor.constant_level_weights(lv), keep=True)
        ch = chamfer_vs_truth(c["map"], cam, list(range(len(poses))), poses=poses)
        c["map"].close()
        bound[f"all_new_at_level_{lv}"] = {"ms_per_scan": round(c["ms_per_scan"], 5),
                                           "chamfer_mm": round(1000 * ch["chamfer"], 4),
                                           "live_blocks": c["live_blocks"]}
    keys, feats, _ = p["map"].features()
    ex = p["map"].extract()
    y = predictor.level_labels(keys.cpu().numpy(), ex["keys"].cpu().numpy(), ex["levels"].cpu().numpy())
    ok = y >= 0
    xe = feats[torch.from_numpy(ok).cuda()].contiguous()
    ye = torch.from_numpy(y[ok]).cuda()
    pred = predictor.predicted_levels(net, xe)
    misclass = float((pred != ye).float().mean().item())
    ch_p = chamfer_vs_truth(p["map"], cam, list(range(len(poses))), poses=poses)
    ch_l = chamfer_vs_truth(q["map"], cam, list(range(len(poses))), poses=poses)
    p["map"].close()
    q["map"].close()
    pm, lm = spread(plain_ms), spread(learned_ms)
    rays = p["rays"] / (n_scans - warmup)
    return {"workload": f"lidar-128x2048-street, fresh scene seed {lw.seed}, {n_scans} scans ({warmup} warm-up)",
            "value": rays / (lm["mean"] / 1000.0), "unit": "points/s", "plain_value": rays / (pm["mean"] / 1000.0),
            "speedup_vs_plain": pm["mean"] / lm["mean"], "ms_per_scan": {"plain": pm, "learned": lm},
            "misclassification": round(misclass, 4),
            "label_histogram": np.bincount(ye.cpu().numpy(), minlength=3).tolist(),
            "predicted_histogram": np.bincount(pred.cpu().numpy(), minlength=3).tolist(),
            "fused_observations": {"plain": p["observations"], "learned": q["observations"]},
            "touched_blocks_per_level": {"plain": p["touched_level"], "learned": q["touched_level"]},
            "live_blocks": {"plain": p["live_blocks"], "learned": q["live_blocks"]},
            "chamfer_mm": {"plain": round(1000 * ch_p["chamfer"], 4), "learned": round(1000 * ch_l["chamfer"], 4),
                           "added": round(1000 * (ch_l["chamfer"] - ch_p["chamfer"]), 4)},
            "fscore_10cm": {"plain": round(ch_p["fscore"], 5), "learned": round(ch_l["fscore"], 5)},
            "upper_bound": bound}


def _packed_keys(keys):
    """Block keys (n, 3) int tensor -> one sortable int64 per key."""
    import torch
    k = keys.to(torch.int64) + (1 << 20)
    return (k[:, 0] << 42) | (k[:, 1] << 21) | k[:, 2]


def block_statistics(ex, rows, T, wl):
    """The 16 TSDF-statistics features of existing blocks (rows of an extract, CUDA): mean / min / max D
    over observed voxels (/ tau), mean / max variance S2 / W (/ theta_0), mean / min / max W (W / (8 + W)), the
    observed fraction, the normal spread 1 - |mean unit gradient| over observed voxels with |D| < tau, the largest W
    (frames that observed the block, W / (8 + W)), the distance r of the block centre to the sensor, the cosine
    between the viewing ray and the mean gradient, the level, E / r, the sensor type (0). Measurement code for the
    feature study; the library's own predictor reads the range image."""
    import torch
    E = float(np.float32(wl.base_voxel) / np.float32(2 ** (wl.n_levels - 1))) * 8.0
    tau, th0 = float(wl.truncation), float(wl.var_threshold[0])
    out = torch.zeros((len(rows), 16), dtype=torch.float32, device=ex["D"].device)
    lv = ex["levels"][rows].long()
    off = ex["offsets"]
    o = torch.as_tensor(T[:3, 3], dtype=torch.float32, device=out.device)
    for l in range(wl.n_levels):
        sel = (lv == l).nonzero().flatten()
        if len(sel) == 0:
            continue
        n = 8 >> l
        b = rows[sel]
        idx = off[b][:, None] + torch.arange(n ** 3, device=out.device)[None, :]
        D, W, S2 = ex["D"][idx], ex["W"][idx], ex["S2"][idx]
        obs = W > 0
        cnt = obs.sum(1).clamp(min=1).float()
        Dm = torch.where(obs, D, torch.zeros_like(D))
        var = torch.where(obs, S2 / W.clamp(min=1e-30), torch.zeros_like(D))
        big = torch.full_like(D, 1e30)
        f = torch.zeros((len(sel), 16), dtype=torch.float32, device=out.device)
        f[:, 0] = Dm.sum(1) / cnt / tau
        f[:, 1] = torch.where(obs, D, big).min(1).values.clamp(max=tau) / tau
        f[:, 2] = torch.where(obs, D, -big).max(1).values.clamp(min=-tau) / tau
        f[:, 3] = var.sum(1) / cnt / th0
        f[:, 4] = var.max(1).values / th0
        Wobs = torch.where(obs, W, torch.zeros_like(W))
        f[:, 5] = (Wobs.sum(1) / cnt) / (8.0 + Wobs.sum(1) / cnt)
        wmin = torch.where(obs, W, big).min(1).values
        wmin = torch.where(obs.any(1), wmin, torch.zeros_like(wmin))
        f[:, 6] = wmin / (8.0 + wmin)
        wmax = Wobs.max(1).values
        f[:, 7] = wmax / (8.0 + wmax)
        f[:, 8] = obs.float().mean(1)
        g = Dm.view(-1, n, n, n)  # z, y, x
        gx = torch.zeros_like(g)
        gy = torch.zeros_like(g)
        gz = torch.zeros_like(g)
        if n > 1:
            gx[:, :, :, :-1] = g[:, :, :, 1:] - g[:, :, :, :-1]
            gy[:, :, :-1, :] = g[:, :, 1:, :] - g[:, :, :-1, :]
            gz[:, :-1, :, :] = g[:, 1:, :, :] - g[:, :-1, :, :]
        gv = torch.stack([gx, gy, gz], -1).view(len(sel), -1, 3)
        gn = gv / gv.norm(dim=-1, keepdim=True).clamp(min=1e-12)
        band = (obs & (D.abs() < tau)).float()[..., None]
        mg = (gn * band).sum(1) / band.sum(1).clamp(min=1)
        f[:, 9] = 1.0 - mg.norm(dim=-1)
        f[:, 10] = f[:, 7]
        centre = (ex["keys"][b].float() + 0.5) * E - o
        r = centre.norm(dim=-1)
        f[:, 11] = r
        mgn = mg / mg.norm(dim=-1, keepdim=True).clamp(min=1e-12)
        f[:, 12] = ((centre / r[:, None]) * mgn).sum(-1)
        f[:, 13] = float(l)
        f[:, 14] = E / r
        f[:, 15] = 0.0
        out[sel] = f
    return out


def run_feature_study(wl, train_seeds=(11, 12), eval_seed=1, n_frames=100, epochs=30, obs_frames=4):
    """Which features predict a block's final level (the plain rule's) best? For every new block of each sequence:
    (a) the library's range-image features at creation; (b) TSDF statistics of the block after the frame that
    created it; (c) TSDF statistics when it has first been observed by `obs_frames` frames (an existing block). One
    network per feature set, trained by the library's kernels on the training sequences, scored on the evaluation
    sequence's blocks against the plain rule's final levels (with the all-finest answer as the baseline)."""
    import dataclasses
    import torch
    import paper_2511_21459_b300 as mrh
    from paper_2511_21459_b300 import predictor
    t0 = time.perf_counter()
    K = mrh.pinhole_from(wl)

    def sequence(seed):
        w = dataclasses.replace(wl, seed=seed)
        frs = camera_frames(w, 0, n_frames)
        m = mrh.Map(mrh.params_from(w))
        m.set_feature_capture(1 << 20)
        ka, fa, kb, fb, kc, fc = [], [], [], [], [], []
        done = torch.empty(0, dtype=torch.int64, device="cuda")
        for d, c, T in frs:
            m.integrate_depth(K, T, torch.from_numpy(d).cuda(), torch.from_numpy(c).cuda())
            keys, feats, _ = m.features(reset=True)
            ex = m.extract()
            pk = _packed_keys(ex["keys"])  # extract is sorted by key
            if len(keys):
                rows = torch.searchsorted(pk, _packed_keys(keys))
                rows = rows.clamp(max=len(pk) - 1)
                ok = pk[rows] == _packed_keys(keys)
                ka.append(keys[ok])
                fa.append(feats[ok])
                kb.append(keys[ok])
                fb.append(block_statistics(ex, rows[ok], T, w))
            # blocks whose most-observed voxel has reached obs_frames observations, first time
            nb = len(pk)
            seg = torch.repeat_interleave(torch.arange(nb, device="cuda"), ex["offsets"][1:] - ex["offsets"][:-1])
            wmax = torch.zeros(nb, device="cuda").scatter_reduce_(0, seg, ex["W"], "amax")
            cand = (wmax >= obs_frames).nonzero().flatten()
            cand = cand[~torch.isin(pk[cand], done)]
            if len(cand):
                done = torch.cat([done, pk[cand]])
                kc.append(ex["keys"][cand])
                fc.append(block_statistics(ex, cand, T, w))
        ex = m.extract()
        fk, fl = ex["keys"].cpu().numpy(), ex["levels"].cpu().numpy()
        m.close()

        def lab(ks, fs):
            ks = torch.cat(ks)
            fs = torch.cat(fs)
            y = predictor.level_labels(ks.cpu().numpy(), fk, fl)
            ok = torch.from_numpy(y >= 0).cuda()
            return fs[ok].contiguous(), torch.from_numpy(y[y >= 0]).cuda()

        return {"a": lab(ka, fa), "b": lab(kb, fb), "c": lab(kc, fc)}

    train = [sequence(sd) for sd in train_seeds]
    ev = sequence(eval_seed)
    out = {}
    names = {"a": "range image at creation (the library's predictor)", "b": "TSDF statistics after the creating frame",
             "c": f"TSDF statistics once observed by {obs_frames} frames"}
    for key, name in names.items():
        x = torch.cat([t[key][0] for t in train])
        y = torch.cat([t[key][1] for t in train])
        net, hist = predictor.train(x, y, epochs=epochs, batch=4096, lr=2e-3, seed=0)
        xe, ye = ev[key]
        pred = predictor.predicted_levels(net, xe)
        out[key] = {"features": name, "train_samples": int(x.shape[0]), "eval_samples": int(xe.shape[0]),
                    "misclassification": round(float((pred != ye).float().mean().item()), 4),
                    "all_finest_misclassification": round(float((ye != 0).float().mean().item()), 4),
                    "coarse_recall": round(float(((pred > 0) & (ye > 0)).sum().item() / max(1, (ye > 0).sum().item())), 4),
                    "train_loss": [round(hist[0], 4), round(hist[-1], 4)]}
    out["frames_per_sequence"] = n_frames
    out["train_seeds"] = list(train_seeds)
    out["eval_seed"] = eval_seed
    out["wall_s"] = round(time.perf_counter() - t0, 1)
    return out


def run_learned(wl, frames, warmup, timed, flush, plain, train_frames=150, epochs=12, lidar_train_scans=500,
                lidar_scans=500, repeats=5, cam_train_scenes=3, lidar_train_streets=2):
    """The learned level predictor against the plain rule. One network is trained on the plain rule's levels of
    other seeded RGB-D scenes and other seeded LiDAR streets (features recorded by the library, labels = final
    levels); then the RGB-D bench sequence is timed with and without it (`repeats` interleaved runs each) and a fresh
    LiDAR street likewise, comparing fused work, misclassification and Chamfer error, next to constant networks that
    start every new block at one coarser level (the most a "go coarse" predictor could change)."""
    import dataclasses
    import torch
    import paper_2511_21459_b300 as mrh
    from paper_2511_21459_b300 import predictor
    t0 = time.perf_counter()
    K = mrh.pinhole_from(wl)

    def captured_run(w, frs):
        m = mrh.Map(mrh.params_from(w))
        m.set_feature_capture(1 << 21)
        for d, c, T in frs:
            m.integrate_depth(K, T, torch.from_numpy(d).cuda(), torch.from_numpy(c).cuda())
        keys, feats, _ = m.features()
        ex = m.extract()
        y = predictor.level_labels(keys.cpu().numpy(), ex["keys"].cpu().numpy(), ex["levels"].cpu().numpy())
        ok = torch.from_numpy(y >= 0).cuda()
        m.close()
        return feats[ok].contiguous(), torch.from_numpy(y[y >= 0]).cuda()

    cam_seeds = [wl.seed + 10 + k for k in range(cam_train_scenes)]
    parts = [captured_run(w, camera_frames(w, 0, train_frames))
             for w in (dataclasses.replace(wl, seed=sd) for sd in cam_seeds)]
    xc, yc = torch.cat([a for a, _ in parts]), torch.cat([b for _, b in parts])
    lw = synth.lidar()
    parts, linfo = [], []
    for k in range(lidar_train_streets):
        a, b, info = lidar_training_data(dataclasses.replace(lw, seed=lw.seed + 10 + k), lidar_train_scans)
        parts.append((a, b))
        linfo.append(info)
    xl, yl = torch.cat([a for a, _ in parts]), torch.cat([b for _, b in parts])
    x, y = torch.cat([xc, xl]), torch.cat([yc, yl])
    tt = time.perf_counter()
    net, hist = predictor.train(x, y, epochs=epochs, batch=4096, lr=2e-3, seed=0)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - tt
    pred_c = predictor.predicted_levels(net, xc)
    pred_l = predictor.predicted_levels(net, xl)
    _, w_bf16 = net.weights()
    # misclassification on the evaluation sequence: the features of its new blocks do not depend on levels
    xe, ye = captured_run(wl, frames[:max(timed) + 1])
    misclass = float((predictor.predicted_levels(net, xe) != ye).float().mean().item())
    plain_ms, learned_ms = [], []
    for r in range(repeats):
        plain_ms.append(run_camera_gpu(wl, frames, warmup, timed, flush)["ms"] / len(timed))
        learned_ms.append(run_camera_gpu(wl, frames, warmup, timed, flush, predictor=w_bf16)["ms"] / len(timed))
    learned = run_camera_gpu(wl, frames, warmup, timed, flush, predictor=w_bf16, keep=True)
    plain_map = run_camera_gpu(wl, frames, warmup, timed, flush, keep=True)
    steps = len(timed)
    views = timed[::max(1, steps // 10)]
    ch_l = chamfer_vs_truth(learned["map"], wl, views)
    ch_p = chamfer_vs_truth(plain_map["map"], wl, views)
    learned["map"].close()
    plain_map["map"].close()
    bound = {}
    for lv in range(1, wl.n_levels):
        c = run_camera_gpu(wl, frames, warmup, timed, flush, predictor=predictor.constant_level_weights(lv), keep=True)
        ch = chamfer_vs_truth(c["map"], wl, views)
        c["map"].close()
        bound[f"all_new_at_level_{lv}"] = {"ms_per_step": round(c["ms"] / steps, 5),
                                           "chamfer_mm": round(1000 * ch["chamfer"], 4)}
    pm, lm = spread(plain_ms), spread(learned_ms)
    rays = plain["rays"] / steps
    lid = run_learned_lidar(lw, w_bf16, net, flush, n_scans=lidar_scans, repeats=repeats)
    return {"value": rays / (lm["mean"] / 1000.0), "unit": "points/s",
            "plain_value": rays / (pm["mean"] / 1000.0),
            "speedup_vs_plain": pm["mean"] / lm["mean"],
            "ms_per_step": {"plain": pm, "learned": lm},
            "misclassification": round(misclass, 4),
            "train": {"rgbd": {"scene_seeds": cam_seeds, "frames": train_frames, "samples": int(xc.shape[0]),
                               "error": round(float((pred_c != yc).float().mean().item()), 4),
                               "labels": np.bincount(yc.cpu().numpy(), minlength=3).tolist()},
                      "lidar": dict(streets=linfo, samples=int(xl.shape[0]),
                                    error=round(float((pred_l != yl).float().mean().item()), 4),
                                    labels=np.bincount(yl.cpu().numpy(), minlength=3).tolist()),
                      "samples": int(x.shape[0]), "epochs": epochs, "batch": 4096, "train_s": round(train_s, 2),
                      "loss": [round(hist[0], 4), round(hist[-1], 4)]},
            "label_histogram": np.bincount(ye.cpu().numpy(), minlength=3).tolist(),
            "fused_observations": {"plain": plain_map["observations"], "learned": learned["observations"]},
            "touched_blocks_per_level": {"plain": plain_map["touched_level"], "learned": learned["touched_level"]},
            "chamfer_mm": {"plain": round(1000 * ch_p["chamfer"], 4), "learned": round(1000 * ch_l["chamfer"], 4),
                           "added": round(1000 * (ch_l["chamfer"] - ch_p["chamfer"]), 4)},
            "fscore_10cm": {"plain": round(ch_p["fscore"], 5), "learned": round(ch_l["fscore"], 5)},
            "kernels_ms": {"plain": {g: round(v[0], 3) for g, v in plain_map["prof"].items() if v[1] > 0},
                           "learned": {g: round(v[0], 3) for g, v in learned["prof"].items() if v[1] > 0}},
            "upper_bound": bound,
            "lidar": lid,
            "wall_s": round(time.perf_counter() - t0, 1)}


def run_camera_e2e(wl, frames, warmup, timed, flush):
    """The same timed frames through the public API with host buffers: each timed step copies its depth + colour
    frame from pinned host memory to the device, integrates it, raycasts it and copies the raycast depth, normals and
    colours back to pinned host memory, all on one stream between the step's CUDA events (no overlap with other
    steps), with L2 flushed before each step as in the device-timed arm. Untimed frames are integrated from device
    copies made outside the timed region."""
    import torch
    import paper_2511_21459_b300 as mrh
    K = mrh.pinhole_from(wl)
    m = mrh.Map(mrh.params_from(wl), device=torch.cuda.current_device())
    last = max(timed)
    tset = set(timed)
    host = [(torch.from_numpy(d).pin_memory(), torch.from_numpy(c).pin_memory(), T) for d, c, T in frames[:last + 1]]
    d_dev = torch.empty((wl.height, wl.width), dtype=torch.float32, device="cuda")
    c_dev = torch.empty((wl.height, wl.width, 3), dtype=torch.uint8, device="cuda")
    out = torch.empty((wl.height, wl.width), dtype=torch.float32, device="cuda")
    nrm = torch.empty((wl.height, wl.width, 3), dtype=torch.float32, device="cuda")
    col = torch.empty((wl.height, wl.width, 3), dtype=torch.uint8, device="cuda")
    out_host = torch.empty((wl.height, wl.width), dtype=torch.float32).pin_memory()
    nrm_host = torch.empty((wl.height, wl.width, 3), dtype=torch.float32).pin_memory()
    col_host = torch.empty((wl.height, wl.width, 3), dtype=torch.uint8).pin_memory()
    stream = torch.cuda.current_stream()
    ms = 0.0
    for k in range(last + 1):
        d, c, T = host[k]
        if k < warmup or k not in tset:
            d_dev.copy_(d, non_blocking=True)
            c_dev.copy_(c, non_blocking=True)
            m.integrate_depth(K, T, d_dev, c_dev)
            if k < warmup:
                m.raycast(K, T, out, normals=nrm, rgb=col)
            continue
        flush.zero_()
        torch.cuda.synchronize()
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        d_dev.copy_(d, non_blocking=True)
        c_dev.copy_(c, non_blocking=True)
        m.integrate_depth(K, T, d_dev, c_dev)
        m.raycast(K, T, out, normals=nrm, rgb=col)
        out_host.copy_(out, non_blocking=True)
        nrm_host.copy_(nrm, non_blocking=True)
        col_host.copy_(col, non_blocking=True)
        z.record(stream)
        torch.cuda.synchronize()
        ms += a.elapsed_time(z)
    m.close()
    h2d = wl.width * wl.height * (4 + 3)
    d2h = wl.width * wl.height * (4 + 12 + 3)
    return ms, h2d, d2h


def mesh_bytes(stats, wl, n_tris):
    """Algorithmic bytes of one mesh extraction: every voxel's distance and weight read once, 36 B per triangle."""
    per_voxel = (2 if wl.fp16 else 4) + 4
    voxels = sum(n * (8 >> l) ** 3 for l, n in enumerate(stats["live_blocks"]))
    return voxels * per_voxel + 36 * n_tris


def run_mesh(wl, m, reps=5, prefix=(0, 10, 20, 30)):
    """Multi-resolution Marching Cubes (Sec. 3.4): the whole map the benchmark built (device time of the extraction
    kernel, from the library's event profiler, average of `reps`), and a small map of the sequence's frames `prefix`
    on the GPU and in the oracle (one thread), the same triangles timed on both."""
    import torch
    import oracle
    import paper_2511_21459_b300 as mrh
    n = len(m.extract_mesh())
    m.set_profiling(True)
    m.profile(reset=True)
    for _ in range(reps):
        m.extract_mesh(capacity=n)
    torch.cuda.synchronize()
    kms = m.profile()["mesh"][0] / reps
    st = m.stats()
    b = mesh_bytes(st, wl, n)
    full = {"triangles": n, "ms": round(kms, 4), "triangles_per_s": n / (kms / 1000.0),
            "algorithmic_bytes": b, "achieved_GBps": round(b / (kms / 1000.0) / 1e9, 1),
            "live_blocks": st["live_blocks"]}
    # vertex collapse on a grid of an eighth of the finest voxel: the paper's vertex / face counts (memory proxy)
    delta = wl.base_voxel / (1 << (wl.n_levels - 1)) / 8
    soup = m.extract_mesh(capacity=n)
    m.profile(reset=True)
    verts, faces = m.weld_mesh(soup, delta)
    torch.cuda.synchronize()
    full.update({"collapse_delta_m": delta, "vertices": int(verts.shape[0]), "faces": int(faces.shape[0]),
                 "collapse_ms": round(m.profile()["mesh"][0] / 2, 4)})
    del soup, verts, faces
    # the same small map on both sides
    scene = wl.scene()
    frames = [synth.render_depth(wl, k, scene=scene) for k in prefix]
    g = mrh.Map(mrh.params_from(wl), device=torch.cuda.current_device())
    o = oracle.OracleMap(oracle.params_from(wl, "f32s"))
    Kg, Ko = mrh.pinhole_from(wl), oracle.pinhole_from(wl)
    for d, c, T in frames:
        g.integrate_depth(Kg, T, torch.from_numpy(d).cuda(), torch.from_numpy(c).cuda())
        o.integrate_depth(Ko, T, d, c)
    ng = len(g.extract_mesh())
    g.set_profiling(True)
    g.profile(reset=True)
    for _ in range(reps):
        g.extract_mesh(capacity=ng)
    torch.cuda.synchronize()
    gms = g.profile()["mesh"][0] / reps
    t0 = time.perf_counter()
    no = len(o.extract_mesh())
    cms = 1000.0 * (time.perf_counter() - t0)
    g.close()
    o.close()
    small = {"frames": list(prefix), "triangles_gpu": ng, "triangles_oracle": no, "gpu_ms": round(gms, 4),
             "oracle_ms_1_thread": round(cms, 1), "gpu_triangles_per_s": ng / (gms / 1000.0),
             "oracle_triangles_per_s": no / (cms / 1000.0)}
    return {"full_map": full, "prefix_map": small}


def run_quadtree(wl, frames, reps=3, threshold=0.1, min_size=1, oracle_frames=3):
    """Contrast quadtree (Sec. 3.5, Eq. 10, Algorithm 1; the paper's threshold 0.1, minimum size 1 px) of the colour
    frames of the sequence: device time per frame (CUDA events on the stream around the call, which includes its
    scratch allocation and the leaf-count read-back), leaves per frame, and the oracle (one thread) on the first frames,
    with the leaf sets checked equal."""
    import torch
    import oracle
    import paper_2511_21459_b300 as mrh
    imgs = [torch.from_numpy(c).cuda() for _, c, _ in frames]
    stream = torch.cuda.current_stream()
    for im in imgs[:2]:
        mrh.quadtree(im, threshold, min_size)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_leaves = 0
    a.record(stream)
    for _ in range(reps):
        for im in imgs:
            n_leaves += int(mrh.quadtree(im, threshold, min_size).shape[0])
    b.record(stream)
    torch.cuda.synchronize()
    gms = a.elapsed_time(b) / (reps * len(imgs))
    t0 = time.perf_counter()
    same = True
    for (_, c, _), im in zip(frames[:oracle_frames], imgs):
        o = oracle.quadtree(c, threshold, min_size)
        g = mrh.quadtree(im, threshold, min_size).cpu().numpy()
        same = same and len(o) == len(g) and np.array_equal(o[np.lexsort(o.T[::-1])], g[np.lexsort(g.T[::-1])])
    cms = 1000.0 * (time.perf_counter() - t0) / oracle_frames
    return {"frames": len(imgs), "threshold": threshold, "min_size": min_size,
            "leaves_per_frame": n_leaves / (reps * len(imgs)), "gpu_ms_per_frame": round(gms, 4),
            "frames_per_s": 1000.0 / gms, "oracle_ms_per_frame_1_thread": round(cms, 2),
            "oracle_frames_checked_equal": same}


def run_ablation(wl, n_frames=120, sigmas=(0.001, 0.003, 0.006, 0.01, 0.02, 0.04), views=(20, 50, 80, 110),
                 singles=(0.01, 0.02, 0.04)):
    """Variance-threshold sweep on the RGB-D sequence (the synthetic analogue of Sec. 5.1): for each sigma the
    thresholds are (sigma^2, 4 sigma^2); then single-resolution maps with one level of each voxel size in `singles`
    (the single- vs multi-resolution comparison), same truncation. After n_frames frames each row reports the device
    time per frame (integration only), blocks and payload bytes per level, the collapsed mesh's vertices and faces
    (one collapse spacing for every row: an eighth of the finest multi-resolution voxel), and accuracy, completeness
    and Chamfer-L1 of the map's raycast depth against noise-free renders at `views`."""
    import dataclasses
    import torch
    import paper_2511_21459_b300 as mrh
    frames = camera_frames(wl, 0, n_frames)
    dev = [(torch.from_numpy(d).cuda(), torch.from_numpy(c).cuda(), T) for d, c, T in frames]
    warm = mrh.Map(mrh.params_from(wl), device=torch.cuda.current_device())  # first-use costs outside the timing
    for d, c, T in dev[:10]:
        warm.integrate_depth(mrh.pinhole_from(wl), T, d, c)
    torch.cuda.synchronize()
    warm.close()
    out = []
    delta = wl.voxel0 / 8
    rows = [(f"sigma {sig}", dataclasses.replace(wl, var_threshold=(sig * sig, 4 * sig * sig)), sig) for sig in sigmas]
    rows += [(f"single {v * 100:g} cm", dataclasses.replace(wl, base_voxel=v, n_levels=1), None) for v in singles]
    for label, w2, sig in rows:
        m = mrh.Map(mrh.params_from(w2), device=torch.cuda.current_device())
        K = mrh.pinhole_from(w2)
        stream = torch.cuda.current_stream()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for d, c, T in dev:
            m.integrate_depth(K, T, d, c)
        b.record(stream)
        torch.cuda.synchronize()
        st = m.stats()
        vb = voxel_bytes(w2)
        live = st["live_blocks"]
        soup = m.extract_mesh()
        verts, faces = m.weld_mesh(soup, delta)
        ch = chamfer_vs_truth(m, w2, views)
        out.append({"map": label, "levels_cm": [round(100 * w2.voxel0 * (1 << l), 3) for l in range(w2.n_levels)],
                    "sigma": sig, "theta": [sig * sig, 4 * sig * sig] if sig else None,
                    "ms_per_frame": round(a.elapsed_time(b) / n_frames, 4),
                    "live_blocks": live, "payload_MB": [round(n * (8 >> l) ** 3 * vb / 1e6, 1) for l, n in enumerate(live)],
                    "vertices": int(verts.shape[0]), "faces": int(faces.shape[0]),
                    "acc_mm": round(1e3 * ch["acc"], 3), "comp_mm": round(1e3 * ch["comp"], 3),
                    "chamfer_mm": round(1e3 * ch["chamfer"], 3)})
        del soup, verts, faces
        m.close()
    return out


def run_ablation_lidar(n_scans=40, sigmas=(0.01, 0.02, 0.04, 0.08), singles=(0.05, 0.1, 0.2),
                       view_x=(5.0, 15.0, 25.0, 35.0)):
    """The same sweep on the LiDAR street (FP16 storage): n_scans scans, thresholds (sigma^2, 4 sigma^2), then
    single-resolution maps of each voxel size in `singles` (same truncation). Chamfer-L1 of the map's raycast depth
    from 640 x 480 pinhole views at 1.8 m height looking down the street from x = `view_x`, against noise-free renders
    of the street from the same views."""
    import dataclasses
    import torch
    import paper_2511_21459_b300 as mrh
    lw = synth.lidar()
    scene = lw.scene()
    scans = [synth.render_lidar(lw, k, scene=scene) for k in range(n_scans)]
    dev = [(torch.from_numpy(x).cuda(), T) for x, T in scans]
    poses = [synth.look_at((x, 0.0, 1.8), (x + 10.0, 0.0, 1.5)) for x in view_x]
    out = []
    rows = [(f"sigma {sig}", dataclasses.replace(lw, var_threshold=(sig * sig, 4 * sig * sig)), sig) for sig in sigmas]
    rows += [(f"single {v * 100:g} cm", dataclasses.replace(lw, base_voxel=v, n_levels=1), None) for v in singles]
    for label, w2, sig in rows:
        m = mrh.Map(mrh.params_from(w2), device=torch.cuda.current_device())
        stream = torch.cuda.current_stream()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for x, T in dev:
            m.integrate_points(T, x)
        b.record(stream)
        torch.cuda.synchronize()
        st = m.stats()
        vb = voxel_bytes(w2)
        live = st["live_blocks"]
        cam = dataclasses.replace(w2, sensor="camera", width=640, height=480, fx=400.0, fy=400.0, cx=319.5, cy=239.5,
                                  min_depth=0.5, max_depth=60.0, extra={"scene": "lidar"})
        ch = chamfer_vs_truth(m, cam, list(range(len(poses))), poses=poses)
        out.append({"map": label, "levels_cm": [round(100 * w2.voxel0 * (1 << l), 3) for l in range(w2.n_levels)],
                    "sigma": sig, "theta": [sig * sig, 4 * sig * sig] if sig else None,
                    "ms_per_scan": round(a.elapsed_time(b) / n_scans, 4), "status": st["status_code"],
                    "live_blocks": live, "payload_MB": [round(n * (8 >> l) ** 3 * vb / 1e6, 1) for l, n in enumerate(live)],
                    "acc_mm": round(1e3 * ch["acc"], 3), "comp_mm": round(1e3 * ch["comp"], 3),
                    "chamfer_mm": round(1e3 * ch["chamfer"], 3)})
        m.close()
    return out


def run_splat(wl, n=1_000_000, views=tuple(range(0, 300, 20)), reps=3, small=((150, 110), 20000, 20)):
    """Tile-based splat rendering (Sec. 3.5, Eqs. 7-9): n seeded Gaussians on the scene's surfaces rendered at the
    640 x 480 camera from `views` of the orbit, `reps` times each (CUDA events around the calls, which include the
    library's one host read of the pair count per render); and a small camera and Gaussian set rendered by the GPU
    and by the oracle (one thread, brute force over every pixel and Gaussian), the images checked within 2e-4."""
    import dataclasses
    import torch
    import oracle
    import paper_2511_21459_b300 as mrh
    g = synth.gaussians(wl, n)
    gd = {k: torch.from_numpy(v).cuda() for k, v in g.items()}
    K = mrh.pinhole_from(wl)
    out = torch.empty((wl.height, wl.width, 3), device="cuda")
    tr = torch.empty((wl.height, wl.width), device="cuda")
    args = (gd["means"], gd["covs"], gd["opacity"], gd["colors"], K)
    for v in views[:3]:
        mrh.splat_render(*args, wl.pose(v), out=out, trans=tr)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pairs = 0
    a.record(stream)
    for _ in range(reps):
        for v in views:
            pairs += mrh.splat_render(*args, wl.pose(v), out=out, trans=tr)[2]
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / (reps * len(views))
    (w, h), n_small, view = small
    s = w / wl.width
    ws = dataclasses.replace(wl, width=w, height=h, fx=wl.fx * s, fy=wl.fy * s, cx=(w - 1) / 2, cy=(h - 1) / 2)
    gs = synth.gaussians(wl, n_small)
    gsd = {k: torch.from_numpy(v).cuda() for k, v in gs.items()}
    Ks = mrh.pinhole_from(ws)
    T = ws.pose(view)
    mrh.splat_render(gsd["means"], gsd["covs"], gsd["opacity"], gsd["colors"], Ks, T)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(10):
        rgb_g, tr_g, _ = mrh.splat_render(gsd["means"], gsd["covs"], gsd["opacity"], gsd["colors"], Ks, T)
    b.record(stream)
    torch.cuda.synchronize()
    small_gpu_ms = a.elapsed_time(b) / 10
    t0 = time.perf_counter()
    rgb_o, tr_o, _ = oracle.splat_render(gs["means"], gs["covs"], gs["opacity"], gs["colors"], oracle.pinhole_from(ws), T)
    small_cpu_ms = 1000.0 * (time.perf_counter() - t0)
    err = max(float(np.abs(rgb_g.cpu().numpy() - rgb_o).max()), float(np.abs(tr_g.cpu().numpy() - tr_o).max()))
    return {"gaussians": n, "views": len(views), "reps": reps, "ms_per_frame": round(ms, 4),
            "frames_per_s": round(1000.0 / ms, 1), "gaussians_per_s": n * 1000.0 / ms,
            "pairs_per_frame": pairs / (reps * len(views)),
            "small_case": {"camera": [w, h], "gaussians": n_small, "gpu_ms": round(small_gpu_ms, 4),
                           "oracle_ms_1_thread": round(small_cpu_ms, 1), "max_abs_diff": err, "within_2e-4": err <= 2e-4}}


def run_streaming(wl, n_scans=150, pools=(1 << 18, 1 << 16, 1 << 16), fraction=0.5, radius=80.0,
                  archive=1 << 19):
    """Capacity-driven streaming (Sec. 3.3) on the LiDAR street: n_scans full scans 1 m apart into pools of `pools`
    blocks, streaming on at `fraction` with a `radius` m LiDAR radius; the same scans without streaming for the block
    count it would reach. Device time per scan (CUDA events over all scans, eviction and restore included)."""
    import dataclasses
    import torch
    import paper_2511_21459_b300 as mrh
    w2 = dataclasses.replace(wl, max_blocks=pools)
    scene = w2.scene()
    scans = [synth.render_lidar(w2, k, scene=scene) for k in range(n_scans)]
    dev = [(torch.from_numpy(x).cuda(), T) for x, T in scans]
    res = {}
    for on in (True, False):
        m = mrh.Map(mrh.params_from(w2), device=torch.cuda.current_device())
        if on:
            m.set_streaming(fraction, radius, archive)
        stream = torch.cuda.current_stream()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev = rs = rays = done = 0
        peak = 0
        a.record(stream)
        for x, T in dev:
            m.integrate_points(T, x)
            st = m.stats()
            if st["status_code"] != 0:
                break
            done += 1
            ev += st["evicted"]
            rs += st["restored"]
            rays += st["valid_rays"]
            peak = max(peak, sum(st["live_blocks"]))
        b.record(stream)
        torch.cuda.synchronize()
        st = m.stats()
        key = "streaming" if on else "no_streaming"
        res[key] = {"scans": done, "status": st["status_code"],
                    "ms_per_scan": round(a.elapsed_time(b) / max(done, 1), 4),
                    "points_per_s": rays / (a.elapsed_time(b) / 1000.0), "peak_resident_blocks": peak,
                    "resident_blocks_end": sum(st["live_blocks"]), "evicted": ev, "restored": rs,
                    "archived_end": st["archived"]}
        m.close()
    res.update({"pools": list(pools), "fraction": fraction, "radius_m": radius, "archive_blocks": archive,
                "note": "stats are read after every scan (a host sync inside the timed span, both runs alike)"})
    return res


def run_lidar_gpu(wl, warmup, steps, flush):
    import torch
    import paper_2511_21459_b300 as mrh
    scene = wl.scene()
    scans = [synth.render_lidar(wl, k, scene=scene) for k in range(warmup + steps)]
    dev = [(torch.from_numpy(x).cuda(), T) for x, T in scans]
    m = mrh.Map(mrh.params_from(wl), device=torch.cuda.current_device())
    for k in range(warmup):
        m.integrate_points(dev[k][1], dev[k][0])
    torch.cuda.synchronize()
    m.set_profiling(True)
    m.profile(reset=True)
    stream = torch.cuda.current_stream()
    rays, ms, fbytes = 0, 0.0, 0
    for k in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        m.integrate_points(dev[warmup + k][1], dev[warmup + k][0])
        b.record(stream)
        st = m.stats()
        if st["status_code"] != 0:
            raise RuntimeError(f"LiDAR map status {st['status_code']} at step {k}")
        ms += a.elapsed_time(b)
        rays += st["valid_rays"]
        fbytes += fuse_bytes_lidar(st, wl.n_beams * wl.n_azimuth, voxel_bytes(wl))
    prof = m.profile()
    m.close()
    return dict(ms=ms, rays=rays, steps=steps, prof=prof, fuse_bytes=fbytes)


def run_batched(warmup, steps, flush):
    """16 maps with uneven frame sizes (integrate + raycast per map per step): the per-map API ("plain") against one
    batched call per step (graph-captured after autotuning), on the same frames; both time steps after warm-up."""
    import torch
    import paper_2511_21459_b300 as mrh
    wls = synth.batched()
    for wl in wls:
        wl.max_blocks = (1 << 17, 1 << 16, 1 << 16)
    n_frames = warmup + steps
    frames = []
    for wl in wls:
        sc = wl.scene()
        frames.append([(torch.from_numpy(d).cuda(), torch.from_numpy(c).cuda(), T)
                       for d, c, T in (synth.render_depth(wl, k, scene=sc) for k in range(n_frames))])
    cams = [mrh.pinhole_from(wl) for wl in wls]
    outs = [torch.empty((wl.height, wl.width), device="cuda") for wl in wls]
    stream = torch.cuda.Stream()

    def timed(step_fn, after=None):
        ms, rays = 0.0, 0
        for k in range(n_frames):
            flush.zero_()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                a.record(stream)
                step_fn(k)
                b.record(stream)
            stream.synchronize()
            if k >= warmup:
                ms += a.elapsed_time(b)
            if after is not None:
                after(k)
        return ms

    plain_maps = [mrh.Map(mrh.params_from(wl)) for wl in wls]

    def plain_step(k):
        for i in range(len(wls)):
            d, c, T = frames[i][k]
            plain_maps[i].integrate_depth(cams[i], T, d, c, stream=stream)
            plain_maps[i].raycast(cams[i], T, outs[i], stream=stream)

    ms_plain = timed(plain_step)
    rays = 0
    for m in plain_maps:
        rays += m.stats()["valid_rays"]
    batch_maps = [mrh.Map(mrh.params_from(wl)) for wl in wls]
    batch = mrh.Batch(batch_maps, cams)
    fuse = {"ms": 0.0, "bytes": 0, "steps": 0}

    def batch_step(k):
        batch.integrate([(frames[i][k][2], frames[i][k][0], frames[i][k][1], outs[i]) for i in range(len(wls))],
                        stream=stream)

    def batch_fuse_account(k):
        # the fusion kernel's own device time (events at the phase boundaries of the step, inside the graph) and the
        # algorithmic bytes of every map's fusion in this step
        if k < warmup:
            return
        fuse["ms"] += batch.last_step_ms()["fuse"]
        fuse["bytes"] += sum(fuse_bytes_camera(m.stats(), wl, voxel_bytes(wl)) for m, wl in zip(batch_maps, wls))
        fuse["steps"] += 1

    ms_batch = timed(batch_step, after=batch_fuse_account)
    # valid rays of the timed steps (identical in both forms; counted from the depth images)
    rays_timed = 0
    for i, wl in enumerate(wls):
        for k in range(warmup, n_frames):
            d = frames[i][k][0]
            rays_timed += int(((d >= wl.min_depth) & (d <= wl.max_depth)).sum().item())
    cfg = batch.config()
    batch.close()
    for m in plain_maps + batch_maps:
        m.close()
    return dict(rays=rays_timed, ms_plain=ms_plain, ms_batch=ms_batch, config=cfg,
                sizes=[f"{wl.width}x{wl.height}" for wl in wls], fuse=fuse)


# ----------------------------------------------------------------------------------------------------- CPU oracle

def oracle_camera_sample(wl, frames, budget_s, max_frames):
    """The CPU oracle (f32s mode, single thread) on the first frames of the same sequence: integrate + raycast."""
    import oracle
    om = oracle.OracleMap(oracle.params_from(wl, "f32s"))
    K = oracle.pinhole_from(wl)
    rays, t_total, n = 0, 0.0, 0
    for depth, rgb, T in frames[:max_frames]:
        t0 = time.perf_counter()
        st = om.integrate_depth(K, T, depth, rgb)
        om.raycast(K, T, normals=True, rgb=True)
        t_total += time.perf_counter() - t0
        rays += st["valid_rays"]
        n += 1
        if t_total > budget_s:
            break
    om.close()
    return rays, t_total, n


def _oracle_replica(seed_frames, budget_s, barrier, queue):
    """One CPU replica (a process of its own): the oracle map on the first frames of the sequence."""
    import oracle
    wl = synth.rgbd()
    scene = wl.scene()
    frames = [synth.render_depth(wl, k, scene=scene) for k in range(seed_frames)]
    om = oracle.OracleMap(oracle.params_from(wl, "f32s"))
    K = oracle.pinhole_from(wl)
    barrier.wait()
    rays, t_total, n = 0, 0.0, 0
    for depth, rgb, T in frames:
        t0 = time.perf_counter()
        st = om.integrate_depth(K, T, depth, rgb)
        om.raycast(K, T, normals=True, rgb=True)
        t_total += time.perf_counter() - t0
        rays += st["valid_rays"]
        n += 1
        if t_total > budget_s:
            break
    queue.put((rays, t_total, n))


def oracle_camera_replicas(n_procs, n_frames, budget_s):
    """Independent oracle replicas, one map per process on every host core (started with spawn, before any GPU work);
    aggregate points/s = all replicas' points / the slowest replica's time."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(n_procs)
    queue = ctx.Queue()
    procs = [ctx.Process(target=_oracle_replica, args=(n_frames, budget_s, barrier, queue)) for _ in range(n_procs)]
    for p in procs:
        p.start()
    res = [queue.get() for _ in procs]
    for p in procs:
        p.join()
    return sum(r[0] for r in res), max(r[1] for r in res), min(r[2] for r in res)


def main():
    args = parse_args()
    if args.profile_case:
        return profile_case(args.profile_case)
    wl = synth.rgbd()
    hbm, peak_kind = peaks()

    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        if rank != 0:
            return 0
        warm = min(args.warmup, 1)
        frames = camera_frames(wl, 0, warm + min(args.steps, 200))
        import oracle
        om = oracle.OracleMap(oracle.params_from(wl, "f32s"))
        K = oracle.pinhole_from(wl)
        for depth, rgb, T in frames[:warm]:
            om.integrate_depth(K, T, depth, rgb)
            om.raycast(K, T, normals=True, rgb=True)
        rays, t_total, n = 0, 0.0, 0
        budget = 150.0
        for depth, rgb, T in frames[warm:]:
            t0 = time.perf_counter()
            st = om.integrate_depth(K, T, depth, rgb)
            om.raycast(K, T, normals=True, rgb=True)
            t_total += time.perf_counter() - t0
            rays += st["valid_rays"]
            n += 1
            if t_total > budget:
                break
        value = rays / t_total
        sample = (f"frames {warm}..{warm + n - 1} of the RGB-D sequence after {warm} untimed, integrate + full "
                  f"640x480 raycast (depth, normal, colour) per frame, oracle f32s mode, 1 thread (time-boxed at "
                  f"{budget:.0f} s)")
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": args.gpus,
                "steps": n, "warmup": warm, "ms_per_step": 1000.0 * t_total / n, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": RGBD_WORKLOAD},
                "frames_per_s": n / t_total,
                "cpu_baseline": {"value": value, "unit": "points/s", "cores": 1, "kind": "oracle", "sample": sample,
                                 "host": host_cpu()},
                "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    import torch
    if args.ablation:
        from paper_2511_21459_b300 import build as _b
        _b.build()
        print(json.dumps({"ablation": run_ablation(wl), "workload": "rgbd-640x480 sequence, first 120 frames",
                          "lidar": run_ablation_lidar(), "lidar_workload": "lidar-128x2048 street, first 40 scans",
                          "data": "synthetic"}))
        return 0
    rank, world, local = dist_setup(args.gpus)
    from paper_2511_21459_b300 import build
    if rank == 0 or local == 0:
        build.build()
    barrier(world)

    n_frames = max(wl.n_frames, args.warmup + args.steps)
    frames = camera_frames(wl, 0, n_frames)
    timed = timed_frames(n_frames, args.warmup, args.steps)

    # CPU baseline first (host only, before the GPU work is timed)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rays_c, t_c, n_c = oracle_camera_sample(wl, frames, args.cpu_budget_s, 8)
        cpu = {"value": rays_c / t_c, "unit": "points/s", "cores": 1, "kind": "oracle", "host": host_cpu(),
               "sample": f"first {n_c} frames of the RGB-D sequence, integrate + full 640x480 raycast (depth, "
                         f"normal, colour) each, f32s mode, single thread ({t_c:.1f} s)"}
        n_procs = max(1, min(args.cpu_replicas, os.cpu_count() or 1))
        if n_procs > 1:
            rays_r, t_r, n_r = oracle_camera_replicas(n_procs, 4, args.cpu_budget_s)
            cpu["replicas"] = {"value": rays_r / t_r, "unit": "points/s", "cores": n_procs,
                               "sample": f"{n_procs} independent oracle maps, one process per core, each on the "
                                         f"first {n_r} frames ({t_r:.1f} s for the slowest)"}

    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    res = run_camera_gpu(wl, frames, args.warmup, timed, flush, keep=True)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    main_map = res.pop("map")

    ms_max = max_over_ranks(res["ms"], world)
    rays_all = sum_over_ranks(res["rays"], world)
    value = rays_all / (ms_max / 1000.0)
    fps = world * args.steps / (ms_max / 1000.0)

    prof = res["prof"]
    step_ms_sum = res["ms"]
    kernels = {g: {"ms_total": round(v[0], 4), "launches": int(v[1]), "share": round(v[0] / step_ms_sum, 4)}
               for g, v in prof.items() if v[1] > 0}
    launches = sum(v[1] for v in prof.values())
    fuse_ms = prof["fuse"][0]
    achieved = res["fuse_bytes"] / (fuse_ms / 1000.0) / 1e9
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "fuse_depth_rgbd.json")
    if os.path.exists(tpath):
        with open(tpath) as f:
            tr = json.load(f)
        if tr.get("source_sha256") == fusion_source_sha256():
            # one ncu capture of a full-size frame of the same sequence, scaled to this run's launches by the
            # algorithmic bytes (units) they process
            traffic = int(tr["dram_bytes_per_algorithmic_byte"] * res["fuse_bytes"] / args.steps)
    roofline_ray = None
    if prof.get("raycast", (0, 0))[1] > 0:
        n_sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        roofline_ray = raycast_roofline(prof["raycast"][0] / prof["raycast"][1], wl.width * wl.height, clk, n_sms)
    roofline = {"kernel": "k_fuse_depth (fusion + block variance + re-level)", "bound": "hbm",
                "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s", "frac": round(achieved / hbm, 4),
                "peak_kind": peak_kind, "traffic": traffic,
                "algorithmic_bytes_per_launch": int(res["fuse_bytes"] / args.steps),
                "launch_ms_avg": round(fuse_ms / args.steps, 5)}

    e2e = None
    if world >= 1:
        e_ms, h2d, d2h = run_camera_e2e(wl, frames, args.warmup, timed, flush)
        e_ms = max_over_ranks(e_ms, world)
        e2e = {"value": rays_all / (e_ms / 1000.0), "unit": "points/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": e_ms / args.steps,
               "note": "each timed step uploads its depth + colour frame from pinned host memory, integrates, raycasts "
                       "and reads depth, normals and colours back to pinned host memory on one stream, with no overlap "
                       "between steps; L2 flushed before each step as in the device-timed arm"}

    mesh = None
    if rank == 0 and not args.no_mesh:
        mesh = run_mesh(wl, main_map)
    main_map.close()
    quad = None
    if rank == 0 and not args.no_quadtree:
        quad = run_quadtree(wl, frames[:20])

    lidar = None
    roofline_lidar = None
    if not args.no_lidar:
        lw = synth.lidar()
        lres = run_lidar_gpu(lw, 3, args.lidar_steps, flush)
        l_ms = max_over_ranks(lres["ms"], world)
        l_rays = sum_over_ranks(lres["rays"], world)
        lprof = lres["prof"]
        lidar = {"value": l_rays / (l_ms / 1000.0), "unit": "points/s", "frames_per_s": world * lres["steps"] /
                 (l_ms / 1000.0), "steps": lres["steps"], "ms_per_step": l_ms / lres["steps"],
                 "workload": "lidar-128x2048-street (3 levels 5/10/20 cm, tau 60 cm, FP16 storage)",
                 "kernels": {g: {"ms_total": round(v[0], 3), "launches": int(v[1])} for g, v in lprof.items()
                             if v[1] > 0},
                 "fuse_achieved_GBps": round(lres["fuse_bytes"] / (lprof["fuse"][0] / 1000.0) / 1e9, 1)}
        # fusion of a scan = the observation passes (grouping the rays' voxel crossings) + the fusion kernel
        l_fuse_ms = lprof["fuse"][0] + lprof.get("lidar_obs", (0.0, 0))[0]
        l_ach = lres["fuse_bytes"] / (l_fuse_ms / 1000.0) / 1e9
        roofline_lidar = {"kernel": "LiDAR fusion: observation passes + k_fuse_points (fusion + block variance + "
                                    "re-level)", "bound": "hbm", "achieved": round(l_ach, 1), "peak": hbm,
                          "unit": "GB/s", "frac": round(l_ach / hbm, 4), "peak_kind": peak_kind,
                          "traffic": stored_traffic("lidar_fusion_traffic", LIDAR_FUSION_SOURCES,
                                                    lres["fuse_bytes"] / lres["steps"]),
                          "algorithmic_bytes_per_launch": int(lres["fuse_bytes"] / lres["steps"]),
                          "launch_ms_avg": round(l_fuse_ms / lres["steps"], 5),
                          "bytes_formula": "12 N_points + 2 s_v updated_voxels + 16 touched (s_v = 10 B, FP16, no "
                                           "colour)"}
        lidar["roofline"] = roofline_lidar

    streaming = None
    if rank == 0 and not args.no_lidar and not args.no_streaming:
        streaming = run_streaming(synth.lidar())

    splat = None
    if rank == 0 and not args.no_splat:
        splat = run_splat(wl)

    batched = None
    if not args.no_batched:
        bres = run_batched(6, args.batched_steps, flush)
        b_ms = max_over_ranks(bres["ms_batch"], world)
        p_ms = max_over_ranks(bres["ms_plain"], world)
        rays_b = sum_over_ranks(bres["rays"], world)
        batched = {"value": rays_b / (b_ms / 1000.0), "unit": "points/s",
                   "plain_value": rays_b / (p_ms / 1000.0), "speedup_vs_plain": p_ms / b_ms,
                   "steps": args.batched_steps, "ms_per_step": b_ms / args.batched_steps,
                   "plain_ms_per_step": p_ms / args.batched_steps,
                   "workload": "16 RGB-D-style maps, frame sizes " + ",".join(bres["sizes"]) +
                               " (1/2/4 cm, FP16 storage, colour) + raycast per map per step",
                   "tuned_config": bres["config"]}
        bf = bres["fuse"]
        if bf["steps"] and bf["ms"] > 0:
            b_ach = bf["bytes"] / (bf["ms"] / 1000.0) / 1e9
            batched["roofline"] = {"kernel": "k_batch_fuse (all maps' fusion + block variance + re-level, one launch)",
                                   "bound": "hbm", "achieved": round(b_ach, 1), "peak": hbm, "unit": "GB/s",
                                   "frac": round(b_ach / hbm, 4), "peak_kind": peak_kind,
                                   "traffic": stored_traffic("batch_fuse_traffic", BATCH_FUSE_SOURCES,
                                                             bf["bytes"] / bf["steps"]),
                                   "algorithmic_bytes_per_launch": int(bf["bytes"] / bf["steps"]),
                                   "launch_ms_avg": round(bf["ms"] / bf["steps"], 5)}

    learned = None
    if rank == 0 and not args.no_learned:  # a comparison on one GPU (its synthetic scans render on the host cores)
        learned = run_learned(wl, frames, args.warmup, timed, flush, res, epochs=args.learned_epochs,
                              lidar_train_scans=args.learned_lidar_train_scans,
                              lidar_scans=args.learned_lidar_scans, repeats=args.learned_repeats)
        if not args.no_feature_study:
            learned["feature_study"] = run_feature_study(wl)

    if rank == 0:
        final = res["final"]
        line = {"metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic (seeded procedural RGB-D room sequence; stands in for ScanNet/Replica)",
                "config": {"workload": RGBD_WORKLOAD,
                           "frames": f"{len(timed)} timed frames spread over the {n_frames}-frame orbit ({timed[0]}, "
                                     f"{timed[1] if len(timed) > 1 else ''}, ... {timed[-1]}); {args.warmup} warm-up "
                                     f"frames, every other frame integrated untimed in sequence order",
                           "l2": "flushed between steps (256 MiB write outside the timed events)",
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
                "frames_per_s": fps, "roofline": roofline, "roofline_raycast": roofline_ray,
                "roofline_lidar": roofline_lidar, "cpu_baseline": cpu,
                "e2e": e2e,
                "gpu_launches": int(launches), "clocks": clk, "kernels": kernels,
                "map": {"live_blocks": final["live_blocks"], "touched_last": final["touched"]},
                "lidar": lidar, "batched": batched, "learned": learned, "mesh": mesh, "quadtree": quad,
                "streaming": streaming, "splat": splat}
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
