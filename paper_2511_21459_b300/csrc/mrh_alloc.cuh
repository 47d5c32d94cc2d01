// Ray -> block allocation (Sec. 3.2: blocks met by the rays are allocated with a DDA walk; Eq. 4 hashing): device
// code shared by the single-map kernels (mrh_alloc.cu) and the batched kernels (mrh_batch.cu).
//
// One thread per pixel (camera) or point (LiDAR) computes the ray's truncation band [max(rho - tau, 0), rho + tau],
// quantises its two end points to fixed point (1/65536 of a block edge) and walks the blocks the closed segment meets
// with an Amanatides-Woo walk whose crossings are compared exactly in integers, so the block set is exactly defined
// by the end points. Camera rays are set up in float in a fixed operation order (compiled without multiply-add
// contraction), LiDAR rays in double.
//
// Deduplication is two-level: every CTA first inserts its rays' blocks into a shared-memory set (neighbouring rays
// share most blocks), then groups of PW lanes take the CTA's unique keys and probe the global table cooperatively:
// PW consecutive slots per step, a ballot finds the key or the first empty slot, one lane claims it with a 64-bit
// atomicCAS. A slot joins this frame's touched list when its frame stamp is swapped by this frame. The CTA pixel tile
// (TW x TH) and the probe width PW are tuning parameters; every choice computes the same result.
#pragma once
#include "mrh_internal.cuh"

namespace mrh {
namespace {

constexpr int kSetCap = 2048;  // per-CTA shared-memory key set

__device__ inline uint32_t set_hash(unsigned long long k) {
  return (uint32_t)((k * 0x9E3779B97F4A7C15ULL) >> 40) & (kSetCap - 1);
}

// true if the key is now in the set
__device__ inline bool set_insert(unsigned long long* set, unsigned long long key) {
  uint32_t h = set_hash(key);
  for (int p = 0; p < kSetCap; ++p) {
    uint32_t s = (h + p) & (kSetCap - 1);
    unsigned long long cur = ((volatile unsigned long long*)set)[s];
    if (cur == key) return true;
    if (cur != kEmptyKey) continue;
    unsigned long long old = atomicCAS(&set[s], kEmptyKey, key);
    if (old == kEmptyKey || old == key) return true;
  }
  return false;
}

// Cooperative find-or-insert by a group of PW lanes (gmask: the group's lanes, gbase: its first lane, gl: lane within
// the group). Every lane of the group gets the slot index, or -1 when the probe limit is hit.
template <int PW>
__device__ int group_find_or_insert(const MapDev& m, unsigned long long key, unsigned gmask, int gbase, int gl) {
  const uint32_t h = hash_key(key, m.slot_mask);
  const int windows = kMaxProbeWindows * (32 / PW);
  for (int w = 0; w < windows; ++w) {
    const uint32_t s = (h + (uint32_t)(w * PW + gl)) & m.slot_mask;
    const unsigned long long k = *(volatile unsigned long long*)&m.slots[s].key;
    const unsigned hit = (__ballot_sync(gmask, k == key) >> gbase) & (PW == 32 ? ~0u : ((1u << PW) - 1u));
    if (hit) return __shfl_sync(gmask, (int)s, gbase + __ffs(hit) - 1);
    unsigned empty = (__ballot_sync(gmask, k == kEmptyKey) >> gbase) & (PW == 32 ? ~0u : ((1u << PW) - 1u));
    while (empty) {
      const int src = __ffs(empty) - 1;
      unsigned long long old = 0;
      if (gl == src) old = atomicCAS(&m.slots[s].key, kEmptyKey, key);
      old = __shfl_sync(gmask, old, gbase + src);
      if (old == kEmptyKey || old == key) return __shfl_sync(gmask, (int)s, gbase + src);
      empty &= empty - 1;
    }
  }
  if (gl == 0) set_status(m.st, kStHashFull);
  return -1;
}

// Single-thread find-or-insert (fallback when a CTA's shared set overflows).
__device__ int thread_find_or_insert(const MapDev& m, unsigned long long key) {
  uint32_t h = hash_key(key, m.slot_mask);
  for (int p = 0; p < kMaxProbes; ++p) {
    uint32_t s = (h + (uint32_t)p) & m.slot_mask;
    unsigned long long k = *(volatile unsigned long long*)&m.slots[s].key;
    if (k == key) return (int)s;
    if (k != kEmptyKey) continue;
    unsigned long long old = atomicCAS(&m.slots[s].key, kEmptyKey, key);
    if (old == kEmptyKey || old == key) return (int)s;
  }
  set_status(m.st, kStHashFull);
  return -1;
}

__device__ inline void touch(const MapDev& m, int slot, uint32_t frame) {
  uint32_t old = atomicExch(&m.slots[slot].stamp, frame);
  if (old != frame) {
    uint32_t i = atomicAdd(&m.st->touched_all, 1u);
    if (i < m.max_touched) m.touched_all[i] = (uint32_t)slot;
    else set_status(m.st, kStListFull);
  }
}

__device__ inline void add_cells(const MapDev& m, unsigned long long* s_set, const long long A[3],
                                 const long long B[3], uint32_t frame) {
  bool ok = walk_cells(A, B, kBlockShift, kMaxSegmentCells, [&](const int* c) {
    unsigned long long key = pack_key(c[0], c[1], c[2]);
    if (!set_insert(s_set, key)) {
      int s = thread_find_or_insert(m, key);
      if (s >= 0) touch(m, s, frame);
    }
  });
  if (!ok) set_status(m.st, kStSegment);
}

// After the CTA's rays are in the shared set: groups of PW lanes insert the unique keys into the global table.
template <int PW>
__device__ inline void flush_set(const MapDev& m, unsigned long long* s_set, uint32_t frame) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int group = lane / PW, gbase = group * PW, gl = lane % PW;
  const unsigned gmask = (PW == 32 ? ~0u : ((1u << PW) - 1u)) << gbase;
  constexpr int kGroups = 32 / PW;
  for (int base = warp * 32; base < kSetCap; base += nwarps * 32) {
    const unsigned long long k = s_set[base + lane];
    unsigned pending = __ballot_sync(~0u, k != kEmptyKey);
    while (pending) {
      // the group takes the group-th pending key of this chunk (if there are that many)
      unsigned rest = pending;
      for (int g = 0; g < group && rest; ++g) rest &= rest - 1;
      const int src = rest ? __ffs(rest) - 1 : 0;
      const unsigned long long key = __shfl_sync(~0u, k, src);
      if (rest) {
        const int slot = group_find_or_insert<PW>(m, key, gmask, gbase, gl);
        if (gl == 0 && slot >= 0) touch(m, slot, frame);
      }
      __syncwarp();
      for (int g = 0; g < kGroups && pending; ++g) pending &= pending - 1;
    }
  }
}

// Pixel (u, v) of a CTA tile TW x TH (256 threads): each warp covers an 8 x 4 sub-tile.
template <int TW, int TH>
__device__ inline void tile_pixel(int tile_x, int tile_y, int* u, int* v) {
  static_assert(TW * TH == 256 && TW % 8 == 0 && TH % 4 == 0, "tile");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int wx = TW / 8;
  *u = tile_x * TW + (warp % wx) * 8 + (lane & 7);
  *v = tile_y * TH + (warp / wx) * 4 + (lane >> 3);
}

// One CTA of camera allocation. Besides allocating, writes the frame's range image (rho = z |q|, -1 for invalid
// depth) and its colour packed as r | g << 8 | b << 16 (when rgb is given) for the fusion kernel.
template <int TW, int TH, int PW>
__device__ inline void alloc_depth_tile(const MapDev& m, const CamArgs& c, const float* __restrict__ depth,
                                        const uint8_t* __restrict__ rgb, float* __restrict__ rho_img,
                                        uint32_t* __restrict__ rgb_img, int tile_x, int tile_y,
                                        unsigned long long* s_set, uint32_t* s_valid) {
  for (int i = threadIdx.x; i < kSetCap; i += blockDim.x) s_set[i] = kEmptyKey;
  if (threadIdx.x == 0) *s_valid = 0;
  __syncthreads();
  const uint32_t frame = m.st->frame;
  int u, v;
  tile_pixel<TW, TH>(tile_x, tile_y, &u, &v);
  if (u < c.width && v < c.height) {
    const size_t pix = (size_t)v * c.width + u;
    float z = depth[pix];
    if (rgb_img)
      rgb_img[pix] = (uint32_t)rgb[3 * pix] | ((uint32_t)rgb[3 * pix + 1] << 8) | ((uint32_t)rgb[3 * pix + 2] << 16);
    if (!(z >= c.min_depth && z <= c.max_depth)) rho_img[pix] = -1.0f;
    if (z >= c.min_depth && z <= c.max_depth) {
      float qx = ((float)u - c.cx) / c.fx;
      float qy = ((float)v - c.cy) / c.fy;
      float nq = sqrtf(qx * qx + qy * qy + 1.0f);
      float rho = z * nq;
      rho_img[pix] = rho;
      float rc0 = qx / nq, rc1 = qy / nq, rc2 = 1.0f / nq;
      float r[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) r[a] = c.R[3 * a + 0] * rc0 + c.R[3 * a + 1] * rc1 + c.R[3 * a + 2] * rc2;
      float t0 = rho - m.tau;
      if (t0 < 0.0f) t0 = 0.0f;
      float t1 = rho + m.tau;
      long long A[3], B[3];
      bool ok = true;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        ok = ok && to_fixed_f(c.t[a] + t0 * r[a], m.fix_scale, &A[a]);
        ok = ok && to_fixed_f(c.t[a] + t1 * r[a], m.fix_scale, &B[a]);
      }
      if (ok && key_ok(floor_div(A[0], kBlockUnit), floor_div(A[1], kBlockUnit), floor_div(A[2], kBlockUnit)) &&
          key_ok(floor_div(B[0], kBlockUnit), floor_div(B[1], kBlockUnit), floor_div(B[2], kBlockUnit))) {
        atomicAdd(s_valid, 1u);
        add_cells(m, s_set, A, B, frame);
      }
    }
  }
  __syncthreads();
  flush_set<PW>(m, s_set, frame);
  if (threadIdx.x == 0 && *s_valid) atomicAdd(&m.st->valid_rays, *s_valid);
}

// One CTA of LiDAR allocation: points [first, first + blockDim.x).
template <int PW>
__device__ inline void alloc_points_cta(const MapDev& m, const PoseD& P, const float* __restrict__ xyz, uint64_t n,
                                        uint64_t first, unsigned long long* s_set, uint32_t* s_valid) {
  for (int i = threadIdx.x; i < kSetCap; i += blockDim.x) s_set[i] = kEmptyKey;
  if (threadIdx.x == 0) *s_valid = 0;
  __syncthreads();
  const uint32_t frame = m.st->frame;
  const uint64_t j = first + threadIdx.x;
  if (j < n) {
    LidarRay ray;
    double rho, rhat[3], p[3];
    const bool ok = lidar_ray(m, P, xyz, j, ray.A, ray.B, &rho, rhat, m.lidar_end ? p : nullptr);
    ray.rho = ok ? (float)rho : -1.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) ray.rh[a] = (float)rhat[a];
    m.rays[j] = ray;  // reused by the observation passes
    if (m.lidar_end) {  // the end point in fixed point, for the learned predictor's moments
      long long e[3];
      const bool eok = ok && to_fixed_d(p[0], m.fix_scale64, &e[0]) && to_fixed_d(p[1], m.fix_scale64, &e[1]) &&
                       to_fixed_d(p[2], m.fix_scale64, &e[2]);
#pragma unroll
      for (int a = 0; a < 3; ++a) m.lidar_end[3 * j + a] = eok ? e[a] : kNoEndPoint;
    }
    if (ok) {
      atomicAdd(s_valid, 1u);
      add_cells(m, s_set, ray.A, ray.B, frame);
    }
  }
  __syncthreads();
  flush_set<PW>(m, s_set, frame);
  if (threadIdx.x == 0 && *s_valid) atomicAdd(&m.st->valid_rays, *s_valid);
}

// Archive entry of a key (streaming), or -1.
__device__ inline int archive_find(const MapDev& m, unsigned long long key) {
  uint32_t e = (uint32_t)hash_key(key, m.ar_mask);
  for (uint32_t p = 0; p <= m.ar_mask; ++p, e = (e + 1) & m.ar_mask) {
    const unsigned long long k = m.ar_keys[e];
    if (k == key) return (int)e;
    if (k == kEmptyKey) return -1;
  }
  return -1;
}

// Touched entry i of this frame, first half: a new block gets a heap block of the finest level (Sec. 3.2.1: "we
// initialize the voxel blocks to the finest resolution"), or of new_level when the learned predictor gave one, and
// its brick is recorded for the raycaster; a block streamed out earlier comes back at its archived level and queues
// the copy of its payload (Sec. 3.3). Returns the block's level and heap value, or -1 when the block has no storage
// (its level's heap is empty: it is not fused and is retried in later frames).
__device__ inline int bin_entry(const MapDev& m, uint32_t s, int new_level, uint32_t* val_out) {
  uint32_t val = m.slots[s].val;
  if (val == kValPending) {
    int l = new_level;
    int ar = -1;
    uint32_t ar_val = 0;
    if (m.ar_keys) {
      ar = archive_find(m, m.slots[s].key);
      if (ar >= 0) {
        ar_val = m.ar_vals[ar];
        if (ar_val & kArPresent) l = (int)((ar_val >> 28) & 3u);
        else ar = -1;
      }
    }
    {
      int bx, by, bz;
      unpack_key(m.slots[s].key, &bx, &by, &bz);
      const int rx = bx >> kBrickShift, ry = by >> kBrickShift, rz = bz >> kBrickShift;
      bool ok = occupancy_insert(m.brick_keys, m.brick_bits, m.brick_mask, rx, ry, rz, cell_bit(bx, by, bz));
      ok = ok && occupancy_insert(m.super_keys, m.super_bits, m.super_mask, rx >> kSuperShift, ry >> kSuperShift,
                                  rz >> kSuperShift, cell_bit(rx, ry, rz));
      if (!ok) set_status(m.st, kStHashFull);
    }
    int t = atomicSub(&m.st->free_top[l], 1);
    if (t <= 0) {
      atomicAdd(&m.st->free_top[l], 1);
      set_status(m.st, kStPoolEmpty);
      return -1;
    }
    uint32_t id = m.free_stack[l][t - 1];
    val = id | ((uint32_t)l << 28) | (ar >= 0 ? 0u : kValNew);
    m.slots[s].val = val;
    atomicAdd(&m.st->new_blocks, 1u);
    if (ar >= 0) {
      const uint32_t j = atomicAdd(&m.st->n_restore, 1u);
      m.restore_jobs[j] = make_uint2(val, ar_val & 0x0FFFFFFFu);
      m.ar_vals[ar] = ar_val & ~kArPresent;
      atomicAdd(&m.st->restored, 1u);
      atomicSub(&m.st->ar_present, 1u);
    }
  }
  *val_out = val;
  return (int)((val >> 28) & 3u);
}

// Warp-collective: append each lane's binned entry (level l >= 0; -1 = nothing) to its level's list (Sec. 3.2: the
// per-level work lists of the fusion pass) with one atomic per level per warp. All 32 lanes must call it.
__device__ inline void append_binned(const MapDev& m, int l, uint32_t s, uint32_t val) {
  const int lane = threadIdx.x & 31;
  for (int L = 0; L < m.L; ++L) {
    const unsigned mask = __ballot_sync(0xffffffffu, l == L);
    if (!mask) continue;
    const int leader = __ffs(mask) - 1;
    uint32_t j = 0;
    if (lane == leader) j = atomicAdd(&m.st->touched_count[L], (uint32_t)__popc(mask));
    j = __shfl_sync(0xffffffffu, j, leader) + (uint32_t)__popc(mask & ((1u << lane) - 1u));
    if (l == L) {
      m.touched[L][j] = s;
      m.slot_pos[s] = ((uint32_t)L << 28) | j;
      BlockMeta bm;
      bm.key = m.slots[s].key;
      bm.val = val;
      bm.slot = s;
      m.meta[L][j] = bm;
    }
  }
}

// Bins the touched entries first_warp_thread + lane, + stride, ... (a warp-uniform loop: first_warp_thread and
// stride are multiples of 32).
__device__ inline void bin_entries(const MapDev& m, uint32_t first_warp_thread, uint32_t stride) {
  const uint32_t n = min(m.st->touched_all, m.max_touched);
  const int lane = threadIdx.x & 31;
  for (uint32_t base = first_warp_thread; base < n; base += stride) {
    const uint32_t i = base + lane;
    int l = -1;
    uint32_t s = 0, val = 0;
    if (i < n) {
      s = m.touched_all[i];
      l = bin_entry(m, s, 0, &val);
    }
    append_binned(m, l, s, val);
  }
}

// Heap blocks freed by re-levelling go back to their free stacks.
__device__ inline void release_one(const MapDev& m, uint32_t i) {
  const uint32_t r = m.retire[i];
  const uint32_t l = r >> 28, id = r & kPtrMask;
  const int t = atomicAdd(&m.st->free_top[l], 1);
  m.free_stack[l][t] = id;
}

// Frame number + 1, per-frame counters to zero.
__device__ inline void begin_frame(DevState* st) {
  st->frame += 1;
  st->touched_all = 0;
  for (int l = 0; l < 4; ++l) st->touched_count[l] = 0;
  st->retire_count = 0;
  st->new_blocks = st->merged = st->split = st->rechecks = st->valid_rays = 0;
  st->observations = 0;
  st->updated_voxels = 0;
  st->n_over = 0;
  st->max_vox_obs = 0;
  st->n_fresh = 0;
  st->item_next = 0;
  st->evicted = st->restored = st->n_restore = 0;
}

}  // namespace
}  // namespace mrh
