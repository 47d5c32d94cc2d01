// Ray -> block allocation (Sec. 3.2: blocks met by the rays are allocated with a DDA walk; Eq. 4 hashing).
//
// One thread per pixel (camera) or point (LiDAR) computes the ray's truncation band [max(rho - tau, 0), rho + tau],
// quantises its two end points to fixed point (1/65536 of a block edge) and walks the blocks the closed segment meets
// with an Amanatides-Woo walk whose crossings are compared exactly in integers, so the block set is exactly defined
// by the end points. Camera rays are set up in float in a fixed operation order (this file is compiled without
// multiply-add contraction), LiDAR rays in double.
//
// Deduplication is two-level: every CTA first inserts its rays' blocks into a shared-memory set (neighbouring rays
// share most blocks), then each warp takes the CTA's unique keys one at a time and probes the global table
// cooperatively: 32 consecutive slots per step, a ballot finds the key or the first empty slot, one lane claims it
// with a 64-bit atomicCAS. A slot joins this frame's touched list when its frame stamp is swapped by this frame.
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

// Warp-cooperative find-or-insert; every lane gets the slot index (or -1 when the probe limit is hit).
__device__ int warp_find_or_insert(const MapDev& m, unsigned long long key, int lane) {
  uint32_t h = hash_key(key, m.slot_mask);
  for (int w = 0; w < kMaxProbeWindows; ++w) {
    uint32_t s = (h + (uint32_t)(w * 32 + lane)) & m.slot_mask;
    unsigned long long k = *(volatile unsigned long long*)&m.slots[s].key;
    unsigned hit = __ballot_sync(~0u, k == key);
    if (hit) return __shfl_sync(~0u, (int)s, __ffs(hit) - 1);
    unsigned empty = __ballot_sync(~0u, k == kEmptyKey);
    while (empty) {
      int src = __ffs(empty) - 1;
      unsigned long long old = 0;
      if (lane == src) old = atomicCAS(&m.slots[s].key, kEmptyKey, key);
      old = __shfl_sync(~0u, old, src);
      if (old == kEmptyKey || old == key) return __shfl_sync(~0u, (int)s, src);
      empty &= empty - 1;
    }
  }
  if (lane == 0) set_status(m.st, kStHashFull);
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
  bool ok = walk_cells(A, B, kBlockUnit, kMaxSegmentCells, [&](const long long* c) {
    unsigned long long key = pack_key(c[0], c[1], c[2]);
    if (!set_insert(s_set, key)) {
      int s = thread_find_or_insert(m, key);
      if (s >= 0) touch(m, s, frame);
    }
  });
  if (!ok) set_status(m.st, kStSegment);
}

// After the CTA's rays are in the shared set: every warp inserts a share of the unique keys into the global table.
__device__ inline void flush_set(const MapDev& m, unsigned long long* s_set, uint32_t frame) {
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int base = warp * 32; base < kSetCap; base += nwarps * 32) {
    unsigned long long k = s_set[base + lane];
    unsigned pending = __ballot_sync(~0u, k != kEmptyKey);
    while (pending) {
      int src = __ffs(pending) - 1;
      pending &= pending - 1;
      unsigned long long key = __shfl_sync(~0u, k, src);
      int slot = warp_find_or_insert(m, key, lane);
      if (lane == 0 && slot >= 0) touch(m, slot, frame);
    }
  }
}

// Besides allocating, writes the frame's range image (rho = z |q|, -1 for invalid depth) and its colour packed as
// r | g << 8 | b << 16 (when rgb is given) for the fusion kernel.
__global__ void __launch_bounds__(256) k_alloc_depth(MapDev m, CamArgs c, const float* __restrict__ depth,
                                                     const uint8_t* __restrict__ rgb, float* __restrict__ rho_img,
                                                     uint32_t* __restrict__ rgb_img) {
  __shared__ unsigned long long s_set[kSetCap];
  __shared__ uint32_t s_valid;
  for (int i = threadIdx.x; i < kSetCap; i += blockDim.x) s_set[i] = kEmptyKey;
  if (threadIdx.x == 0) s_valid = 0;
  __syncthreads();
  const uint32_t frame = m.st->frame;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // CTA tile 32 x 8 pixels, each warp an 8 x 4 sub-tile (rays of a warp share blocks)
  const int u = blockIdx.x * 32 + (warp & 3) * 8 + (lane & 7);
  const int v = blockIdx.y * 8 + (warp >> 2) * 4 + (lane >> 3);
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
        atomicAdd(&s_valid, 1u);
        add_cells(m, s_set, A, B, frame);
      }
    }
  }
  __syncthreads();
  flush_set(m, s_set, frame);
  if (threadIdx.x == 0 && s_valid) atomicAdd(&m.st->valid_rays, s_valid);
}

__global__ void __launch_bounds__(256) k_alloc_points(MapDev m, PoseD P, const float* __restrict__ xyz, uint64_t n) {
  __shared__ unsigned long long s_set[kSetCap];
  __shared__ uint32_t s_valid;
  for (int i = threadIdx.x; i < kSetCap; i += blockDim.x) s_set[i] = kEmptyKey;
  if (threadIdx.x == 0) s_valid = 0;
  __syncthreads();
  const uint32_t frame = m.st->frame;
  const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) {
    long long A[3], B[3];
    double rho, rhat[3];
    if (lidar_ray(m, P, xyz, j, A, B, &rho, rhat)) {
      atomicAdd(&s_valid, 1u);
      add_cells(m, s_set, A, B, frame);
    }
  }
  __syncthreads();
  flush_set(m, s_set, frame);
  if (threadIdx.x == 0 && s_valid) atomicAdd(&m.st->valid_rays, s_valid);
}

// Bin this frame's touched slots by level and give new blocks a heap block of the finest level (Sec. 3.2.1:
// "we initialize the voxel blocks to the finest resolution"). A block whose heap is empty keeps no storage, is not
// fused, and is retried in later frames.
__global__ void __launch_bounds__(256) k_bin(MapDev m) {
  uint32_t n = min(m.st->touched_all, m.max_touched);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    uint32_t s = m.touched_all[i];
    uint32_t val = m.slots[s].val;
    if (val == kValPending) {
      // a new block: record its brick for the raycaster's empty-space skipping (idempotent)
      {
        int bx, by, bz;
        unpack_key(m.slots[s].key, &bx, &by, &bz);
        bx >>= kBrickShift;
        by >>= kBrickShift;
        bz >>= kBrickShift;
        const unsigned long long bkey = pack_key(bx, by, bz);
        const uint32_t h = hash_xyz(bx, by, bz, m.brick_mask);
        for (uint32_t p = 0; p <= m.brick_mask && p < (uint32_t)kMaxProbes; ++p) {
          unsigned long long* slot = &m.brick_keys[(h + p) & m.brick_mask];
          const unsigned long long cur = *(volatile unsigned long long*)slot;
          if (cur == bkey) break;
          if (cur != kEmptyKey) continue;
          const unsigned long long old = atomicCAS(slot, kEmptyKey, bkey);
          if (old == kEmptyKey || old == bkey) break;
        }
      }
      const int l = 0;
      int t = atomicSub(&m.st->free_top[l], 1);
      if (t <= 0) {
        atomicAdd(&m.st->free_top[l], 1);
        set_status(m.st, kStPoolEmpty);
        continue;
      }
      uint32_t id = m.free_stack[l][t - 1];
      val = id | ((uint32_t)l << 28) | kValNew;
      m.slots[s].val = val;
      atomicAdd(&m.st->new_blocks, 1u);
    }
    uint32_t l = (val >> 28) & 3u;
    uint32_t j = atomicAdd(&m.st->touched_count[l], 1u);
    m.touched[l][j] = s;
    m.slot_pos[s] = (l << 28) | j;
    BlockMeta bm;
    bm.key = m.slots[s].key;
    bm.val = val;
    bm.slot = s;
    m.meta[l][j] = bm;
  }
}

}  // namespace

void launch_alloc_depth(const MapDev& m, const CamArgs& c, const float* depth, const uint8_t* rgb, float* rho_img,
                        uint32_t* rgb_img, cudaStream_t s) {
  dim3 grid((c.width + 31) / 32, (c.height + 7) / 8);
  k_alloc_depth<<<grid, 256, 0, s>>>(m, c, depth, rgb, rho_img, rgb ? rgb_img : nullptr);
}

void launch_alloc_points(const MapDev& m, const double* T, const float* xyz, uint64_t n, cudaStream_t s) {
  if (n == 0) return;
  PoseD P;
  for (int i = 0; i < 16; ++i) P.T[i] = T[i];
  unsigned blocks = (unsigned)((n + 255) / 256);
  k_alloc_points<<<blocks, 256, 0, s>>>(m, P, xyz, n);
}

void launch_bin(const MapDev& m, cudaStream_t s, int sms) { k_bin<<<sms * 2, 256, 0, s>>>(m); }

}  // namespace mrh
