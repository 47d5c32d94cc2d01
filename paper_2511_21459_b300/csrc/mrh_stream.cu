// Capacity-driven streaming (Sec. 3.3): blocks leave the device when a level's pool fills up, and come back when a
// frame allocates them again.
//
// Before a frame, when some level holds more than `stream_fraction` of its pool (float comparison of the counts),
// every block outside the frame's view moves to the archive with its level and payload: for a camera, a block whose
// circumscribed sphere misses the pinhole's view cone between min and max depth; for a LiDAR scan, a block whose centre
// lies farther than `stream_radius` from the scan origin. Its hash slot becomes a tombstone (skipped by every probe),
// its heap block returns to the free stack. A frame that allocates the key again gets it back at its archived level
// (binning queues the copy, k_restore performs it before fusion).
//
// The archive is pinned host memory mapped into the device's address space, indexed by a device-side hash: eviction
// and restore are kernels with no host round trip. Each key keeps the slot it got at its first eviction.
#include <cuda_runtime.h>

#include "mrh_internal.cuh"

namespace mrh {
namespace {

__device__ inline bool stream_due(const MapDev& m) {
  for (int l = 0; l < m.L; ++l) {
    const float live = (float)(m.max_blocks[l] - (uint32_t)max(m.st->free_top[l], 0));
    if (live > m.stream_fraction * (float)m.max_blocks[l]) return true;
  }
  return false;
}

// warp-collective copy of n bytes (a multiple of 16, both ends 16-byte aligned)
__device__ inline void warp_copy(uint8_t* dst, const uint8_t* src, uint32_t n, int lane) {
  const uint4* s = reinterpret_cast<const uint4*>(src);
  uint4* d = reinterpret_cast<uint4*>(dst);
  for (uint32_t i = lane; i < n / 16; i += 32) d[i] = s[i];
}

// archive entry for key (inserted when absent); its slot in *slot, or false when the archive is full
__device__ inline int archive_entry(const MapDev& m, unsigned long long key, uint32_t* slot) {
  uint32_t e = (uint32_t)hash_key(key, m.ar_mask);
  for (uint32_t p = 0; p <= m.ar_mask; ++p, e = (e + 1) & m.ar_mask) {
    const unsigned long long k = m.ar_keys[e];
    if (k == key) {
      *slot = m.ar_vals[e] & 0x0FFFFFFFu;
      return (int)e;
    }
    if (k == kEmptyKey) {
      const unsigned long long old = atomicCAS(&m.ar_keys[e], kEmptyKey, key);
      if (old == kEmptyKey) {
        const uint32_t sl = atomicAdd(&m.st->ar_used, 1u);
        if (sl >= m.ar_cap) {
          m.ar_vals[e] = 0x0FFFFFFFu;  // no storage: this key is never archived
          set_status(m.st, kStArchiveFull);
          return -1;
        }
        m.ar_vals[e] = sl;
        *slot = sl;
        return (int)e;
      }
      if (old == key) {
        *slot = m.ar_vals[e] & 0x0FFFFFFFu;
        return (int)e;
      }
    }
  }
  set_status(m.st, kStArchiveFull);
  return -1;
}

// The capacity check of this frame, taken once before any block is freed (the eviction pass changes the counts).
__global__ void k_stream_check(MapDev m) {
  if (threadIdx.x == 0 && blockIdx.x == 0) m.st->evict_go = stream_due(m) ? 1u : 0u;
}

// One warp per 32 hash slots: every resident block for which outside(centre) holds is archived and freed.
template <class Outside>
__device__ inline void evict_pass(const MapDev& m, const Outside& outside) {
  if (!m.st->evict_go) return;
  const int lane = threadIdx.x & 31;
  const uint32_t nslots = m.slot_mask + 1;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t base = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32u; base < nslots; base += nw * 32u) {
    const uint32_t sl = base + lane;
    const unsigned long long key = sl < nslots ? m.slots[sl].key : kEmptyKey;
    const uint32_t val = sl < nslots ? m.slots[sl].val : kValPending;
    bool go = key != kEmptyKey && key != kTombKey && val != kValPending && !(val & kValNew);
    if (go) {
      int x, y, z;
      unpack_key(key, &x, &y, &z);
      const float c[3] = {((float)x + 0.5f) * m.E, ((float)y + 0.5f) * m.E, ((float)z + 0.5f) * m.E};
      go = outside(c);
    }
    unsigned todo = __ballot_sync(~0u, go);
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1;
      const unsigned long long k = __shfl_sync(~0u, key, src);
      const uint32_t v = __shfl_sync(~0u, val, src);
      const uint32_t s = base + (uint32_t)src;
      uint32_t slot = 0;
      int e = 0;
      if (lane == 0) e = archive_entry(m, k, &slot);
      e = __shfl_sync(~0u, e, 0);
      slot = __shfl_sync(~0u, slot, 0);
      if (e < 0) continue;  // archive full: the block stays
      const int l = (int)((v >> 28) & 3u);
      const uint32_t id = v & kPtrMask;
      warp_copy(m.ar_data + (size_t)slot * m.ar_slot_bytes, m.heap[l] + (size_t)id * m.block_bytes[l],
                m.block_bytes[l], lane);
      __syncwarp();
      if (lane == 0) {
        m.ar_vals[e] = slot | ((uint32_t)l << 28) | kArPresent;
        m.slots[s].key = kTombKey;
        m.slots[s].val = kValPending;
        const int t = atomicAdd(&m.st->free_top[l], 1);
        m.free_stack[l][t] = id;
        atomicAdd(&m.st->evicted, 1u);
        atomicAdd(&m.st->ar_present, 1u);
      }
    }
  }
}

struct OutsideCamera {
  CamArgs c;
  float rad, tx, ty, kx, ky;
  __device__ bool operator()(const float p[3]) const {
    const float d0 = p[0] - c.t[0], d1 = p[1] - c.t[1], d2 = p[2] - c.t[2];
    const float xc = c.R[0] * d0 + c.R[3] * d1 + c.R[6] * d2;
    const float yc = c.R[1] * d0 + c.R[4] * d1 + c.R[7] * d2;
    const float zc = c.R[2] * d0 + c.R[5] * d1 + c.R[8] * d2;
    const bool inside = zc + rad >= c.min_depth && zc - rad <= c.max_depth && fabsf(xc) <= zc * tx + rad * kx &&
                        fabsf(yc) <= zc * ty + rad * ky;
    return !inside;
  }
};

struct OutsideRadius {
  float o[3];
  float r2;
  __device__ bool operator()(const float p[3]) const {
    const float d0 = p[0] - o[0], d1 = p[1] - o[1], d2 = p[2] - o[2];
    return d0 * d0 + d1 * d1 + d2 * d2 > r2;
  }
};

__global__ void __launch_bounds__(256) k_evict_camera(MapDev m, OutsideCamera f) { evict_pass(m, f); }
__global__ void __launch_bounds__(256) k_evict_lidar(MapDev m, OutsideRadius f) { evict_pass(m, f); }

// one warp per restore job: the archived payload back into the block's new heap block
__global__ void __launch_bounds__(256) k_restore(MapDev m) {
  const int lane = threadIdx.x & 31;
  const uint32_t n = m.st->n_restore;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < n; j += nw) {
    const uint2 job = m.restore_jobs[j];
    const int l = (int)((job.x >> 28) & 3u);
    warp_copy(m.heap[l] + (size_t)(job.x & kPtrMask) * m.block_bytes[l], m.ar_data + (size_t)job.y * m.ar_slot_bytes,
              m.block_bytes[l], lane);
  }
}

}  // namespace

void launch_evict_camera(const MapDev& m, const CamArgs& c, cudaStream_t s, int sms) {
  OutsideCamera f;
  f.c = c;
  f.rad = 0.8660254f * m.E;
  f.tx = fmaxf(c.cx, (float)c.width - c.cx) / c.fx;
  f.ty = fmaxf(c.cy, (float)c.height - c.cy) / c.fy;
  f.kx = sqrtf(1.0f + f.tx * f.tx);
  f.ky = sqrtf(1.0f + f.ty * f.ty);
  k_stream_check<<<1, 32, 0, s>>>(m);
  k_evict_camera<<<sms * 4, 256, 0, s>>>(m, f);
}

void launch_evict_lidar(const MapDev& m, const double* T, cudaStream_t s, int sms) {
  OutsideRadius f;
  f.o[0] = (float)T[3];
  f.o[1] = (float)T[7];
  f.o[2] = (float)T[11];
  f.r2 = m.stream_radius * m.stream_radius;
  k_stream_check<<<1, 32, 0, s>>>(m);
  k_evict_lidar<<<sms * 4, 256, 0, s>>>(m, f);
}

void launch_restore(const MapDev& m, cudaStream_t s, int sms) { k_restore<<<sms * 2, 256, 0, s>>>(m); }

}  // namespace mrh
