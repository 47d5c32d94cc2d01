// Kernels and launchers of fusion for one map, and the LiDAR observation passes (device code in mrh_fuse.cuh).
#include <cstddef>

#include "mrh_fuse.cuh"

namespace mrh {
namespace {

// lookup_slot reading each probed slot with one 16-byte load, so that the heap value of a hit comes with its key.
// Returns the slot index or -1; *val = the slot's heap value on a hit.
__device__ inline int probe_slot(const Slot* __restrict__ slots, uint32_t mask, unsigned long long key, uint32_t* val) {
  static_assert(sizeof(Slot) == 16 && offsetof(Slot, val) == 8, "a slot is read as one ulonglong2");
  const uint32_t h = hash_key(key, mask);
  const ulonglong2* sl = reinterpret_cast<const ulonglong2*>(slots);
  for (int p = 0; p < kMaxProbes; ++p) {
    const uint32_t s = (h + (uint32_t)p) & mask;
    const ulonglong2 e = sl[s];
    if (e.x == key) {
      *val = (uint32_t)e.y;
      return (int)s;
    }
    if (e.x == kEmptyKey) return -1;
  }
  return -1;
}

constexpr int kCamWarps = 8;

template <bool FP16, bool COLOR>
__global__ void __launch_bounds__(32 * kCamWarps, 4) k_fuse_depth(MapDev m, CamArgs c, const float* __restrict__ rho,
                                                                 const uint32_t* __restrict__ rgb) {
  CameraObs<FP16, COLOR> obs{c, rho, rgb};
  const int warp = threadIdx.x >> 5;
  fuse_warp_body<FP16, COLOR>(m, obs, warp, blockIdx.x * kCamWarps + warp, gridDim.x * kCamWarps);
}

// Items are handed out one per warp from a counter (zeroed when the frame begins), the level-1 and level-2 items
// first: they hold the most observations per voxel and are the longest, so they must not start last.
template <bool FP16, bool COLOR>
__global__ void __launch_bounds__(32 * kLidarWarps) k_fuse_points(MapDev m) {
  __shared__ LidarSmem s_lidar;
  LidarObs<FP16> obs{&s_lidar, nullptr};
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const ItemCounts ic = item_counts(m);
  const uint32_t items = ic.items(), coarse = items - ic.it0;
  unsigned long long my_obs = 0, my_vox = 0;
  for (;;) {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(&m.st->item_next, 1u);
    t = __shfl_sync(~0u, t, 0);
    if (t >= items) break;
    fuse_item<FP16, COLOR>(m, obs, warp, ic, t < coarse ? ic.it0 + t : t - coarse, my_obs, my_vox);
  }
  uint32_t vmax = obs.vmax;
  for (int o = 16; o > 0; o >>= 1) {
    my_obs += __shfl_xor_sync(~0u, my_obs, o);
    my_vox += __shfl_xor_sync(~0u, my_vox, o);
    vmax = max(vmax, __shfl_xor_sync(~0u, vmax, o));
  }
  if (lane == 0 && my_obs) atomicAdd(&m.st->observations, my_obs);
  if (lane == 0 && my_vox) atomicAdd(&m.st->updated_voxels, my_vox);
  if (lane == 0 && vmax) atomicMax(&m.st->max_vox_obs, vmax);
}

// -------------------------------------------------------------------------------------------- LiDAR observation passes

// One point: the walk over the finest cells of its ray's band (Sec. 3.1, Eq. 1), one observation (point index << 9 |
// voxel, d) per voxel of the crossed block's own level.
//   STAGE: count each block's observations and stage the point's runs (a header {kStageHeader | block, length}
//          followed by the run's records) in its kStageCap entries; a point whose runs do not fit is listed in
//          stage_over and only counted.
//   FILL:  for the listed points: write the records straight into the blocks' segments.
template <bool FILL>
__device__ inline void lidar_point(const MapDev& m, const PoseD& P, uint64_t j) {
  const LidarRay& ray = m.rays[j];  // computed by the allocation pass
  const float rho_f = ray.rho;
  if (!(rho_f >= 0.0f)) {
    if constexpr (!FILL) m.stage_len[j] = 0;
    return;
  }
  long long A[3], B[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    A[a] = ray.A[a];
    B[a] = ray.B[a];
  }
  const uint32_t n0 = min(m.st->touched_count[0], m.max_touched);
  const uint32_t n1 = min(m.st->touched_count[1], m.max_touched);
  const float rh[3] = {ray.rh[0], ray.rh[1], ray.rh[2]};
  const float o_f[3] = {(float)P.T[3], (float)P.T[7], (float)P.T[11]};

  int cb[3] = {0, 0, 0}, lg[3] = {0, 0, 0};
  bool have_block = false, cur_ok = false, have_last = false;
  int cl = 0;
  uint32_t cur_P = 0, run = 0;
  float ob[3] = {0.f, 0.f, 0.f};
  // STAGE: the point's entries; FILL: the current run's reserved range
  uint2* const stage = m.stage + (size_t)j * kStageCap;
  uint32_t pos = 0, hpos = 0;
  bool fits = true;

  auto close_run = [&]() {
    if (!cur_ok || run == 0) return;
    if constexpr (!FILL) {
      atomicAdd(&m.blk_count[cur_P], run);
      if (fits) stage[hpos] = make_uint2(kStageHeader | cur_P, run);
    }
    run = 0;
  };

  bool ok = walk_cells(A, B, kVoxelShift, kMaxVoxelCells, [&](const int* f) {
    const int bk[3] = {f[0] >> 3, f[1] >> 3, f[2] >> 3};  // finest cell -> block (floor division by 8)
    if (!have_block || bk[0] != cb[0] || bk[1] != cb[1] || bk[2] != cb[2]) {
      close_run();
      have_block = true;
      cb[0] = bk[0]; cb[1] = bk[1]; cb[2] = bk[2];
      have_last = false;
      cur_ok = false;
      uint32_t val = kValPending;
      const int s = probe_slot(m.slots, m.slot_mask, pack_key(bk[0], bk[1], bk[2]), &val);
      if (s >= 0) {
        if (val != kValPending) {
          uint32_t sp = m.slot_pos[s];
          uint32_t lv = sp >> 28, jj = sp & kPtrMask;
          // the position is this frame's only if the level list points back at the slot
          const uint32_t cnt_lv = min(m.st->touched_count[lv], m.max_touched);
          if (lv == ((val >> 28) & 3u) && (int)lv < m.L && jj < cnt_lv && m.touched[lv][jj] == (uint32_t)s) {
            cl = (int)lv;
            cur_P = jj + (lv >= 1 ? n0 : 0) + (lv >= 2 ? n1 : 0);
            cur_ok = true;
            ob[0] = (float)bk[0] * m.E - o_f[0];
            ob[1] = (float)bk[1] * m.E - o_f[1];
            ob[2] = (float)bk[2] * m.E - o_f[2];
            if constexpr (!FILL) {
              hpos = pos;  // the run's header slot, written when the run closes
              if (fits && pos + 1 > (uint32_t)kStageCap) fits = false;
              pos += 1;
            }
          }
        }
      }
    }
    if (!cur_ok) return;
    const int g[3] = {f[0] >> cl, f[1] >> cl, f[2] >> cl};  // voxel of the block's level containing the cell
    if (have_last && g[0] == lg[0] && g[1] == lg[1] && g[2] == lg[2]) return;
    have_last = true;
    lg[0] = g[0]; lg[1] = g[1]; lg[2] = g[2];
    const int nl = kFineDim >> cl;
    const int li[3] = {g[0] - cb[0] * nl, g[1] - cb[1] * nl, g[2] - cb[2] * nl};
    const float vl = m.v[cl];
    const float xr0 = ob[0] + ((float)li[0] + 0.5f) * vl;
    const float xr1 = ob[1] + ((float)li[1] + 0.5f) * vl;
    const float xr2 = ob[2] + ((float)li[2] + 0.5f) * vl;
    float d = rho_f - (xr0 * rh[0] + xr1 * rh[1] + xr2 * rh[2]);
    if (d < -m.tau) d = -m.tau;
    if (d > m.tau) d = m.tau;
    const uint32_t key = ((uint32_t)j << 9) | (uint32_t)(li[0] + nl * (li[1] + nl * li[2]));
    const uint2 rec = make_uint2(key, __float_as_uint(d));
    if constexpr (FILL) {
      // one record at a time into the block's segment (the overflow path is rare)
      const uint32_t at = m.blk_off[cur_P] + atomicAdd(&m.blk_fill[cur_P], 1u);
      if (at < m.max_obs) m.obs_rec[at] = rec;
      else set_status(m.st, kStObsFull);
    } else {
      if (fits && pos + 1 > (uint32_t)kStageCap) fits = false;
      if (fits) stage[pos] = rec;
      pos += 1;
    }
    ++run;
  });
  close_run();
  if constexpr (!FILL) {
    if (fits) {
      m.stage_len[j] = pos;
    } else {
      m.stage_len[j] = kStageOverflow;
      const uint32_t t = atomicAdd(&m.st->n_over, 1u);
      m.stage_over[t] = (uint32_t)j;
    }
  }
  if (!ok && !FILL) set_status(m.st, kStSegment);
}

__global__ void __launch_bounds__(128) k_lidar_stage(MapDev m, PoseD P, uint64_t n) {
  const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) lidar_point<false>(m, P, j);
}

__global__ void __launch_bounds__(128) k_lidar_fill_over(MapDev m, PoseD P) {
  const uint32_t n_over = m.st->n_over;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n_over; t += gridDim.x * blockDim.x)
    lidar_point<true>(m, P, m.stage_over[t]);
}

// One warp per point: copy the point's staged runs into the blocks' segments. Lane i takes entry i of each group of
// 32; a header lane reserves its run's range with one atomic, and the record lanes after it (or, before the first
// header of the group, the run carried over from the previous group) write at consecutive positions.
__global__ void __launch_bounds__(256) k_lidar_scatter(MapDev m, uint64_t n) {
  const int lane = threadIdx.x & 31;
  const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t j = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < n; j += n_warps) {  // warp-uniform
    const uint32_t len = m.stage_len[j];
    if (len == 0 || len == kStageOverflow) continue;
    const uint2* e = m.stage + (size_t)j * kStageCap;
    uint32_t run_base = 0, run_pos = 0;
    bool run_ok = false;
    for (uint32_t c0 = 0; c0 < len; c0 += 32) {
      const uint32_t i = c0 + (uint32_t)lane;
      const uint2 v = i < len ? e[i] : make_uint2(0u, 0u);
      const bool hdr = i < len && (v.x & kStageHeader) != 0;
      uint32_t base = 0;
      bool ok = false;
      if (hdr) {
        const uint32_t P = v.x & ~kStageHeader, rl = v.y;
        base = m.blk_off[P] + atomicAdd(&m.blk_fill[P], rl);
        ok = base + rl <= m.max_obs;
        if (!ok) set_status(m.st, kStObsFull);
      }
      const unsigned hmask = __ballot_sync(~0u, hdr);
      const unsigned okmask = __ballot_sync(~0u, ok);
      const unsigned upto = hmask & (lane == 31 ? 0xFFFFFFFFu : ((2u << lane) - 1u));
      const int h = upto ? 31 - __clz(upto) : -1;
      const uint32_t hb = __shfl_sync(~0u, base, h < 0 ? 0 : h);
      if (i < len && !hdr) {
        const bool good = h >= 0 ? ((okmask >> h) & 1u) != 0 : run_ok;
        const uint32_t dst = h >= 0 ? hb + (uint32_t)(lane - h - 1) : run_base + run_pos + (uint32_t)lane;
        if (good) m.obs_rec[dst] = v;
      }
      const int last_h = hmask ? 31 - __clz(hmask) : -1;
      if (last_h >= 0) {
        run_base = __shfl_sync(~0u, base, last_h);
        run_ok = ((okmask >> last_h) & 1u) != 0;
        run_pos = (uint32_t)(31 - last_h);
      } else {
        run_pos += 32;
      }
    }
  }
}

__global__ void k_zero_obs_counts(MapDev m) {
  const uint32_t total = min(m.st->touched_count[0], m.max_touched) + min(m.st->touched_count[1], m.max_touched) +
                         min(m.st->touched_count[2], m.max_touched);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    m.blk_count[i] = 0;
    m.blk_fill[i] = 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    m.st->obs_total = 0;
    m.st->n_over = 0;
  }
}

// One thread per fusion work item (the grouping of k_fuse_points: one level-0 block, two level-1 blocks or sixteen
// level-2 blocks): the item's blocks get consecutive ranges of one segment of the observation buffer, the segment
// taken from a running total with one atomic per warp. Segments of different items may lie in any order.
__global__ void __launch_bounds__(256) k_obs_segments(MapDev m) {
  const ItemCounts ic = item_counts(m);
  const uint32_t items = ic.items();
  const int lane = threadIdx.x & 31;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < items; base += stride) {
    const uint32_t item = base + lane;
    uint32_t first = 0, nb = 0;
    if (item < ic.it0) {
      first = item;
      nb = 1;
    } else if (item < ic.it0 + ic.it1) {
      const uint32_t idx = (item - ic.it0) * 2;
      first = ic.n0 + idx;
      nb = min(2u, ic.n1 - idx);
    } else if (item < items) {
      const uint32_t idx = (item - ic.it0 - ic.it1) * 16;
      first = ic.n0 + ic.n1 + idx;
      nb = min(16u, ic.n2 - idx);
    }
    uint32_t sum = 0;
    for (uint32_t g = 0; g < nb; ++g) sum += m.blk_count[first + g];
    uint32_t incl = sum;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(~0u, incl, o);
      if (lane >= o) incl += t;
    }
    uint32_t seg = 0;
    if (lane == 31) seg = atomicAdd(&m.st->obs_total, incl);
    uint32_t start = __shfl_sync(~0u, seg, 31) + incl - sum;
    for (uint32_t g = 0; g < nb; ++g) {
      m.blk_off[first + g] = start;
      start += m.blk_count[first + g];
    }
  }
}

}  // namespace

void launch_fuse_depth(const MapDev& m, const CamArgs& c, const float* rho, const uint32_t* rgb, cudaStream_t s,
                       int sms) {
  const int grid = sms * 8;
  if (m.fp16) {
    if (m.color) k_fuse_depth<true, true><<<grid, 32 * kCamWarps, 0, s>>>(m, c, rho, rgb);
    else k_fuse_depth<true, false><<<grid, 32 * kCamWarps, 0, s>>>(m, c, rho, rgb);
  } else {
    if (m.color) k_fuse_depth<false, true><<<grid, 32 * kCamWarps, 0, s>>>(m, c, rho, rgb);
    else k_fuse_depth<false, false><<<grid, 32 * kCamWarps, 0, s>>>(m, c, rho, rgb);
  }
}

void launch_lidar_observations(const MapDev& m, const double* T, const float* xyz, uint64_t n, cudaStream_t s,
                               int sms) {
  PoseD P;
  for (int i = 0; i < 16; ++i) P.T[i] = T[i];
  k_zero_obs_counts<<<sms * 2, 256, 0, s>>>(m);
  if (n == 0) {
    k_obs_segments<<<sms * 2, 256, 0, s>>>(m);
    return;
  }
  const unsigned blocks = (unsigned)((n + 127) / 128);
  k_lidar_stage<<<blocks, 128, 0, s>>>(m, P, n);
  k_obs_segments<<<sms * 2, 256, 0, s>>>(m);
  k_lidar_scatter<<<sms * 8, 256, 0, s>>>(m, n);
  k_lidar_fill_over<<<sms * 4, 128, 0, s>>>(m, P);  // points whose runs did not fit the stage (usually none)
}

void launch_fuse_points(const MapDev& m, const double*, const float*, uint64_t, cudaStream_t s, int sms) {
  const int grid = sms * 8;  // more CTAs than fit (5 per SM at 96 registers); the warps take items from a counter
  if (m.fp16) {
    if (m.color) k_fuse_points<true, true><<<grid, 32 * kLidarWarps, 0, s>>>(m);
    else k_fuse_points<true, false><<<grid, 32 * kLidarWarps, 0, s>>>(m);
  } else {
    if (m.color) k_fuse_points<false, true><<<grid, 32 * kLidarWarps, 0, s>>>(m);
    else k_fuse_points<false, false><<<grid, 32 * kLidarWarps, 0, s>>>(m);
  }
}

}  // namespace mrh
