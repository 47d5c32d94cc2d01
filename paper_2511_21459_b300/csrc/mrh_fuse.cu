// Kernels and launchers of fusion for one map, and the LiDAR observation passes (device code in mrh_fuse.cuh).
#include "mrh_fuse.cuh"

namespace mrh {
namespace {

constexpr int kCamWarps = 8;

template <bool FP16, bool COLOR>
__global__ void __launch_bounds__(32 * kCamWarps, 3) k_fuse_depth(MapDev m, CamArgs c, const float* __restrict__ rho,
                                                                 const uint32_t* __restrict__ rgb) {
  CameraObs<FP16, COLOR> obs{c, rho, rgb};
  const int warp = threadIdx.x >> 5;
  fuse_warp_body<FP16, COLOR>(m, obs, warp, blockIdx.x * kCamWarps + warp, gridDim.x * kCamWarps);
}

template <bool FP16, bool COLOR>
__global__ void __launch_bounds__(32 * kLidarWarps) k_fuse_points(MapDev m) {
  __shared__ uint32_t s_bins[kLidarWarps][3][512];
  LidarObs<FP16> obs{s_bins, 0};
  const int warp = threadIdx.x >> 5;
  fuse_warp_body<FP16, COLOR>(m, obs, warp, blockIdx.x * kLidarWarps + warp, gridDim.x * kLidarWarps);
}

// -------------------------------------------------------------------------------------------- LiDAR observation passes

// FILL = false: count each block's observations; FILL = true: write them (point index, voxel, d).
template <bool FILL>
__global__ void __launch_bounds__(128) k_lidar_walk(MapDev m, PoseD P, const float* __restrict__ xyz, uint64_t n) {
  const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  long long A[3], B[3];
  double rho;
  double rhat[3];
  if (!lidar_ray(m, P, xyz, j, A, B, &rho, rhat)) return;
  const uint32_t n0 = min(m.st->touched_count[0], m.max_touched);
  const uint32_t n1 = min(m.st->touched_count[1], m.max_touched);
  const float rho_f = (float)rho;
  const float rh[3] = {(float)rhat[0], (float)rhat[1], (float)rhat[2]};
  const float o_f[3] = {(float)P.T[3], (float)P.T[7], (float)P.T[11]};

  int cb[3] = {0, 0, 0}, lg[3] = {0, 0, 0};
  bool have_block = false, cur_ok = false, have_last = false;
  int cl = 0;
  uint32_t cur_P = 0, run = 0;
  float ob[3] = {0.f, 0.f, 0.f};
  constexpr int kRunCap = 32;
  uint32_t rk[FILL ? kRunCap : 1];
  float rd[FILL ? kRunCap : 1];

  auto flush = [&]() {
    if (!cur_ok || run == 0) return;
    if constexpr (!FILL) {
      atomicAdd(&m.blk_count[cur_P], run);
    } else {
      uint32_t base = m.blk_off[cur_P] + atomicAdd(&m.blk_fill[cur_P], run);
      if (base + run <= m.max_obs) {
        for (uint32_t i = 0; i < run; ++i) m.obs_rec[base + i] = make_uint2(rk[i], __float_as_uint(rd[i]));
      } else {
        set_status(m.st, kStObsFull);
      }
    }
    run = 0;
  };

  bool ok = walk_cells(A, B, kVoxelShift, kMaxVoxelCells, [&](const int* f) {
    const int bk[3] = {f[0] >> 3, f[1] >> 3, f[2] >> 3};  // finest cell -> block (floor division by 8)
    if (!have_block || bk[0] != cb[0] || bk[1] != cb[1] || bk[2] != cb[2]) {
      flush();
      have_block = true;
      cb[0] = bk[0]; cb[1] = bk[1]; cb[2] = bk[2];
      have_last = false;
      cur_ok = false;
      int s = lookup_slot(m.slots, m.slot_mask, pack_key(bk[0], bk[1], bk[2]));
      if (s >= 0) {
        uint32_t val = m.slots[s].val;
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
    if constexpr (FILL) {
      if (run == kRunCap) flush();  // cannot happen at level 0 (<= 22 voxels of one block per ray), kept as a guard
      const float vl = m.v[cl];
      float xr0 = ob[0] + ((float)li[0] + 0.5f) * vl;
      float xr1 = ob[1] + ((float)li[1] + 0.5f) * vl;
      float xr2 = ob[2] + ((float)li[2] + 0.5f) * vl;
      float d = rho_f - (xr0 * rh[0] + xr1 * rh[1] + xr2 * rh[2]);
      if (d < -m.tau) d = -m.tau;
      if (d > m.tau) d = m.tau;
      rk[run] = ((uint32_t)j << 9) | (uint32_t)(li[0] + nl * (li[1] + nl * li[2]));
      rd[run] = d;
    }
    ++run;
  });
  flush();
  if (!ok) set_status(m.st, kStSegment);
}

__global__ void k_zero_obs_counts(MapDev m) {
  const uint32_t total = min(m.st->touched_count[0], m.max_touched) + min(m.st->touched_count[1], m.max_touched) +
                         min(m.st->touched_count[2], m.max_touched);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    m.blk_count[i] = 0;
    m.blk_fill[i] = 0;
  }
}

// exclusive prefix sum of the per-block observation counts (one CTA, 16 consecutive entries per thread)
__global__ void __launch_bounds__(1024) k_scan_obs(MapDev m) {
  __shared__ uint32_t s_w[32];
  __shared__ uint32_t s_carry;
  const uint32_t total = min(m.st->touched_count[0], m.max_touched) + min(m.st->touched_count[1], m.max_touched) +
                         min(m.st->touched_count[2], m.max_touched);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_carry = 0;
  __syncthreads();
  for (uint32_t base = 0; base < total; base += 1024u * 16u) {
    uint32_t v[16], sum = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      uint32_t i = base + (uint32_t)tid * 16u + k;
      v[k] = i < total ? m.blk_count[i] : 0u;
      sum += v[k];
    }
    uint32_t incl = sum;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(~0u, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      uint32_t w = s_w[lane];
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(~0u, w, o);
        if (lane >= o) w += t;
      }
      s_w[lane] = w;
    }
    __syncthreads();
    uint32_t run = s_carry + (warp > 0 ? s_w[warp - 1] : 0u) + incl - sum;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      uint32_t i = base + (uint32_t)tid * 16u + k;
      if (i < total) m.blk_off[i] = run;
      run += v[k];
    }
    __syncthreads();
    if (tid == 0) s_carry += s_w[31];
    __syncthreads();
  }
  if (tid == 0) m.blk_off[total] = s_carry;
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
    k_scan_obs<<<1, 1024, 0, s>>>(m);
    return;
  }
  const unsigned blocks = (unsigned)((n + 127) / 128);
  k_lidar_walk<false><<<blocks, 128, 0, s>>>(m, P, xyz, n);
  k_scan_obs<<<1, 1024, 0, s>>>(m);
  k_lidar_walk<true><<<blocks, 128, 0, s>>>(m, P, xyz, n);
}

void launch_fuse_points(const MapDev& m, const double*, const float*, uint64_t, cudaStream_t s, int sms) {
  const int grid = sms * 8;
  if (m.fp16) {
    if (m.color) k_fuse_points<true, true><<<grid, 32 * kLidarWarps, 0, s>>>(m);
    else k_fuse_points<true, false><<<grid, 32 * kLidarWarps, 0, s>>>(m);
  } else {
    if (m.color) k_fuse_points<false, true><<<grid, 32 * kLidarWarps, 0, s>>>(m);
    else k_fuse_points<false, false><<<grid, 32 * kLidarWarps, 0, s>>>(m);
  }
}

}  // namespace mrh
