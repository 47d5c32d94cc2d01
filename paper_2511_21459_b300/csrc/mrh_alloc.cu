// Kernels and launchers of ray -> block allocation for one map (device code in mrh_alloc.cuh).
#include "mrh_alloc.cuh"
#include "mrh_mlp.cuh"

namespace mrh {
namespace {

// single-map shapes (the batched path tunes its own): 4-lane probe groups measured fastest among 4, 8, 16, 32
constexpr int kTileW = 32, kTileH = 8, kProbeW = 4;

__global__ void __launch_bounds__(256) k_alloc_depth(MapDev m, CamArgs c, const float* __restrict__ depth,
                                                     const uint8_t* __restrict__ rgb, float* __restrict__ rho_img,
                                                     uint32_t* __restrict__ rgb_img) {
  __shared__ unsigned long long s_set[kSetCap];
  __shared__ uint32_t s_valid;
  alloc_depth_tile<kTileW, kTileH, kProbeW>(m, c, depth, rgb, rho_img, rgb_img, blockIdx.x, blockIdx.y, s_set,
                                            &s_valid);
}

__global__ void __launch_bounds__(256) k_alloc_points(MapDev m, PoseD P, const float* __restrict__ xyz, uint64_t n) {
  __shared__ unsigned long long s_set[kSetCap];
  __shared__ uint32_t s_valid;
  alloc_points_cta<kProbeW>(m, P, xyz, n, (uint64_t)blockIdx.x * blockDim.x, s_set, &s_valid);
}

__global__ void __launch_bounds__(256) k_bin(MapDev m) {
  bin_entries(m, blockIdx.x * blockDim.x + (threadIdx.x & ~31u), gridDim.x * blockDim.x);
}

// Camera frames with the learned predictor or feature capture on: binning with the prediction folded in. Lane k of
// warp w takes entry w + k W (W = warps in the grid), so that the new blocks of a frame, which sit next to each other
// in the touched list, fall into different warps. For each new block of its 32 entries the warp computes the features
// and, with a predictor, the level (warp_block_features, warp_mlp_level, the weights staged in shared memory); with
// capture on, lane 0 appends (key, features). Then the entries are binned as in k_bin.
__global__ void __launch_bounds__(256) k_bin_predict(MapDev m, CamArgs c, const float* __restrict__ rho_img) {
  __shared__ __align__(16) uint16_t s_w[(kMlpParams + 7) & ~7];
  if (m.pred_w) {
    for (int t = threadIdx.x; t < kMlpParams; t += blockDim.x) s_w[t] = m.pred_w[t];
  }
  __syncthreads();
  const uint32_t n = min(m.st->touched_all, m.max_touched);
  const int lane = threadIdx.x & 31;
  const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  for (uint32_t base = warp; base < n; base += n_warps * 32u) {  // warp-uniform
    const uint32_t i = base + (uint32_t)lane * n_warps;
    uint32_t s = 0;
    bool fresh = false;
    if (i < n) {
      s = m.touched_all[i];
      fresh = m.slots[s].val == kValPending;
    }
    unsigned todo = __ballot_sync(0xffffffffu, fresh);
    int my_level = 0;
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1;
      const uint32_t ss = __shfl_sync(0xffffffffu, s, src);
      int bx, by, bz;
      unpack_key(m.slots[ss].key, &bx, &by, &bz);
      float f[kMlpIn];
      if (!warp_block_features(m, c, rho_img, bx, by, bz, f)) continue;  // same answer on every lane
      const int l = m.pred_w ? warp_mlp_level(s_w, f, m.L) : 0;
      if (lane == src) my_level = l;
      if (m.cap_feat && lane == 0) {
        const uint32_t r = atomicAdd(m.cap_count, 1u);
        if (r < m.cap_max) {
          m.cap_keys[3 * r] = bx;
          m.cap_keys[3 * r + 1] = by;
          m.cap_keys[3 * r + 2] = bz;
          for (int k = 0; k < kMlpIn; ++k) m.cap_feat[(size_t)kMlpIn * r + k] = f[k];
        }
      }
    }
    int l = -1;
    uint32_t val = 0;
    if (i < n) l = bin_entry(m, s, my_level, &val);
    append_binned(m, l, s, val);
  }
}

// LiDAR scans with the learned predictor or feature capture on, after allocation (Sec. 3.2.1 would start every new
// block at the finest level; the predictor picks its level here). Four passes, each balanced over the grid:
//   k_lidar_fresh     each new block of the scan (pending slot among the touched entries) is listed in `fresh`,
//                     records its touched index in slot_pos (binning overwrites it) and zeroes its moments;
//   k_lidar_moments   per point: the end point's block, when new to the scan, takes the point's moments;
//   k_lidar_levels    one warp per listed block: lane 0 computes its 16 features (lidar_block_features), the warp
//                     evaluates the network (warp_mlp_level) and keeps the level per touched index; with capture
//                     on, lane 0 appends the (key, features) record;
//   k_bin_levels      binning as k_bin, a new block at its predicted level.
__global__ void __launch_bounds__(256) k_lidar_fresh(MapDev m) {
  const uint32_t n = min(m.st->touched_all, m.max_touched);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t s = m.touched_all[i];
    if (m.slots[s].val != kValPending) continue;
    m.slot_pos[s] = i;
    for (int k = 0; k < kLidarMoments; ++k) m.lidar_mom[(size_t)kLidarMoments * i + k] = 0ull;
    m.fresh_level[i] = 0;
    m.fresh[atomicAdd(&m.st->n_fresh, 1u)] = i;
  }
}

__global__ void __launch_bounds__(256) k_lidar_moments(MapDev m, uint64_t n) {
  const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const long long e[3] = {m.lidar_end[3 * j], m.lidar_end[3 * j + 1], m.lidar_end[3 * j + 2]};
  if (e[0] == kNoEndPoint) return;
  const long long k[3] = {floor_div(e[0], kBlockUnit), floor_div(e[1], kBlockUnit), floor_div(e[2], kBlockUnit)};
  if (!key_ok(k[0], k[1], k[2])) return;
  const int s = lookup_slot(m.slots, m.slot_mask, pack_key(k[0], k[1], k[2]));
  if (s < 0 || m.slots[s].val != kValPending) return;
  const uint32_t i = m.slot_pos[s];
  if (i >= min(m.st->touched_all, m.max_touched) || m.touched_all[i] != (uint32_t)s) return;
  unsigned long long q[3];  // position in the block, units of E / 1024
#pragma unroll
  for (int a = 0; a < 3; ++a) q[a] = (unsigned long long)((e[a] - k[a] * kBlockUnit) >> (kFracBits - 10));
  unsigned long long* M = m.lidar_mom + (size_t)kLidarMoments * i;
  atomicAdd(&M[0], 1ull);
  atomicAdd(&M[1], q[0]);
  atomicAdd(&M[2], q[1]);
  atomicAdd(&M[3], q[2]);
  atomicAdd(&M[4], q[0] * q[0]);
  atomicAdd(&M[5], q[1] * q[1]);
  atomicAdd(&M[6], q[2] * q[2]);
  atomicAdd(&M[7], q[0] * q[1]);
  atomicAdd(&M[8], q[0] * q[2]);
  atomicAdd(&M[9], q[1] * q[2]);
}

__global__ void __launch_bounds__(256) k_lidar_levels(MapDev m, PoseD P) {
  __shared__ __align__(16) uint16_t s_w[(kMlpParams + 7) & ~7];
  if (m.pred_w) {
    for (int t = threadIdx.x; t < kMlpParams; t += blockDim.x) s_w[t] = m.pred_w[t];
  }
  __syncthreads();
  const uint32_t nf = m.st->n_fresh;
  const int lane = threadIdx.x & 31;
  const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t f = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; f < nf; f += n_warps) {  // warp-uniform
    const uint32_t i = m.fresh[f];
    int bx, by, bz;
    unpack_key(m.slots[m.touched_all[i]].key, &bx, &by, &bz);
    float x[kMlpIn];
    if (lane == 0) lidar_block_features(m.lidar_mom + (size_t)kLidarMoments * i, P.T, m.E, m.tau, bx, by, bz, x);
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) x[k] = __shfl_sync(0xffffffffu, x[k], 0);
    if (m.pred_w) {
      const int l = warp_mlp_level(s_w, x, m.L);
      if (lane == 0) m.fresh_level[i] = (uint8_t)l;
    }
    if (m.cap_feat && lane == 0) {
      const uint32_t r = atomicAdd(m.cap_count, 1u);
      if (r < m.cap_max) {
        m.cap_keys[3 * r] = bx;
        m.cap_keys[3 * r + 1] = by;
        m.cap_keys[3 * r + 2] = bz;
        for (int k = 0; k < kMlpIn; ++k) m.cap_feat[(size_t)kMlpIn * r + k] = x[k];
      }
    }
  }
}

__global__ void __launch_bounds__(256) k_bin_levels(MapDev m) {
  const uint32_t n = min(m.st->touched_all, m.max_touched);
  const int lane = threadIdx.x & 31;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < n; base += stride) {
    const uint32_t i = base + lane;
    int l = -1;
    uint32_t s = 0, val = 0;
    if (i < n) {
      s = m.touched_all[i];
      l = bin_entry(m, s, m.fresh_level[i], &val);  // used for a pending slot only: k_lidar_fresh set it
    }
    append_binned(m, l, s, val);
  }
}

}  // namespace

void launch_alloc_depth(const MapDev& m, const CamArgs& c, const float* depth, const uint8_t* rgb, float* rho_img,
                        uint32_t* rgb_img, cudaStream_t s) {
  dim3 grid((c.width + kTileW - 1) / kTileW, (c.height + kTileH - 1) / kTileH);
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

void launch_bin_points(const MapDev& m, const double* T, const float* xyz, uint64_t n, cudaStream_t s, int sms) {
  (void)xyz;
  PoseD P;
  for (int i = 0; i < 16; ++i) P.T[i] = T[i];
  k_lidar_fresh<<<sms * 2, 256, 0, s>>>(m);
  if (n) k_lidar_moments<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(m, n);
  k_lidar_levels<<<sms * 2, 256, 0, s>>>(m, P);
  k_bin_levels<<<sms * 2, 256, 0, s>>>(m);
}

void launch_bin_camera(const MapDev& m, const CamArgs& c, const float* rho_img, cudaStream_t s, int sms) {
  if (m.pred_w || m.cap_feat) k_bin_predict<<<sms * 2, 256, 0, s>>>(m, c, rho_img);
  else k_bin<<<sms * 2, 256, 0, s>>>(m);
}

}  // namespace mrh
