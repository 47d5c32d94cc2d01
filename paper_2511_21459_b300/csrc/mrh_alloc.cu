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

void launch_bin_camera(const MapDev& m, const CamArgs& c, const float* rho_img, cudaStream_t s, int sms) {
  if (m.pred_w || m.cap_feat) k_bin_predict<<<sms * 2, 256, 0, s>>>(m, c, rho_img);
  else k_bin<<<sms * 2, 256, 0, s>>>(m);
}

}  // namespace mrh
