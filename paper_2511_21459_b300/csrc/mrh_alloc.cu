// Kernels and launchers of ray -> block allocation for one map (device code in mrh_alloc.cuh).
#include "mrh_alloc.cuh"

namespace mrh {
namespace {

constexpr int kTileW = 32, kTileH = 8, kProbeW = 32;  // single-map shapes (the batched path tunes its own)

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
  const uint32_t n = min(m.st->touched_all, m.max_touched);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) bin_one(m, i);
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

}  // namespace mrh
