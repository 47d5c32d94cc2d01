// Tile-based Gaussian-splat rasteriser of the rendering branch (Sec. 3.5): every 3D Gaussian is projected to the
// image (Eq. 7) and the projected Gaussians are alpha-blended front to back at every pixel (Eqs. 8, 9).
//
// What a pixel receives. Camera-frame mean R^T (mu - t) with the camera-to-world pose (R, t); Gaussians whose camera z
// lies outside [min_depth, max_depth] or whose image covariance Sigma_I = J R^T Sigma_W R J^T is not positive definite
// are not drawn. Gaussian m reaches pixel (u, v) (image coordinates u, v) when its squared Mahalanobis distance
// q <= 9 and |u - mu_u| <= 3 sqrt(Sigma_uu), |v - mu_v| <= 3 sqrt(Sigma_vv). The pixel's colour is
// sum_m C_m a_m exp(-q_m / 2) prod_{l in front of m} (1 - a_l exp(-q_l / 2)) over the Gaussians that reach it in
// increasing camera z (ties by index); the remaining product is its transmittance. The projection, the reach test and
// the depth order are float computations with a fixed operation order (this file is compiled without multiply-add
// contraction). A pixel stops once its transmittance falls below kSplatStop: the colour it would still receive is
// below kSplatStop times the largest colour, and its transmittance is off by less than kSplatStop.
//
// The work (one stream; one host read, of the number of tile-Gaussian pairs):
//   k_splat_project  one thread per Gaussian: Eq. 7, the three-sigma box, the tiles it overlaps (16 x 16 pixels)
//                    less those its q <= 9 ellipse cannot reach (tile_reached), a 48-byte record {mu_u, mu_v, ru,
//                    rv}, {conic uu, 2 conic uv, conic vv, alpha}, {colour, z} and its depth key (the bits of z:
//                    positive floats order as their bits; all ones when not drawn)
//   depth sort       stable least-significant-digit radix sort (8-bit digits) of the Gaussians by depth key, so
//                    equal depths stay in index order
//   k_splat_counts   the pair counts in depth order and each Gaussian's rank in it; then their exclusive prefix
//   k_splat_pairs    every (tile, Gaussian) pair, key = tile, value = Gaussian index, laid out in depth order
//   tile sort        the same stable radix sort over the tile bits only: a tile's pairs end up contiguous and keep
//                    the depth order
//   k_splat_ranges   each tile's first and last pair
//   k_splat_render   one CTA of 16 x 16 threads per tile; the tile's records are staged 256 at a time in shared
//                    memory and every thread blends its pixel through them; the CTA leaves when all its pixels
//                    have stopped
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "mrh_internal.cuh"
#include "mrh_sort.cuh"

namespace mrh {
namespace {

constexpr int kTile = 16;
constexpr float kSplatStop = 1e-4f;

struct SplatRec {
  float4 a;  // mu_u, mu_v, ru, rv
  float4 b;  // conic uu, 2 conic uv, conic vv, alpha
  float4 c;  // colour r, g, b, camera z
};

struct SplatGeo {
  int width, height, tiles_x, tiles_y;
};

// Gaussians whose box covers at most this many tiles have each tile tested against their ellipse; larger ones keep
// every tile of the box, so that no thread loops long
constexpr int kEllipseTest = 64;

// false when no pixel centre of tile (tx, ty) can satisfy the float reach test q <= 9: the least q over the
// rectangle spanned by the tile's pixel centres (zero when it holds the mean, else the least of the four edges'
// constrained minima) exceeds 9 by more than the float evaluations of q, here and per pixel, can err (a few ulps of
// a u^2 + 2 |b u v| + c v^2 over the rectangle, allowed for with a factor of 1e-5, plus 1e-3)
__device__ inline bool tile_reached(const SplatRec& o, int tx, int ty) {
  const float u0 = (float)(tx * kTile) - o.a.x, u1 = (float)(tx * kTile + kTile - 1) - o.a.x;
  const float v0 = (float)(ty * kTile) - o.a.y, v1 = (float)(ty * kTile + kTile - 1) - o.a.y;
  if (u0 <= 0.0f && u1 >= 0.0f && v0 <= 0.0f && v1 >= 0.0f) return true;
  const float a = o.b.x, b = 0.5f * o.b.y, c = o.b.z;
  float qmin = 3.0e38f;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const float ue = e ? u1 : u0, ve = e ? v1 : v0;
    const float dv = fminf(fmaxf(-(b * ue) / c, v0), v1);  // edge u = ue
    qmin = fminf(qmin, a * ue * ue + 2.0f * b * ue * dv + c * dv * dv);
    const float du = fminf(fmaxf(-(b * ve) / a, u0), u1);  // edge v = ve
    qmin = fminf(qmin, a * du * du + 2.0f * b * du * ve + c * ve * ve);
  }
  const float U = fmaxf(fabsf(u0), fabsf(u1)), V = fmaxf(fabsf(v0), fabsf(v1));
  const float mag = a * U * U + 2.0f * fabsf(b) * U * V + c * V * V;
  return !(qmin > 9.0f + 1e-5f * mag + 1e-3f);
}

// ---------------------------------------------------------------------------------------------------- projection

__global__ void __launch_bounds__(256) k_splat_project(SplatInputs in, CamArgs c, SplatGeo g, SplatRec* rec,
                                                       int4* rect, unsigned long long* reach, uint32_t* npairs,
                                                       uint32_t* zkey, uint32_t* zval) {
  for (uint64_t m = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; m < in.n; m += (uint64_t)gridDim.x * blockDim.x) {
    unsigned long long pairs = 0;
    int4 box = make_int4(0, 0, 0, 0);  // tiles [x, z) x [y, w); empty when the Gaussian is not drawn
    const float* mean = in.means + 3 * m;
    const float* cv = in.covs + 6 * m;
    const float* R = c.R;
    const float d0 = mean[0] - c.t[0], d1 = mean[1] - c.t[1], d2 = mean[2] - c.t[2];
    const float x = R[0] * d0 + R[3] * d1 + R[6] * d2;
    const float y = R[1] * d0 + R[4] * d1 + R[7] * d2;
    const float z = R[2] * d0 + R[5] * d1 + R[8] * d2;
    if (z >= c.min_depth && z <= c.max_depth) {
      const float iz = 1.0f / z;
      const float xz = x * iz, yz = y * iz;
      const float mu_u = c.fx * xz + c.cx, mu_v = c.fy * yz + c.cy;
      const float j00 = c.fx * iz, j02 = -(j00 * xz), j11 = c.fy * iz, j12 = -(j11 * yz);
      float M0[3], M1[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        M0[a] = j00 * R[3 * a] + j02 * R[3 * a + 2];
        M1[a] = j11 * R[3 * a + 1] + j12 * R[3 * a + 2];
      }
      const float S[3][3] = {{cv[0], cv[1], cv[2]}, {cv[1], cv[3], cv[4]}, {cv[2], cv[4], cv[5]}};
      float V0[3], V1[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        V0[a] = S[a][0] * M0[0] + S[a][1] * M0[1] + S[a][2] * M0[2];
        V1[a] = S[a][0] * M1[0] + S[a][1] * M1[1] + S[a][2] * M1[2];
      }
      const float suu = M0[0] * V0[0] + M0[1] * V0[1] + M0[2] * V0[2];
      const float suv = M1[0] * V0[0] + M1[1] * V0[1] + M1[2] * V0[2];
      const float svv = M1[0] * V1[0] + M1[1] * V1[1] + M1[2] * V1[2];
      const float det = suu * svv - suv * suv;
      if (det > 0.0f && suu > 0.0f) {
        const float ru = 3.0f * sqrtf(suu), rv = 3.0f * sqrtf(svv);
        // pixels within the box, widened by one pixel against rounding of the bounds, clamped to the image
        const float u0 = fmaxf(floorf(mu_u - ru) - 1.0f, 0.0f), u1 = fminf(ceilf(mu_u + ru) + 1.0f, g.width - 1.0f);
        const float v0 = fmaxf(floorf(mu_v - rv) - 1.0f, 0.0f), v1 = fminf(ceilf(mu_v + rv) + 1.0f, g.height - 1.0f);
        if (u0 <= u1 && v0 <= v1) {  // false for NaN bounds as well
          box = make_int4((int)u0 / kTile, (int)v0 / kTile, (int)u1 / kTile + 1, (int)v1 / kTile + 1);
          SplatRec o;
          o.a = make_float4(mu_u, mu_v, ru, rv);
          const float cb = -(suv / det);
          o.b = make_float4(svv / det, cb + cb, suu / det, in.opacity[m]);
          o.c = make_float4(in.colors[3 * m], in.colors[3 * m + 1], in.colors[3 * m + 2], z);
          rec[m] = o;
          const int tiles = (box.z - box.x) * (box.w - box.y);
          if (tiles <= kEllipseTest) {  // bit (ty - y) * width + (tx - x) of the box: tile reached
            unsigned long long bits = 0;
            int k = 0;
            for (int ty = box.y; ty < box.w; ++ty)
              for (int tx = box.x; tx < box.z; ++tx, ++k)
                if (tile_reached(o, tx, ty)) bits |= 1ull << k;
            reach[m] = bits;
            pairs = (unsigned long long)__popcll(bits);
          } else {
            pairs = (unsigned long long)tiles;
          }
        }
      }
    }
    rect[m] = box;
    npairs[m] = (uint32_t)pairs;
    zkey[m] = pairs ? __float_as_uint(z) : 0xFFFFFFFFu;
    zval[m] = (uint32_t)m;
  }
}

// pair count of each Gaussian in depth order, and each Gaussian's rank in that order
__global__ void __launch_bounds__(256) k_splat_counts(uint64_t n, const uint32_t* order, const uint32_t* npairs,
                                                      unsigned long long* count, uint32_t* rank) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t m = order[i];
    count[i] = npairs[m];
    rank[m] = (uint32_t)i;
  }
}

// ---------------------------------------------------------------------------------------------------- pairs

// Gaussians in index order (near ones, which overlap the most tiles, are spread over the grid that way), each
// writing its pairs at its place in the depth order (rank = position in the depth-sorted order)
__global__ void __launch_bounds__(256) k_splat_pairs(uint64_t n, const uint32_t* rank, const int4* rect,
                                                     const unsigned long long* reach, const unsigned long long* offset,
                                                     int tiles_x, uint32_t* keys, uint32_t* vals) {
  for (uint64_t m = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; m < n; m += (uint64_t)gridDim.x * blockDim.x) {
    const int4 r = rect[m];
    const int w = r.z - r.x, tiles = w * (r.w - r.y);
    if (tiles <= 0) continue;
    unsigned long long p = offset[rank[m]];
    if (tiles <= kEllipseTest) {  // the reached tiles of the box, in row-major order
      for (unsigned long long bits = reach[m]; bits; bits &= bits - 1, ++p) {
        const int k = __ffsll((long long)bits) - 1;
        keys[p] = (uint32_t)((r.y + k / w) * tiles_x + r.x + k % w);
        vals[p] = (uint32_t)m;
      }
    } else {
      for (int ty = r.y; ty < r.w; ++ty)
        for (int tx = r.x; tx < r.z; ++tx, ++p) {
          keys[p] = (uint32_t)(ty * tiles_x + tx);
          vals[p] = (uint32_t)m;
        }
    }
  }
}

// ---------------------------------------------------------------------------------------------------- render

__global__ void __launch_bounds__(256) k_splat_ranges(const uint32_t* keys, uint32_t n, uint2* ranges) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t t = keys[i];
    if (i == 0 || keys[i - 1] != t) ranges[t].x = i;
    if (i + 1 == n || keys[i + 1] != t) ranges[t].y = i + 1;
  }
}

__global__ void __launch_bounds__(kTile * kTile) k_splat_render(const uint2* ranges, const uint32_t* vals,
                                                               const SplatRec* rec, SplatGeo g, float* rgb,
                                                               float* trans) {
  __shared__ float4 s_a[kTile * kTile], s_b[kTile * kTile], s_c[kTile * kTile];
  const int tile = blockIdx.x;
  const int px = (tile % g.tiles_x) * kTile + (threadIdx.x % kTile);
  const int py = (tile / g.tiles_x) * kTile + (threadIdx.x / kTile);
  const bool inside = px < g.width && py < g.height;
  const uint2 r = ranges[tile];
  const float fu = (float)px, fv = (float)py;
  float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
  bool done = !inside;
  for (uint32_t start = r.x; start < r.y; start += kTile * kTile) {
    // also the barrier before the shared records are overwritten
    if (__syncthreads_count(done) == kTile * kTile) break;
    const uint32_t j = start + threadIdx.x;
    if (j < r.y) {
      const SplatRec& o = rec[vals[j]];
      s_a[threadIdx.x] = o.a;
      s_b[threadIdx.x] = o.b;
      s_c[threadIdx.x] = o.c;
    }
    __syncthreads();
    const int cnt = (int)min((uint32_t)(kTile * kTile), r.y - start);
    for (int k = 0; k < cnt && !done; ++k) {
      const float4 a = s_a[k];
      const float du = fu - a.x, dv = fv - a.y;
      if (!(fabsf(du) <= a.z && fabsf(dv) <= a.w)) continue;
      const float4 b = s_b[k];
      const float q = (b.x * (du * du) + b.y * (du * dv)) + b.z * (dv * dv);
      if (!(q <= 9.0f)) continue;
      const float w = b.w * expf(-0.5f * q);
      const float4 cc = s_c[k];
      C0 = C0 + (cc.x * w) * T;
      C1 = C1 + (cc.y * w) * T;
      C2 = C2 + (cc.z * w) * T;
      T = T * (1.0f - w);
      if (T < kSplatStop) done = true;
    }
  }
  if (inside) {
    const size_t p = (size_t)py * g.width + px;
    rgb[3 * p] = C0;
    rgb[3 * p + 1] = C1;
    rgb[3 * p + 2] = C2;
    if (trans) trans[p] = T;
  }
}

template <class T>
T* carve(uint8_t*& p, size_t count) {
  T* out = reinterpret_cast<T*>(p);
  p += (count * sizeof(T) + 255) & ~(size_t)255;
  return out;
}

size_t carve_bytes(size_t count, size_t size) { return (count * size + 255) & ~(size_t)255; }

}  // namespace

cudaError_t splat_render(const SplatInputs& in, const CamArgs& c, float* rgb, float* trans, uint64_t* n_pairs,
                         int device, cudaStream_t s, int sms) {
  SplatGeo g{c.width, c.height, (c.width + kTile - 1) / kTile, (c.height + kTile - 1) / kTile};
  const uint32_t n_tiles = (uint32_t)(g.tiles_x * g.tiles_y);
  *n_pairs = 0;
  const uint32_t n = (uint32_t)in.n;  // n < 2^32, checked by the caller
  const unsigned grid_n = (unsigned)std::min<uint64_t>((n + 255) / 256 + 1, (uint64_t)sms * 16);
  // phase 1: projection, depth order, pair counts
  const size_t nh1 = radix_scratch_words(n);
  const size_t bytes1 = carve_bytes(n, sizeof(SplatRec)) + carve_bytes(n, sizeof(int4)) + 6 * carve_bytes(n, 4) +
                        carve_bytes(n, 8) +
                        carve_bytes(n, 8) + carve_bytes(scan_sums_count(n), 8) + carve_bytes(nh1, 4) +
                        carve_bytes(scan_sums_count(nh1), 4) + 256;
  void* scratch1 = nullptr;
  cudaError_t e = scratch_alloc(&scratch1, bytes1, device, s);
  if (e != cudaSuccess) return e;
  uint8_t* p = (uint8_t*)scratch1;
  SplatRec* rec = carve<SplatRec>(p, n);
  int4* rect = carve<int4>(p, n);
  uint32_t* zkey[2] = {carve<uint32_t>(p, n), carve<uint32_t>(p, n)};
  uint32_t* zval[2] = {carve<uint32_t>(p, n), carve<uint32_t>(p, n)};
  uint32_t* rank = carve<uint32_t>(p, n);
  uint32_t* npairs = carve<uint32_t>(p, n);
  unsigned long long* reach = carve<unsigned long long>(p, n);
  unsigned long long* count = carve<unsigned long long>(p, n);
  unsigned long long* sums = carve<unsigned long long>(p, scan_sums_count(n));
  uint32_t* hist1 = carve<uint32_t>(p, nh1);
  uint32_t* sums1 = carve<uint32_t>(p, scan_sums_count(nh1));
  unsigned long long* total = carve<unsigned long long>(p, 1);
  int zc = 0;
  if (n > 0) {
    k_splat_project<<<grid_n, 256, 0, s>>>(in, c, g, rec, rect, reach, npairs, zkey[0], zval[0]);
    zc = radix_sort<uint32_t>(zkey, zval, n, 32, hist1, sums1, s);
    k_splat_counts<<<grid_n, 256, 0, s>>>(n, zval[zc], npairs, count, rank);
  }
  exclusive_scan<unsigned long long>(count, n, sums, total, s);  // count becomes each Gaussian's first pair
  unsigned long long P = 0;
  e = cudaMemcpyAsync(&P, total, sizeof(P), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaFreeAsync(scratch1, s);
    return e;
  }
  *n_pairs = P;
  if (P > kSplatMaxPairs) {  // the caller reports the capacity error; nothing is rendered
    cudaFreeAsync(scratch1, s);
    return cudaSuccess;
  }
  // phase 2: pairs in depth order, stable sort by tile, ranges, render
  const uint32_t np = (uint32_t)P;
  const size_t nh2 = radix_scratch_words(np);
  const size_t bytes2 = 4 * carve_bytes(np, 4) + carve_bytes(nh2, 4) + carve_bytes(scan_sums_count(nh2), 4) +
                        carve_bytes(n_tiles, sizeof(uint2)) + 256;
  void* scratch2 = nullptr;
  e = scratch_alloc(&scratch2, bytes2, device, s);
  if (e != cudaSuccess) {
    cudaFreeAsync(scratch1, s);
    return e;
  }
  p = (uint8_t*)scratch2;
  uint32_t* keys[2] = {carve<uint32_t>(p, np), carve<uint32_t>(p, np)};
  uint32_t* vals[2] = {carve<uint32_t>(p, np), carve<uint32_t>(p, np)};
  uint32_t* hist2 = carve<uint32_t>(p, nh2);
  uint32_t* sums2 = carve<uint32_t>(p, scan_sums_count(nh2));
  uint2* ranges = carve<uint2>(p, n_tiles);
  e = cudaMemsetAsync(ranges, 0, n_tiles * sizeof(uint2), s);
  if (e != cudaSuccess) {
    cudaFreeAsync(scratch2, s);
    cudaFreeAsync(scratch1, s);
    return e;
  }
  int cur = 0;
  if (np > 0) {
    k_splat_pairs<<<grid_n, 256, 0, s>>>(n, rank, rect, reach, count, g.tiles_x, keys[0], vals[0]);
    int tile_bits = 1;
    while ((1u << tile_bits) < n_tiles) ++tile_bits;
    cur = radix_sort<uint32_t>(keys, vals, np, tile_bits, hist2, sums2, s);
    k_splat_ranges<<<(unsigned)std::min<uint64_t>((np + 255) / 256, (uint64_t)sms * 16), 256, 0, s>>>(keys[cur], np,
                                                                                                     ranges);
  }
  k_splat_render<<<n_tiles, kTile * kTile, 0, s>>>(ranges, vals[cur], rec, g, rgb, trans);
  e = cudaGetLastError();
  cudaFreeAsync(scratch2, s);
  cudaFreeAsync(scratch1, s);
  return e;
}

}  // namespace mrh
