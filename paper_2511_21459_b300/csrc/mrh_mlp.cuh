// Learned level predictor (an addition; not in the paper): a 16 -> 64 -> 64 -> 3 MLP with GELU that predicts, from
// features of a new block (its neighbourhood in the current range image, or the moments of a LiDAR scan's end points
// inside it), the level the block will end at under the variance rule, so it can be allocated and fused at that level
// from its first frame. The variance rule still runs afterwards and re-levels any block the network got wrong.
//
// Everything that decides a level is computed with +, -, *, / and sqrt only (compiled without multiply-add
// contraction), in a fixed order, so that the CPU oracle reproduces every decision bit for bit:
//   - exp(x): Cody-Waite range reduction x = k ln2 + r with a two-part ln2, degree-6 Taylor polynomial in r (Horner),
//     scaled by 2^k (exact);
//   - erf(x): Abramowitz & Stegun 7.1.26, erf(x) = 1 - (a1 t + ... + a5 t^5) exp(-x^2), t = 1 / (1 + p x), |error| <
//     1.5e-7, odd extension;
//   - GELU(x) = x (1 + erf(x / sqrt 2)) / 2;
//   - BF16 rounding: round to nearest even on the float bit pattern.
// Weights and activations are BF16 values; sums are float, accumulated in index order.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "mrh_internal.cuh"

namespace mrh {

constexpr int kMlpIn = 16, kMlpH = 64, kMlpOut = 3;
// packed parameter layout: W1 [in][h], b1 [h], W2 [h][h], b2 [h], W3 [h][out], b3 [out]
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kMlpIn * kMlpH;
constexpr int kOffW2 = kOffB1 + kMlpH;
constexpr int kOffB2 = kOffW2 + kMlpH * kMlpH;
constexpr int kOffW3 = kOffB2 + kMlpH;
constexpr int kOffB3 = kOffW3 + kMlpH * kMlpOut;
constexpr int kMlpParams = kOffB3 + kMlpOut;  // 5443
static_assert(kMlpParams == MRH_MLP_PARAMS && kMlpIn == MRH_MLP_IN && kMlpH == MRH_MLP_HIDDEN &&
                  kMlpOut == MRH_MLP_LEVELS,
              "packed layout of the C ABI");

__host__ __device__ inline float bf16_round(float x) {
  uint32_t u;
  memcpy(&u, &x, 4);
  if ((u & 0x7F800000u) == 0x7F800000u) return x;  // inf / nan unchanged
  u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
  float r;
  memcpy(&r, &u, 4);
  return r;
}

// BF16 bit pattern -> float (exact)
__host__ __device__ inline float bf16_to_float(uint16_t h) {
  const uint32_t u = (uint32_t)h << 16;
  float r;
  memcpy(&r, &u, 4);
  return r;
}

__host__ __device__ inline uint16_t float_to_bf16(float x) {
  const float r = bf16_round(x);
  uint32_t u;
  memcpy(&u, &r, 4);
  return (uint16_t)(u >> 16);
}

__host__ __device__ inline float mlp_exp(float x) {
  if (x < -87.0f) return 0.0f;
  if (x > 87.0f) x = 87.0f;
  const float inv_ln2 = 1.44269504088896341f;
  const float ln2_hi = 0.693145751953125f, ln2_lo = 1.428606765330187e-06f;
  const float kf = floorf(x * inv_ln2 + 0.5f);
  const float r = (x - kf * ln2_hi) - kf * ln2_lo;
  float p = 1.0f / 720.0f;
  p = p * r + 1.0f / 120.0f;
  p = p * r + 1.0f / 24.0f;
  p = p * r + 1.0f / 6.0f;
  p = p * r + 0.5f;
  p = p * r + 1.0f;
  p = p * r + 1.0f;
  return ldexpf(p, (int)kf);
}

__host__ __device__ inline float mlp_erf(float x) {
  const float ax = x < 0.0f ? -x : x;
  const float t = 1.0f / (1.0f + 0.3275911f * ax);
  float poly = 1.061405429f;
  poly = poly * t - 1.453152027f;
  poly = poly * t + 1.421413741f;
  poly = poly * t - 0.284496736f;
  poly = poly * t + 0.254829592f;
  poly = poly * t;
  const float y = 1.0f - poly * mlp_exp(-(ax * ax));
  return x < 0.0f ? -y : y;
}

__host__ __device__ inline float mlp_gelu(float x) { return 0.5f * x * (1.0f + mlp_erf(x * 0.70710678118654752f)); }

// d GELU / dx = (1 + erf(x / sqrt 2)) / 2 + x exp(-x^2 / 2) / sqrt(2 pi)
__host__ __device__ inline float mlp_gelu_grad(float x) {
  return 0.5f * (1.0f + mlp_erf(x * 0.70710678118654752f)) + x * mlp_exp(-0.5f * x * x) * 0.39894228040143268f;
}

// Inference of one sample: x (kMlpIn, already BF16 values) -> logits. w: BF16 weights (bit patterns). A product of
// two BF16 values is exact in float, so only the sums round, in index order.
__device__ inline void mlp_infer(const uint16_t* __restrict__ w, const float x[kMlpIn], float logits[kMlpOut]) {
  float h1[kMlpH];
  for (int j = 0; j < kMlpH; ++j) {
    float a = bf16_to_float(w[kOffB1 + j]);
    for (int k = 0; k < kMlpIn; ++k) a = a + x[k] * bf16_to_float(w[kOffW1 + k * kMlpH + j]);
    h1[j] = bf16_round(mlp_gelu(a));
  }
  float h2[kMlpH];
  for (int j = 0; j < kMlpH; ++j) {
    float a = bf16_to_float(w[kOffB2 + j]);
    for (int k = 0; k < kMlpH; ++k) a = a + h1[k] * bf16_to_float(w[kOffW2 + k * kMlpH + j]);
    h2[j] = bf16_round(mlp_gelu(a));
  }
  for (int j = 0; j < kMlpOut; ++j) {
    float a = bf16_to_float(w[kOffB3 + j]);
    for (int k = 0; k < kMlpH; ++k) a = a + h2[k] * bf16_to_float(w[kOffW3 + k * kMlpOut + j]);
    logits[j] = a;
  }
}

// The same network evaluated by a whole warp for one sample (every lane passes the same x): lane j owns hidden units
// j and j + 32 and sums their inputs in index order; the other lanes' activations arrive by shuffle. Every lane
// returns the same level (first argmax, clamped to L - 1), bit-identical to mlp_infer's.
__device__ inline int warp_mlp_level(const uint16_t* __restrict__ w, const float x[kMlpIn], int L) {
  const int lane = threadIdx.x & 31;
  float a0 = bf16_to_float(w[kOffB1 + lane]), a1 = bf16_to_float(w[kOffB1 + lane + 32]);
#pragma unroll
  for (int k = 0; k < kMlpIn; ++k) {
    a0 = a0 + x[k] * bf16_to_float(w[kOffW1 + k * kMlpH + lane]);
    a1 = a1 + x[k] * bf16_to_float(w[kOffW1 + k * kMlpH + lane + 32]);
  }
  const float h1a = bf16_round(mlp_gelu(a0)), h1b = bf16_round(mlp_gelu(a1));
  a0 = bf16_to_float(w[kOffB2 + lane]);
  a1 = bf16_to_float(w[kOffB2 + lane + 32]);
#pragma unroll 16
  for (int k = 0; k < kMlpH; ++k) {
    const float hk = __shfl_sync(0xffffffffu, k < 32 ? h1a : h1b, k & 31);
    a0 = a0 + hk * bf16_to_float(w[kOffW2 + k * kMlpH + lane]);
    a1 = a1 + hk * bf16_to_float(w[kOffW2 + k * kMlpH + lane + 32]);
  }
  const float h2a = bf16_round(mlp_gelu(a0)), h2b = bf16_round(mlp_gelu(a1));
  float z[kMlpOut];
#pragma unroll
  for (int c = 0; c < kMlpOut; ++c) z[c] = bf16_to_float(w[kOffB3 + c]);
#pragma unroll 16
  for (int k = 0; k < kMlpH; ++k) {
    const float hk = __shfl_sync(0xffffffffu, k < 32 ? h2a : h2b, k & 31);
#pragma unroll
    for (int c = 0; c < kMlpOut; ++c) z[c] = z[c] + hk * bf16_to_float(w[kOffW3 + k * kMlpOut + c]);
  }
  int best = 0;
#pragma unroll
  for (int c = 1; c < kMlpOut; ++c)
    if (z[c] > z[best]) best = c;
  return best < L - 1 ? best : L - 1;
}

// x / (1 + |x|): maps unbounded ratios (slopes, spreads) into (-1, 1)
__device__ inline float squash(float x) { return x / (1.0f + fabsf(x)); }

// Features of a new block (bx, by, bz) from the frame's range image (rho, -1 = invalid), computed by a whole warp
// (every lane passes the same block and returns the same features): lanes 0..24 fetch the 25 samples, every lane
// then holds all of them and evaluates the statistics serially in sample order. Returns false (on every lane) when
// the block's centre does not project into the image; the variance rule's finest level is used then. Feature values
// are rounded to BF16 (the network's input precision).
__device__ inline bool warp_block_features(const MapDev& m, const CamArgs& c, const float* __restrict__ rho_img,
                                           int bx, int by, int bz, float f[kMlpIn]) {
  const float E = m.E, tau = m.tau;
  const float cw0 = ((float)bx + 0.5f) * E - c.t[0];
  const float cw1 = ((float)by + 0.5f) * E - c.t[1];
  const float cw2 = ((float)bz + 0.5f) * E - c.t[2];
  const float xc = c.R[0] * cw0 + c.R[3] * cw1 + c.R[6] * cw2;
  const float yc = c.R[1] * cw0 + c.R[4] * cw1 + c.R[7] * cw2;
  const float zc = c.R[2] * cw0 + c.R[5] * cw1 + c.R[8] * cw2;
  if (!(zc > 0.0f)) return false;
  const float uf = c.fx * xc / zc + c.cx, vf = c.fy * yc / zc + c.cy;
  if (!(uf >= 0.0f && uf < (float)c.width && vf >= 0.0f && vf < (float)c.height)) return false;
  const int u0 = (int)floorf(uf + 0.5f), v0 = (int)floorf(vf + 0.5f);
  const float dist = sqrtf(xc * xc + yc * yc + zc * zc);
  const float rpix = c.fx * (0.5f * E) / zc;
  int s = (int)floorf(0.5f * rpix);
  if (s < 1) s = 1;
  if (s > 16) s = 16;
  // 5 x 5 samples spaced s pixels around the projection, row by row; lane q < 25 fetches sample q
  const int lane = threadIdx.x & 31;
  float mine = -1.0f;
  if (lane < 25) {
    const int u = u0 + (lane % 5 - 2) * s, v = v0 + (lane / 5 - 2) * s;
    if (u >= 0 && u < c.width && v >= 0 && v < c.height) mine = rho_img[(size_t)v * c.width + u];
  }
  float p[25];
#pragma unroll
  for (int q = 0; q < 25; ++q) p[q] = __shfl_sync(0xffffffffu, mine, q);
  int n = 0;
  float sum = 0.0f, sum2 = 0.0f, mn = 0.0f, mx = 0.0f;
#pragma unroll
  for (int q = 0; q < 25; ++q) {
    const float r = p[q];
    if (r >= 0.0f) {
      if (n == 0 || r < mn) mn = r;
      if (n == 0 || r > mx) mx = r;
      sum = sum + r;
      sum2 = sum2 + r * r;
      n = n + 1;
    }
  }
  float mean = 0.0f, sd = 0.0f;
  if (n > 0) {
    mean = sum / (float)n;
    float var = sum2 / (float)n - mean * mean;
    sd = var > 0.0f ? sqrtf(var) : 0.0f;
  }
  // slopes from the centre row / column, second differences as a noise proxy
  const float pix_m = dist / c.fx * (float)s;  // metres per sample step at the block's distance
  float gu = 0.0f, gv = 0.0f;
  if (p[11] >= 0.0f && p[13] >= 0.0f) gu = (p[13] - p[11]) / (2.0f * pix_m);
  if (p[7] >= 0.0f && p[17] >= 0.0f) gv = (p[17] - p[7]) / (2.0f * pix_m);
  float d2 = 0.0f;
  int nd2 = 0;
#pragma unroll
  for (int j = 0; j < 5; ++j)
#pragma unroll
    for (int i = 1; i < 4; ++i) {
      const float a = p[5 * j + i - 1], b = p[5 * j + i], cc = p[5 * j + i + 1];
      if (a >= 0.0f && b >= 0.0f && cc >= 0.0f) {
        const float q = a - 2.0f * b + cc;
        d2 = d2 + fabsf(q);
        nd2 = nd2 + 1;
      }
    }
  if (nd2 > 0) d2 = d2 / (float)nd2;
  f[0] = dist;
  f[1] = squash(n > 0 ? (mean - dist) / tau : 0.0f);
  f[2] = squash(sd / tau);
  f[3] = squash(n > 0 ? (mx - mn) / E : 0.0f);
  f[4] = (float)n / 25.0f;
  f[5] = E / dist;
  f[6] = squash(fabsf(gu));
  f[7] = squash(fabsf(gv));
  f[8] = squash(d2 / E);
  const float du = uf / (float)c.width - 0.5f, dv = vf / (float)c.height - 0.5f;
  f[9] = 2.0f * fabsf(du);
  f[10] = 2.0f * fabsf(dv);
  f[11] = zc / dist;
  f[12] = 1.0f / dist;
  f[13] = 0.0f;  // sensor type: camera
  f[14] = tau / E;
  f[15] = 1.0f;
#pragma unroll
  for (int k = 0; k < kMlpIn; ++k) f[k] = bf16_round(f[k]);
  return true;
}

// The 16 features of a new block of a LiDAR scan from its kLidarMoments end-point moments (one thread; the block
// centre relative to the sensor in double, the pose's precision, then float in source order: the same values as the
// CPU definition): distance r and unit direction u from the sensor to the block centre; centroid offset o from the
// centre and covariance C of the end points in block units; f0 r; f1 S(o.u E / tau); f2 S(sqrt(u^T C u) E / tau);
// f3 sqrt(tr C - u^T C u); f4 S(n / 16); f5 E / r; f6 sqrt(C_zz); f7 |o - (o.u) u|; f8 [n > 0]; f9 |u_z|; f10 u_z;
// f11 sqrt(tr C); f12 1 / r; f13 1 (LiDAR); f14 tau / E; f15 1 (S(x) = x / (1 + |x|)); each rounded to BF16.
__device__ inline void lidar_block_features(const unsigned long long* __restrict__ mom, const double* T, float E,
                                            float tau, int bx, int by, int bz, float f[kMlpIn]) {
  const double Ed = (double)E;
  const float c0 = (float)(((double)bx + 0.5) * Ed - T[3]);
  const float c1 = (float)(((double)by + 0.5) * Ed - T[7]);
  const float c2 = (float)(((double)bz + 0.5) * Ed - T[11]);
  const float r = sqrtf(c0 * c0 + c1 * c1 + c2 * c2);
  const float u0 = c0 / r, u1 = c1 / r, u2 = c2 / r;
  const unsigned long long cnt = mom[0];
  float along = 0.0f, thick2 = 0.0f, total = 0.0f, czz = 0.0f, lateral_off = 0.0f;
  if (cnt > 0) {
    const float nf = (float)cnt;
    const float mx = (float)mom[1] / nf, my = (float)mom[2] / nf, mz = (float)mom[3] / nf;
    const float ox = (mx + 0.5f) / 1024.0f - 0.5f, oy = (my + 0.5f) / 1024.0f - 0.5f;
    const float oz = (mz + 0.5f) / 1024.0f - 0.5f;
    const float cxx = ((float)mom[4] / nf - mx * mx) / 1048576.0f;
    const float cyy = ((float)mom[5] / nf - my * my) / 1048576.0f;
    czz = ((float)mom[6] / nf - mz * mz) / 1048576.0f;
    const float cxy = ((float)mom[7] / nf - mx * my) / 1048576.0f;
    const float cxz = ((float)mom[8] / nf - mx * mz) / 1048576.0f;
    const float cyz = ((float)mom[9] / nf - my * mz) / 1048576.0f;
    along = ox * u0 + oy * u1 + oz * u2;
    const float cu0 = cxx * u0 + cxy * u1 + cxz * u2;
    const float cu1 = cxy * u0 + cyy * u1 + cyz * u2;
    const float cu2 = cxz * u0 + cyz * u1 + czz * u2;
    thick2 = u0 * cu0 + u1 * cu1 + u2 * cu2;
    total = cxx + cyy + czz;
    const float l0 = ox - along * u0, l1 = oy - along * u1, l2 = oz - along * u2;
    lateral_off = sqrtf(l0 * l0 + l1 * l1 + l2 * l2);
  }
  const float lat2 = total - thick2;
  f[0] = r;
  f[1] = squash(along * E / tau);
  f[2] = squash(sqrtf(thick2 > 0.0f ? thick2 : 0.0f) * E / tau);
  f[3] = sqrtf(lat2 > 0.0f ? lat2 : 0.0f);
  f[4] = squash((float)cnt / 16.0f);
  f[5] = E / r;
  f[6] = sqrtf(czz > 0.0f ? czz : 0.0f);
  f[7] = lateral_off;
  f[8] = cnt > 0 ? 1.0f : 0.0f;
  f[9] = fabsf(u2);
  f[10] = u2;
  f[11] = sqrtf(total > 0.0f ? total : 0.0f);
  f[12] = 1.0f / r;
  f[13] = 1.0f;
  f[14] = tau / E;
  f[15] = 1.0f;
#pragma unroll
  for (int k = 0; k < kMlpIn; ++k) f[k] = bf16_round(f[k]);
}

}  // namespace mrh
