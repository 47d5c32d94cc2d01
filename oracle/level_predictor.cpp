/*
 * CPU oracle of the learned level predictor (an addition to the paper's method: the paper allocates every new block
 * at the finest level, Sec. 3.2.1, and has no predictor).
 *
 * TEST INFRASTRUCTURE ONLY, like mrh_oracle.cpp, and shares no code with the CUDA library. It restates the
 * predictor's definition (16 features of a new block: from the frame's range image for a depth camera, from the
 * moments of the scan's end points inside the block for a LiDAR scan; a 16-64-64-3 GELU network with BF16 weights and
 * activations, first argmax) in plain float arithmetic, one operation at a time in the order the definition
 * gives, so that its level decisions can be compared bit for bit. Compile with -ffp-contract=off.
 *
 * Published methods used (no library math in anything that decides a level):
 *   exp  Cody & Waite argument reduction x = k ln2 + r (ln2 split in a high part with trailing zero bits and a low
 *        part), then the Taylor polynomial of degree 6 in r evaluated by Horner's rule, times 2^k;
 *   erf  Abramowitz & Stegun, Handbook of Mathematical Functions, formula 7.1.26 (|error| <= 1.5e-7), odd extension;
 *   GELU x Phi(x) = x (1 + erf(x / sqrt 2)) / 2 (Hendrycks & Gimpel);
 *   BF16 round to nearest, ties to even, on the float32 bit pattern (inf / NaN passed through).
 *
 * Parity status: the exp / erf / GELU approximations are pinned to math library values within their published error
 * bounds; the forward pass is pinned to an independent float64 evaluation of the same network; the camera features
 * are pinned to closed forms on constant and linear range images, the LiDAR features to closed forms of point sets
 * with known moments and to a brute-force numpy evaluation from the raw points (tests/test_oracle_predictor.py).
 */
#include <cmath>
#include <cstdint>
#include <cstring>

namespace {

constexpr int kIn = 16, kHid = 64, kOut = 3;

float round_bf16(float x) {
  uint32_t bits;
  std::memcpy(&bits, &x, sizeof bits);
  if ((bits & 0x7F800000u) == 0x7F800000u) return x;
  const uint32_t lsb = (bits >> 16) & 1u;
  bits = bits + 0x7FFFu + lsb;
  bits = bits & 0xFFFF0000u;
  float y;
  std::memcpy(&y, &bits, sizeof y);
  return y;
}

float from_bf16(uint16_t h) {
  uint32_t bits = (uint32_t)h << 16;
  float y;
  std::memcpy(&y, &bits, sizeof y);
  return y;
}

float exp_cw(float x) {
  if (x < -87.0f) return 0.0f;
  if (x > 87.0f) x = 87.0f;
  // k = nearest integer to x / ln2; r = x - k ln2 with ln2 = 0.693145751953125 + 1.428606765330187e-06
  const float k = std::floor(x * 1.44269504088896341f + 0.5f);
  const float r = (x - k * 0.693145751953125f) - k * 1.428606765330187e-06f;
  // 1 + r + r^2/2! + ... + r^6/6!, Horner
  const float c[7] = {1.0f, 1.0f, 0.5f, 1.0f / 6.0f, 1.0f / 24.0f, 1.0f / 120.0f, 1.0f / 720.0f};
  float p = c[6];
  for (int i = 5; i >= 0; --i) p = p * r + c[i];
  return std::ldexp(p, (int)k);
}

float erf_as(float x) {
  const float a = x < 0.0f ? -x : x;
  const float t = 1.0f / (1.0f + 0.3275911f * a);
  // a1 t + a2 t^2 + ... + a5 t^5, Horner from a5
  float q = 1.061405429f;
  q = q * t + -1.453152027f;
  q = q * t + 1.421413741f;
  q = q * t + -0.284496736f;
  q = q * t + 0.254829592f;
  q = q * t;
  const float e = 1.0f - q * exp_cw(-(a * a));
  return x < 0.0f ? -e : e;
}

float gelu(float x) { return 0.5f * x * (1.0f + erf_as(x * 0.70710678118654752f)); }

struct Cam {
  float fx, fy, cx, cy;
  int w, h;
};

// The 16 features of the block with integer key (bx, by, bz) (edge E) seen by a camera with float rotation R
// (world <- camera, row-major) and translation t, from the range image rho (h x w, < 0 = invalid).
bool features(const Cam& K, const float* R, const float* t, const float* rho, float E, float tau, int64_t bx,
              int64_t by, int64_t bz, float* f) {
  // block centre, world -> camera (R transposed)
  const float d0 = ((float)bx + 0.5f) * E - t[0];
  const float d1 = ((float)by + 0.5f) * E - t[1];
  const float d2 = ((float)bz + 0.5f) * E - t[2];
  const float X = R[0] * d0 + R[3] * d1 + R[6] * d2;
  const float Y = R[1] * d0 + R[4] * d1 + R[7] * d2;
  const float Z = R[2] * d0 + R[5] * d1 + R[8] * d2;
  if (!(Z > 0.0f)) return false;
  const float pu = K.fx * X / Z + K.cx;
  const float pv = K.fy * Y / Z + K.cy;
  if (!(pu >= 0.0f && pu < (float)K.w && pv >= 0.0f && pv < (float)K.h)) return false;
  const int uc = (int)std::floor(pu + 0.5f);
  const int vc = (int)std::floor(pv + 0.5f);
  const float r = std::sqrt(X * X + Y * Y + Z * Z);
  // sample spacing: half the block's projected half-width, in whole pixels, within [1, 16]
  const float half_width_px = K.fx * (0.5f * E) / Z;
  int step = (int)std::floor(0.5f * half_width_px);
  step = step < 1 ? 1 : (step > 16 ? 16 : step);

  float g[5][5];  // g[row j][column i]
  for (int j = 0; j < 5; ++j)
    for (int i = 0; i < 5; ++i) {
      const int u = uc + (i - 2) * step, v = vc + (j - 2) * step;
      const bool inside = u >= 0 && u < K.w && v >= 0 && v < K.h;
      g[j][i] = inside ? rho[(size_t)v * K.w + u] : -1.0f;
    }
  // statistics of the present samples, visited row by row
  int cnt = 0;
  float s1 = 0.0f, s2 = 0.0f, lo = 0.0f, hi = 0.0f;
  for (int j = 0; j < 5; ++j)
    for (int i = 0; i < 5; ++i) {
      const float x = g[j][i];
      if (!(x >= 0.0f)) continue;
      if (cnt == 0) {
        lo = x;
        hi = x;
      } else {
        if (x < lo) lo = x;
        if (x > hi) hi = x;
      }
      s1 = s1 + x;
      s2 = s2 + x * x;
      cnt = cnt + 1;
    }
  float mean = 0.0f, sd = 0.0f;
  if (cnt > 0) {
    mean = s1 / (float)cnt;
    const float var = s2 / (float)cnt - mean * mean;
    if (var > 0.0f) sd = std::sqrt(var);
  }
  // central differences through the centre sample, per metre of lateral offset
  const float metres_per_step = r / K.fx * (float)step;
  float su = 0.0f, sv = 0.0f;
  if (g[2][1] >= 0.0f && g[2][3] >= 0.0f) su = (g[2][3] - g[2][1]) / (2.0f * metres_per_step);
  if (g[1][2] >= 0.0f && g[3][2] >= 0.0f) sv = (g[3][2] - g[1][2]) / (2.0f * metres_per_step);
  // mean absolute second difference along rows
  float curv = 0.0f;
  int ncurv = 0;
  for (int j = 0; j < 5; ++j)
    for (int i = 1; i <= 3; ++i) {
      const float a = g[j][i - 1], b = g[j][i], c = g[j][i + 1];
      if (!(a >= 0.0f && b >= 0.0f && c >= 0.0f)) continue;
      const float sd2 = a - 2.0f * b + c;
      curv = curv + std::fabs(sd2);
      ncurv = ncurv + 1;
    }
  if (ncurv > 0) curv = curv / (float)ncurv;
  const float ou = pu / (float)K.w - 0.5f, ov = pv / (float)K.h - 0.5f;
  // soft sign s(x) = x / (1 + |x|) bounds the unbounded ratios
  auto soft = [](float x) { return x / (1.0f + std::fabs(x)); };
  f[0] = r;
  f[1] = soft(cnt > 0 ? (mean - r) / tau : 0.0f);
  f[2] = soft(sd / tau);
  f[3] = soft(cnt > 0 ? (hi - lo) / E : 0.0f);
  f[4] = (float)cnt / 25.0f;
  f[5] = E / r;
  f[6] = soft(std::fabs(su));
  f[7] = soft(std::fabs(sv));
  f[8] = soft(curv / E);
  f[9] = 2.0f * std::fabs(ou);
  f[10] = 2.0f * std::fabs(ov);
  f[11] = Z / r;
  f[12] = 1.0f / r;
  f[13] = 0.0f;
  f[14] = tau / E;
  f[15] = 1.0f;
  for (int q = 0; q < kIn; ++q) f[q] = round_bf16(f[q]);
  return true;
}

// The 16 features of a new block of a LiDAR scan, from the moments of the scan's end points that fall inside it.
// Each end point's position in the block is quantised to q in [0, 1024)^3 (units of E / 1024); mom holds
// n, sum q_x, sum q_y, sum q_z, sum q_x^2, sum q_y^2, sum q_z^2, sum q_x q_y, sum q_x q_z, sum q_y q_z. T: the scan's
// pose (world <- sensor, row-major 4 x 4, double). The block centre relative to the sensor is formed in double (the
// pose's precision) and converted to float; everything after runs in float, like the camera features.
void lidar_features(const uint64_t* mom, const double* T, float E, float tau, int64_t bx, int64_t by, int64_t bz,
                    float* f) {
  const double Ed = (double)E;
  const float c0 = (float)(((double)bx + 0.5) * Ed - T[3]);
  const float c1 = (float)(((double)by + 0.5) * Ed - T[7]);
  const float c2 = (float)(((double)bz + 0.5) * Ed - T[11]);
  // unit direction u from the sensor to the block centre, and its distance
  const float r = std::sqrt(c0 * c0 + c1 * c1 + c2 * c2);
  const float u[3] = {c0 / r, c1 / r, c2 / r};
  const uint64_t cnt = mom[0];
  float along = 0.0f, thick2 = 0.0f, total = 0.0f, czz = 0.0f, lateral_off = 0.0f;
  if (cnt > 0) {
    const float nf = (float)cnt;
    float mean[3], off[3];
    for (int a = 0; a < 3; ++a) {
      mean[a] = (float)mom[1 + a] / nf;
      off[a] = (mean[a] + 0.5f) / 1024.0f - 0.5f;  // centroid relative to the block centre, block units
    }
    // covariance of the end points, block units squared
    const float cxx = ((float)mom[4] / nf - mean[0] * mean[0]) / 1048576.0f;
    const float cyy = ((float)mom[5] / nf - mean[1] * mean[1]) / 1048576.0f;
    czz = ((float)mom[6] / nf - mean[2] * mean[2]) / 1048576.0f;
    const float cxy = ((float)mom[7] / nf - mean[0] * mean[1]) / 1048576.0f;
    const float cxz = ((float)mom[8] / nf - mean[0] * mean[2]) / 1048576.0f;
    const float cyz = ((float)mom[9] / nf - mean[1] * mean[2]) / 1048576.0f;
    along = off[0] * u[0] + off[1] * u[1] + off[2] * u[2];
    const float cu0 = cxx * u[0] + cxy * u[1] + cxz * u[2];
    const float cu1 = cxy * u[0] + cyy * u[1] + cyz * u[2];
    const float cu2 = cxz * u[0] + cyz * u[1] + czz * u[2];
    thick2 = u[0] * cu0 + u[1] * cu1 + u[2] * cu2;  // spread along the viewing direction
    total = cxx + cyy + czz;
    const float l0 = off[0] - along * u[0], l1 = off[1] - along * u[1], l2 = off[2] - along * u[2];
    lateral_off = std::sqrt(l0 * l0 + l1 * l1 + l2 * l2);
  }
  const float lat2 = total - thick2;
  auto soft = [](float x) { return x / (1.0f + std::fabs(x)); };
  f[0] = r;
  f[1] = soft(along * E / tau);
  f[2] = soft(std::sqrt(thick2 > 0.0f ? thick2 : 0.0f) * E / tau);
  f[3] = std::sqrt(lat2 > 0.0f ? lat2 : 0.0f);
  f[4] = soft((float)cnt / 16.0f);
  f[5] = E / r;
  f[6] = std::sqrt(czz > 0.0f ? czz : 0.0f);
  f[7] = lateral_off;
  f[8] = cnt > 0 ? 1.0f : 0.0f;
  f[9] = std::fabs(u[2]);
  f[10] = u[2];
  f[11] = std::sqrt(total > 0.0f ? total : 0.0f);
  f[12] = 1.0f / r;
  f[13] = 1.0f;
  f[14] = tau / E;
  f[15] = 1.0f;
  for (int q = 0; q < kIn; ++q) f[q] = round_bf16(f[q]);
}

// logits of one sample; x already BF16 values; w packed W1[16][64], b1, W2[64][64], b2, W3[64][3], b3 as BF16 bits
void forward(const uint16_t* w, const float* x, float* logits) {
  const uint16_t* W1 = w;
  const uint16_t* b1 = W1 + kIn * kHid;
  const uint16_t* W2 = b1 + kHid;
  const uint16_t* b2 = W2 + kHid * kHid;
  const uint16_t* W3 = b2 + kHid;
  const uint16_t* b3 = W3 + kHid * kOut;
  float h1[kHid], h2[kHid];
  for (int j = 0; j < kHid; ++j) {
    float s = from_bf16(b1[j]);
    for (int k = 0; k < kIn; ++k) s = s + x[k] * from_bf16(W1[k * kHid + j]);
    h1[j] = round_bf16(gelu(s));
  }
  for (int j = 0; j < kHid; ++j) {
    float s = from_bf16(b2[j]);
    for (int k = 0; k < kHid; ++k) s = s + h1[k] * from_bf16(W2[k * kHid + j]);
    h2[j] = round_bf16(gelu(s));
  }
  for (int j = 0; j < kOut; ++j) {
    float s = from_bf16(b3[j]);
    for (int k = 0; k < kHid; ++k) s = s + h2[k] * from_bf16(W3[k * kOut + j]);
    logits[j] = s;
  }
}

int first_argmax(const float* z) {
  int best = 0;
  for (int j = 1; j < kOut; ++j)
    if (z[j] > z[best]) best = j;
  return best;
}

}  // namespace

extern "C" {

struct orc_pinhole {  // same layout as in mrh_oracle.cpp
  float fx, fy, cx, cy;
  int width, height;
  float min_depth, max_depth;
};

float orc_bf16_round(float x) { return round_bf16(x); }
float orc_exp_cw(float x) { return exp_cw(x); }
float orc_erf_as(float x) { return erf_as(x); }
float orc_gelu(float x) { return gelu(x); }

void orc_mlp_forward(const uint16_t* w, const float* x, int64_t n, float* logits) {
  for (int64_t i = 0; i < n; ++i) {
    float xi[kIn];
    for (int k = 0; k < kIn; ++k) xi[k] = round_bf16(x[i * kIn + k]);
    forward(w, xi, logits + i * kOut);
  }
}

// Features of one block and the predicted level (-1 when the block does not project into the image; level unset
// when w is null). R, t: float pose (world <- camera). Returns 1 if the features exist.
int orc_block_features(const orc_pinhole* K, const float* R, const float* t, const float* rho, float E, float tau,
                       int64_t bx, int64_t by, int64_t bz, const uint16_t* w, int n_levels, float* f, int* level) {
  Cam c{K->fx, K->fy, K->cx, K->cy, K->width, K->height};
  if (level) *level = -1;
  if (!features(c, R, t, rho, E, tau, bx, by, bz, f)) return 0;
  if (w && level) {
    float z[kOut];
    forward(w, f, z);
    int l = first_argmax(z);
    *level = l < n_levels - 1 ? l : n_levels - 1;
  }
  return 1;
}

// Features of one new block of a LiDAR scan from its end-point moments (10 values, see lidar_features) and the
// predicted level (level unset when w is null). T_ws: the scan pose, double, row-major 4 x 4.
void orc_lidar_block_features(const uint64_t* mom, const double* T_ws, float E, float tau, int64_t bx, int64_t by,
                              int64_t bz, const uint16_t* w, int n_levels, float* f, int* level) {
  lidar_features(mom, T_ws, E, tau, bx, by, bz, f);
  if (w && level) {
    float z[kOut];
    forward(w, f, z);
    int l = first_argmax(z);
    *level = l < n_levels - 1 ? l : n_levels - 1;
  }
}

}  // extern "C"
