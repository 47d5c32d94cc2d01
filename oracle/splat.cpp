// CPU oracle (test infrastructure) for the Gaussian-splat rasteriser of the rendering branch (Sec. 3.5): projection
// of each 3D Gaussian to the image (Eq. 7) and front-to-back alpha blending of the projected Gaussians (Eqs. 8, 9).
// Brute force: every pixel visits every projected Gaussian in depth order. Shares nothing with the CUDA library.
//
// Readings:
//  - The pose is camera-to-world (R_wc, t); a Gaussian's camera-frame mean is R_wc^T (mu - t), its depth the camera
//    z. Gaussians with z outside [min_depth, max_depth] or a projected covariance that is not positive definite are
//    not drawn. The pixel (u, v) sits at image coordinates (u, v), the convention of the rest of the library.
//  - Sigma_I = J R Sigma_W R^T J^T with R = R_wc^T and J the Jacobian of the pinhole projection at the camera-frame
//    mean; only its 2 x 2 image part is formed.
//  - Support: a Gaussian reaches a pixel when the squared Mahalanobis distance q <= 9 and the pixel lies within three
//    standard deviations along each image axis (|du| <= 3 sqrt(Sigma_uu), |dv| <= 3 sqrt(Sigma_vv); implied by q <= 9
//    in exact arithmetic, stated so that the decision does not depend on rounding). The paper gives no cut-off;
//    three standard deviations is the usual one of tile rasterisers.
//  - Order: increasing camera z, ties by Gaussian index. Eq. 8 is evaluated as written: colour = sum of
//    C_m a_m G_m times the product of (1 - a_l G_l) over the Gaussians in front; the remaining product is returned
//    as the pixel's transmittance. No opacity clamp, no early stop.
//  - Precision: the projection, the support test and the depth order are computed in float with a fixed operation
//    order (they decide which Gaussians reach a pixel and in which order, so the CUDA kernels take the same float
//    decisions); G = exp(-q/2) and the blend are accumulated in double.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <vector>

namespace {

struct Camera {
  float fx, fy, cx, cy, min_depth, max_depth;
  float R[9];  // world <- camera rotation, row-major
  float t[3];
};

struct Projected {
  float z, mu_u, mu_v;
  float cov[3];    // Sigma_I: uu, uv, vv
  float conic[3];  // Sigma_I^-1: uu, uv, vv
  float ru, rv;    // three standard deviations along u and v
};

Camera camera(const float* K6, const double* T) {
  Camera c;
  c.fx = K6[0];
  c.fy = K6[1];
  c.cx = K6[2];
  c.cy = K6[3];
  c.min_depth = K6[4];
  c.max_depth = K6[5];
  for (int r = 0; r < 3; ++r) {
    for (int q = 0; q < 3; ++q) c.R[3 * r + q] = (float)T[4 * r + q];
    c.t[r] = (float)T[4 * r + 3];
  }
  return c;
}

// Eq. 7 for one Gaussian (mean: 3 floats; cov: Sigma_W as xx, xy, xz, yy, yz, zz); false when it is not drawn
bool project(const Camera& c, const float* mean, const float* cov, Projected* p) {
  const float d0 = mean[0] - c.t[0], d1 = mean[1] - c.t[1], d2 = mean[2] - c.t[2];
  const float* R = c.R;
  const float x = R[0] * d0 + R[3] * d1 + R[6] * d2;
  const float y = R[1] * d0 + R[4] * d1 + R[7] * d2;
  const float z = R[2] * d0 + R[5] * d1 + R[8] * d2;
  if (!(z >= c.min_depth && z <= c.max_depth)) return false;
  const float iz = 1.0f / z;
  const float xz = x * iz, yz = y * iz;
  p->z = z;
  p->mu_u = c.fx * xz + c.cx;
  p->mu_v = c.fy * yz + c.cy;
  // J (2 x 3): [fx/z, 0, -fx x/z^2; 0, fy/z, -fy y/z^2]; camera-from-world rotation R^T, element (b, a) = R[3a + b]
  const float j00 = c.fx * iz, j02 = -(j00 * xz), j11 = c.fy * iz, j12 = -(j11 * yz);
  float M0[3], M1[3];  // rows of J R^T
  for (int a = 0; a < 3; ++a) {
    M0[a] = j00 * R[3 * a] + j02 * R[3 * a + 2];
    M1[a] = j11 * R[3 * a + 1] + j12 * R[3 * a + 2];
  }
  const float S[3][3] = {{cov[0], cov[1], cov[2]}, {cov[1], cov[3], cov[4]}, {cov[2], cov[4], cov[5]}};
  float V0[3], V1[3];  // Sigma_W M0^T, Sigma_W M1^T
  for (int a = 0; a < 3; ++a) {
    V0[a] = S[a][0] * M0[0] + S[a][1] * M0[1] + S[a][2] * M0[2];
    V1[a] = S[a][0] * M1[0] + S[a][1] * M1[1] + S[a][2] * M1[2];
  }
  const float suu = M0[0] * V0[0] + M0[1] * V0[1] + M0[2] * V0[2];
  const float suv = M1[0] * V0[0] + M1[1] * V0[1] + M1[2] * V0[2];
  const float svv = M1[0] * V1[0] + M1[1] * V1[1] + M1[2] * V1[2];
  const float det = suu * svv - suv * suv;
  if (!(det > 0.0f) || !(suu > 0.0f)) return false;
  p->cov[0] = suu;
  p->cov[1] = suv;
  p->cov[2] = svv;
  p->conic[0] = svv / det;
  p->conic[1] = -(suv / det);
  p->conic[2] = suu / det;
  p->ru = 3.0f * sqrtf(suu);
  p->rv = 3.0f * sqrtf(svv);
  return true;
}

// squared Mahalanobis distance of pixel (u, v), or -1 when the pixel is outside the support
float support_q(const Projected& p, int u, int v) {
  const float du = (float)u - p.mu_u, dv = (float)v - p.mu_v;
  if (!(fabsf(du) <= p.ru && fabsf(dv) <= p.rv)) return -1.0f;
  const float q = (p.conic[0] * (du * du) + (p.conic[1] + p.conic[1]) * (du * dv)) + p.conic[2] * (dv * dv);
  return q <= 9.0f ? q : -1.0f;
}

}  // namespace

extern "C" {

// Eq. 7 for one Gaussian (test hook). K6 = fx, fy, cx, cy, min_depth, max_depth; T = camera-to-world pose (4 x 4
// row-major). out = z, mu_u, mu_v, Sigma_uu, Sigma_uv, Sigma_vv, conic uu, uv, vv. Returns 1 when drawn, else 0.
int orc_splat_project(const float* mean, const float* cov, const float* K6, const double* T, float* out) {
  const Camera c = camera(K6, T);
  Projected p;
  if (!project(c, mean, cov, &p)) return 0;
  const float v[9] = {p.z, p.mu_u, p.mu_v, p.cov[0], p.cov[1], p.cov[2], p.conic[0], p.conic[1], p.conic[2]};
  std::copy(v, v + 9, out);
  return 1;
}

}  // extern "C"

namespace {

// the drawn Gaussians (projections and indices) in blending order: increasing z, ties by index
struct DepthOrder {
  std::vector<Projected> proj;
  std::vector<int64_t> ids;
  std::vector<size_t> order;
};

DepthOrder depth_order(const Camera& c, int64_t n, const float* means, const float* covs) {
  DepthOrder d;
  for (int64_t m = 0; m < n; ++m) {
    Projected p;
    if (project(c, means + 3 * m, covs + 6 * m, &p)) {
      d.proj.push_back(p);
      d.ids.push_back(m);
    }
  }
  d.order.resize(d.proj.size());
  std::iota(d.order.begin(), d.order.end(), (size_t)0);
  std::sort(d.order.begin(), d.order.end(), [&](size_t a, size_t b) {
    return d.proj[a].z < d.proj[b].z || (d.proj[a].z == d.proj[b].z && d.ids[a] < d.ids[b]);
  });
  return d;
}

// Eq. 8 at one pixel: colour sum and the remaining product of (1 - alpha G)
void blend_pixel(const DepthOrder& d, const float* opacity, const float* colors, int u, int v, double* C,
                 double* Tr) {
  C[0] = C[1] = C[2] = 0.0;
  *Tr = 1.0;
  for (size_t k : d.order) {
    const float q = support_q(d.proj[k], u, v);
    if (q < 0.0f) continue;
    const int64_t m = d.ids[k];
    const double w = (double)opacity[m] * std::exp(-0.5 * (double)q);  // alpha G, Eq. 9
    for (int ch = 0; ch < 3; ++ch) C[ch] += (double)colors[3 * m + ch] * w * *Tr;
    *Tr *= 1.0 - w;
  }
}

}  // namespace

extern "C" {

// Eqs. 7-9 for n Gaussians (means n x 3, covs n x 6, opacity n, colors n x 3) on a width x height image: colour
// (height x width x 3) and transmittance (height x width), both double. Returns the number of Gaussians drawn.
int64_t orc_splat_render(int64_t n, const float* means, const float* covs, const float* opacity, const float* colors,
                         const float* K6, const double* T, int width, int height, double* rgb, double* trans) {
  const DepthOrder d = depth_order(camera(K6, T), n, means, covs);
  for (int v = 0; v < height; ++v)
    for (int u = 0; u < width; ++u) {
      const int64_t px = (int64_t)v * width + u;
      blend_pixel(d, opacity, colors, u, v, rgb + 3 * px, trans + px);
    }
  return (int64_t)d.proj.size();
}

// the same at n_px listed pixels (uv: n_px x 2 int32, u then v): rgb n_px x 3, trans n_px
int64_t orc_splat_pixels(int64_t n, const float* means, const float* covs, const float* opacity, const float* colors,
                         const float* K6, const double* T, int64_t n_px, const int32_t* uv, double* rgb,
                         double* trans) {
  const DepthOrder d = depth_order(camera(K6, T), n, means, covs);
  for (int64_t i = 0; i < n_px; ++i) blend_pixel(d, opacity, colors, uv[2 * i], uv[2 * i + 1], rgb + 3 * i, trans + i);
  return (int64_t)d.proj.size();
}

}  // extern "C"
