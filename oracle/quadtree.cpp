// CPU oracle (test infrastructure) for the image-space quadtree of the rendering branch (Sec. 3.5, Eq. 10 contrast,
// Algorithm 1). Plain recursion over the nodes, every sum taken pixel by pixel; shares nothing with the CUDA library.
//
// Reading: RGB values are the image's bytes (0..255; the paper does not give the scale, and at its threshold of 0.1 a
// [0, 1] scale would leave a whole synthetic frame as one leaf). A node's contrast is the Rec. 601 luma weights applied
// to the per-channel mean of squared deviations from the node's mean colour. It is evaluated from exact integer sums:
// for a channel with n pixels, sum S1 and sum of squares S2, the mean squared deviation is (n S2 - S1^2) / n^2 with an
// exact integer numerator N. A node splits when n^2 times its contrast exceeds n^2 times the threshold, both in double:
// l0 N0 + l1 N1 + l2 N2 (in that order) against threshold n n, so that every implementation reaches the same split
// decisions without a division. A node whose contrast exceeds the threshold and whose larger
// side exceeds the minimum size splits at its midpoints (x0 + w/2, y0 + h/2, rounded down) into up to four children
// (empty ones dropped); otherwise it is a leaf.
#include <cstdint>
#include <vector>

namespace {

struct Leaf {
  int32_t x, y, w, h;
};

// n^2 times the contrast (and n^2 in *n2)
double scaled_contrast(const uint8_t* rgb, int width, int x0, int y0, int w, int h, double* n2) {
  const int64_t n = (int64_t)w * h;
  int64_t s1[3] = {0, 0, 0}, s2[3] = {0, 0, 0};
  for (int y = y0; y < y0 + h; ++y)
    for (int x = x0; x < x0 + w; ++x)
      for (int c = 0; c < 3; ++c) {
        const int64_t q = rgb[3 * ((int64_t)y * width + x) + c];
        s1[c] += q;
        s2[c] += q * q;
      }
  const double luma[3] = {0.2989, 0.5870, 0.1140};
  double acc = 0.0;
  for (int c = 0; c < 3; ++c) acc = acc + luma[c] * (double)(n * s2[c] - s1[c] * s1[c]);
  *n2 = (double)n * (double)n;
  return acc;
}

void split(const uint8_t* rgb, int width, int x0, int y0, int w, int h, double thr, int min_size,
           std::vector<Leaf>& out) {
  const int size = w > h ? w : h;
  double n2 = 0.0;
  if (size > min_size && scaled_contrast(rgb, width, x0, y0, w, h, &n2) > thr * n2) {
    const int hw = w / 2, hh = h / 2;
    const int xs[2] = {x0, x0 + hw}, ws[2] = {hw, w - hw};
    const int ys[2] = {y0, y0 + hh}, hs[2] = {hh, h - hh};
    for (int j = 0; j < 2; ++j)
      for (int i = 0; i < 2; ++i)
        if (ws[i] > 0 && hs[j] > 0) split(rgb, width, xs[i], ys[j], ws[i], hs[j], thr, min_size, out);
  } else {
    out.push_back(Leaf{x0, y0, w, h});
  }
}

}  // namespace

extern "C" {

// contrast of one rectangle (test hook)
double orc_qt_contrast(const uint8_t* rgb, int width, int x0, int y0, int w, int h) {
  double n2 = 0.0;
  const double c = scaled_contrast(rgb, width, x0, y0, w, h, &n2);
  return c / n2;
}

// leaves (x, y, w, h) of the image's quadtree, in depth-first order (top-left, top-right, bottom-left, bottom-right);
// returns the number of leaves, writes at most cap
int64_t orc_quadtree(const uint8_t* rgb, int width, int height, double threshold, int min_size, int32_t* out,
                     int64_t cap) {
  std::vector<Leaf> leaves;
  if (width > 0 && height > 0) split(rgb, width, 0, 0, width, height, threshold, min_size, leaves);
  for (int64_t i = 0; i < (int64_t)leaves.size() && i < cap; ++i) {
    out[4 * i] = leaves[i].x;
    out[4 * i + 1] = leaves[i].y;
    out[4 * i + 2] = leaves[i].w;
    out[4 * i + 3] = leaves[i].h;
  }
  return (int64_t)leaves.size();
}

}  // extern "C"
