// Contrast quadtree of an RGB image (the rendering branch, Sec. 3.5, Eq. 10, Algorithm 1).
//
// A node's contrast is the Rec. 601 luma weights applied to the per-channel mean squared deviation of its pixels from
// their mean colour, in byte units. Per channel, with n pixels, sum S1 and sum of squares S2, that mean is
// (n S2 - S1^2) / n^2 with an exact integer numerator N. A node splits when l0 N0 + l1 N1 + l2 N2 (double, in that
// order), n^2 times its contrast, exceeds threshold n n, so every implementation takes the same decisions, and no
// division runs on the GPU's slow double-precision path. A node whose contrast exceeds the threshold and
// whose larger side exceeds the minimum size splits at its midpoints (rounded down) into its non-empty quarters.
//
// The B300 form of Algorithm 1's breadth-first loop: the sums of any rectangle come from integral images of the bytes
// and of their squares (64-bit, built once per image), so a node's contrast is 24 loads instead of a reduction over its
// pixels. The top levels run as one launch each over the previous level's node list (every launch reads its node count
// from device memory, so the whole tree is queued without a host round trip); once nodes are at most 64 pixels on a
// side, one launch expands every remaining subtree, one CTA per subtree with its level lists in shared memory.
#include <cuda_runtime.h>

#include <cstdint>

#include "mrh_internal.cuh"

namespace mrh {
namespace {

struct QtNode {
  int x, y, w, h;
};

struct QtArgs {
  const uint8_t* rgb;
  int width, height;
  double threshold;
  int min_size;
  unsigned long long* ii;  // 6 planes of (height + 1) x (width + 1): sums of R, G, B, then of their squares
  QtNode* queue[2];
  uint32_t* count;         // count[l]: nodes of level l
  int32_t* leaves;
  uint64_t cap;
  unsigned long long* n_leaves;
};

// row pass: one warp per row, inclusive prefix of each plane along x (column 0 and row 0 stay zero)
__global__ void __launch_bounds__(256) k_qt_rows(QtArgs a) {
  const int lane = threadIdx.x & 31;
  const int W = a.width, P = a.width + 1;
  const size_t plane = (size_t)(a.height + 1) * P;
  for (int y = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; y <= a.height; y += (gridDim.x * blockDim.x) >> 5) {
    unsigned long long run[6] = {0, 0, 0, 0, 0, 0};
    if (lane == 0)
      for (int k = 0; k < 6; ++k) a.ii[k * plane + (size_t)y * P] = 0;
    for (int x0 = 0; x0 < W; x0 += 32) {
      const int x = x0 + lane;
      unsigned long long v[6] = {0, 0, 0, 0, 0, 0};
      if (y > 0 && x < W) {
        const uint8_t* px = a.rgb + 3 * ((size_t)(y - 1) * W + x);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          v[c] = px[c];
          v[3 + c] = (unsigned long long)px[c] * px[c];
        }
      }
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        for (int d = 1; d < 32; d <<= 1) {
          const unsigned long long t = __shfl_up_sync(~0u, v[k], d);
          if (lane >= d) v[k] += t;
        }
        v[k] += run[k];
        if (x < W) a.ii[k * plane + (size_t)y * P + x + 1] = v[k];
        run[k] = __shfl_sync(~0u, v[k], 31);
      }
    }
  }
}

// column pass, in kQtSeg segments of rows per (plane, column) so that enough threads run: first each segment's sum,
// then each segment scans its rows starting from the sum of the segments above it (loads coalesced across columns)
constexpr int kQtSeg = 16;

__global__ void __launch_bounds__(256) k_qt_col_sums(QtArgs a, unsigned long long* seg) {
  const int P = a.width + 1, rows = (a.height + kQtSeg - 1) / kQtSeg;
  const size_t plane = (size_t)(a.height + 1) * P;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 6 * P * kQtSeg; i += gridDim.x * blockDim.x) {
    const int x = i % P, k = (i / P) % 6, g = i / (6 * P);
    const unsigned long long* col = a.ii + k * plane + x;
    unsigned long long sum = 0;
    const int y1 = min(a.height, (g + 1) * rows);
    for (int y = 1 + g * rows; y <= y1; ++y) sum += col[(size_t)y * P];
    seg[i] = sum;
  }
}

__global__ void __launch_bounds__(256) k_qt_cols(QtArgs a, const unsigned long long* seg) {
  const int P = a.width + 1, rows = (a.height + kQtSeg - 1) / kQtSeg;
  const size_t plane = (size_t)(a.height + 1) * P;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 6 * P * kQtSeg; i += gridDim.x * blockDim.x) {
    const int x = i % P, k = (i / P) % 6, g = i / (6 * P);
    unsigned long long run = 0;
    for (int h = 0; h < g; ++h) run += seg[(size_t)h * 6 * P + k * P + x];
    unsigned long long* col = a.ii + k * plane + x;
    const int y1 = min(a.height, (g + 1) * rows);
    for (int y = 1 + g * rows; y <= y1; ++y) {
      run += col[(size_t)y * P];
      col[(size_t)y * P] = run;
    }
  }
}

__global__ void k_qt_root(QtArgs a, int levels) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    a.queue[0][0] = QtNode{0, 0, a.width, a.height};
    for (int l = 0; l <= levels; ++l) a.count[l] = l == 0 ? 1u : 0u;
    *a.n_leaves = 0;
  }
}

// n^2 times the node's contrast (n^2 in *n2)
__device__ inline double scaled_contrast(const QtArgs& a, const QtNode& q, double* n2) {
  const int P = a.width + 1;
  const size_t plane = (size_t)(a.height + 1) * P;
  const size_t i00 = (size_t)q.y * P + q.x, i01 = i00 + q.w, i10 = (size_t)(q.y + q.h) * P + q.x, i11 = i10 + q.w;
  const long long n = (long long)q.w * q.h;
  const double luma[3] = {0.2989, 0.5870, 0.1140};
  double acc = 0.0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const unsigned long long* s1 = a.ii + c * plane;
    const unsigned long long* s2 = a.ii + (3 + c) * plane;
    const long long S1 = (long long)(s1[i11] - s1[i01] - s1[i10] + s1[i00]);
    const long long S2 = (long long)(s2[i11] - s2[i01] - s2[i10] + s2[i00]);
    acc = acc + luma[c] * (double)(n * S2 - S1 * S1);
  }
  *n2 = (double)n * (double)n;
  return acc;
}

// one level: every node either splits into its non-empty quarters (next level) or is a leaf
__global__ void __launch_bounds__(256) k_qt_level(QtArgs a, int level) {
  const uint32_t n = a.count[level];
  const QtNode* in = a.queue[level & 1];
  QtNode* out = a.queue[(level + 1) & 1];
  const int lane = threadIdx.x & 31;
  // warp-uniform trip count, so that the appends below can be aggregated over the warp
  for (uint32_t base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; base < n; base += gridDim.x * blockDim.x) {
    const uint32_t i = base + lane;
    QtNode q{0, 0, 0, 0};
    bool live = i < n, split = false;
    if (live) {
      q = in[i];
      const int size = q.w > q.h ? q.w : q.h;
      double n2 = 0.0;
      split = size > a.min_size && scaled_contrast(a, q, &n2) > a.threshold * n2;
    }
    const int hw = q.w / 2, hh = q.h / 2;
    const int kids = split ? (hw > 0 ? 2 : 1) * (hh > 0 ? 2 : 1) : 0;
    // children: one atomic per warp for the next level's list
    int incl = kids;
    for (int d = 1; d < 32; d <<= 1) {
      const int t = __shfl_up_sync(~0u, incl, d);
      if (lane >= d) incl += t;
    }
    uint32_t first = 0;
    if (lane == 31 && incl > 0) first = atomicAdd(&a.count[level + 1], (uint32_t)incl);
    first = __shfl_sync(~0u, first, 31) + (uint32_t)(incl - kids);
    if (split)
      for (int j = 0; j < 2; ++j)
        for (int r = 0; r < 2; ++r) {
          const int cw = r ? q.w - hw : hw, ch = j ? q.h - hh : hh;
          if (cw > 0 && ch > 0) out[first++] = QtNode{r ? q.x + hw : q.x, j ? q.y + hh : q.y, cw, ch};
        }
    // leaves: one atomic per warp
    const bool leaf = live && !split;
    const unsigned bal = __ballot_sync(~0u, leaf);
    unsigned long long lbase = 0;
    if (lane == 0 && bal) lbase = atomicAdd(a.n_leaves, (unsigned long long)__popc(bal));
    lbase = __shfl_sync(~0u, lbase, 0);
    if (leaf) {
      const unsigned long long slot = lbase + __popc(bal & ((1u << lane) - 1u));
      if (slot < a.cap) {
        a.leaves[4 * slot] = q.x;
        a.leaves[4 * slot + 1] = q.y;
        a.leaves[4 * slot + 2] = q.w;
        a.leaves[4 * slot + 3] = q.h;
      }
    }
  }
}

// The subtrees below level T, one CTA per level-T node: its nodes are at most kQtSubSide x kQtSubSide pixels, so no
// level of its subtree holds more than kQtSubSide^2 nodes (they are disjoint non-empty rectangles of its pixels). The
// CTA expands the subtree breadth-first with its two level lists in shared memory (8-byte nodes) and a CTA barrier
// between levels, instead of one launch per level; decisions and children are those of k_qt_level.
constexpr int kQtSubSide = 64, kQtSubCap = kQtSubSide * kQtSubSide;

struct QtNode8 {
  uint16_t x, y, w, h;
};

__global__ void __launch_bounds__(256) k_qt_subtrees(QtArgs a, int level) {
  extern __shared__ QtNode8 s_list[];  // [2][kQtSubCap]
  __shared__ uint32_t s_n[2];
  const uint32_t n_roots = a.count[level];
  const QtNode* roots = a.queue[level & 1];
  const int lane = threadIdx.x & 31;
  for (uint32_t root = blockIdx.x; root < n_roots; root += gridDim.x) {
    if (threadIdx.x == 0) {
      const QtNode q = roots[root];
      s_list[0] = QtNode8{(uint16_t)q.x, (uint16_t)q.y, (uint16_t)q.w, (uint16_t)q.h};
      s_n[0] = 1;
      s_n[1] = 0;
    }
    __syncthreads();
    int cur = 0;
    for (;;) {
      const uint32_t n = s_n[cur];
      if (n == 0) break;  // the same value in every thread (read after a barrier)
      const QtNode8* in = s_list + cur * kQtSubCap;
      QtNode8* out = s_list + (cur ^ 1) * kQtSubCap;
      for (uint32_t base = threadIdx.x & ~31u; base < n; base += blockDim.x) {  // warp-uniform
        const uint32_t i = base + lane;
        QtNode q{0, 0, 0, 0};
        bool live = i < n, split = false;
        if (live) {
          const QtNode8 c = in[i];
          q = QtNode{c.x, c.y, c.w, c.h};
          const int size = q.w > q.h ? q.w : q.h;
          double n2 = 0.0;
          split = size > a.min_size && scaled_contrast(a, q, &n2) > a.threshold * n2;
        }
        const int hw = q.w / 2, hh = q.h / 2;
        const int kids = split ? (hw > 0 ? 2 : 1) * (hh > 0 ? 2 : 1) : 0;
        int incl = kids;
        for (int d = 1; d < 32; d <<= 1) {
          const int t = __shfl_up_sync(~0u, incl, d);
          if (lane >= d) incl += t;
        }
        uint32_t first = 0;
        if (lane == 31 && incl > 0) first = atomicAdd(&s_n[cur ^ 1], (uint32_t)incl);
        first = __shfl_sync(~0u, first, 31) + (uint32_t)(incl - kids);
        if (split)
          for (int j = 0; j < 2; ++j)
            for (int r = 0; r < 2; ++r) {
              const int cw = r ? q.w - hw : hw, ch = j ? q.h - hh : hh;
              if (cw > 0 && ch > 0) {
                if (first < (uint32_t)kQtSubCap)
                  out[first] = QtNode8{(uint16_t)(r ? q.x + hw : q.x), (uint16_t)(j ? q.y + hh : q.y), (uint16_t)cw,
                                       (uint16_t)ch};
                ++first;
              }
            }
        const bool leaf = live && !split;
        const unsigned bal = __ballot_sync(~0u, leaf);
        unsigned long long lbase = 0;
        if (lane == 0 && bal) lbase = atomicAdd(a.n_leaves, (unsigned long long)__popc(bal));
        lbase = __shfl_sync(~0u, lbase, 0);
        if (leaf) {
          const unsigned long long slot = lbase + __popc(bal & ((1u << lane) - 1u));
          if (slot < a.cap) {
            a.leaves[4 * slot] = q.x;
            a.leaves[4 * slot + 1] = q.y;
            a.leaves[4 * slot + 2] = q.w;
            a.leaves[4 * slot + 3] = q.h;
          }
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) s_n[cur] = 0;
      cur ^= 1;
      __syncthreads();
    }
  }
}

}  // namespace

size_t quadtree_scratch_bytes(int width, int height) {
  const size_t plane = (size_t)(height + 1) * (width + 1);
  return 6 * plane * 8 + 2 * (size_t)width * height * sizeof(QtNode) + 64 * 4 + 8 +
         8ull * 6 * (width + 1) * kQtSeg;
}

cudaError_t launch_quadtree(const uint8_t* rgb, int width, int height, double threshold, int min_size,
                            int32_t* leaves, uint64_t cap, void* scratch, unsigned long long** n_leaves_dev,
                            cudaStream_t s, int sms) {
  QtArgs a{};
  a.rgb = rgb;
  a.width = width;
  a.height = height;
  a.threshold = threshold;
  a.min_size = min_size;
  uint8_t* p = (uint8_t*)scratch;
  const size_t plane = (size_t)(height + 1) * (width + 1);
  a.ii = (unsigned long long*)p;
  p += 6 * plane * 8;
  a.queue[0] = (QtNode*)p;
  p += (size_t)width * height * sizeof(QtNode);
  a.queue[1] = (QtNode*)p;
  p += (size_t)width * height * sizeof(QtNode);
  a.count = (uint32_t*)p;
  p += 64 * 4;
  a.n_leaves = (unsigned long long*)p;
  p += 8;
  unsigned long long* seg = (unsigned long long*)p;
  a.leaves = leaves;
  a.cap = cap;
  // a node's larger side halves (rounded up) per level, so the tree has at most this many levels below the root
  int levels = 0;
  for (int side = width > height ? width : height; side > 1; side = (side + 1) / 2) ++levels;
  k_qt_rows<<<sms * 4, 256, 0, s>>>(a);
  const int col_threads = 6 * (width + 1) * kQtSeg;
  k_qt_col_sums<<<(col_threads + 255) / 256, 256, 0, s>>>(a, seg);
  k_qt_cols<<<(col_threads + 255) / 256, 256, 0, s>>>(a, seg);
  k_qt_root<<<1, 32, 0, s>>>(a, levels + 1);
  // one launch per level while nodes are larger than kQtSubSide on a side, then every remaining subtree in one launch
  int top = 0;
  for (int side = width > height ? width : height; side > kQtSubSide; side = (side + 1) / 2) ++top;
  if (top > levels || width > 65535 || height > 65535) top = levels + 1;
  for (int l = 0; l < top; ++l) k_qt_level<<<sms * 2, 256, 0, s>>>(a, l);
  if (top <= levels) {
    const int smem = 2 * kQtSubCap * (int)sizeof(QtNode8);
    cudaError_t e = cudaFuncSetAttribute(k_qt_subtrees, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k_qt_subtrees<<<sms * 3, 256, smem, s>>>(a, top);
  }
  *n_leaves_dev = a.n_leaves;
  return cudaGetLastError();
}

}  // namespace mrh
