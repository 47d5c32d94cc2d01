// Raycast of the adaptive grid (the rendering branch of Fig. 2): one thread per pixel.
//
// The ray marches from min_depth to max_depth (as z-depth). A sample whose block is not allocated jumps to the
// block's exit face: empty space costs one hash probe per block instead of one per voxel. Inside an allocated block
// of level l the ray advances min(v_l, tau / 2). The field at a sample is the trilinear interpolation over the 8
// nearest voxel centres of that level's grid; a corner in a neighbouring block reads that block's voxel containing
// the corner centre, whatever its level, so coarse and fine blocks blend across resolution boundaries. A sample is
// valid only when all 8 corners are observed (W > 0). At the first valid + -> - sign change the linear root is taken,
// evaluated once more, and one secant step refines it. Output is z-depth, 0 where nothing was hit.
//
// Every step follows the oracle's float operation order (this file is compiled without multiply-add contraction),
// so depths agree with the oracle to rounding and hit/miss decisions agree except at exact ties.
#include <cuda_fp16.h>

#include "mrh_internal.cuh"

namespace mrh {
namespace {

// Small per-thread cache of the last looked-up blocks: the 8 corners of a sample almost always fall in 1-2 blocks.
struct BlockCache {
  static constexpr int N = 4;
  unsigned long long key[N];
  uint32_t val[N];
  int next;
  __device__ BlockCache() : next(0) {
#pragma unroll
    for (int i = 0; i < N; ++i) key[i] = kEmptyKey;
  }
  // heap value of block (x, y, z), or kValPending when the block is not allocated or has no storage
  __device__ inline uint32_t get(const MapDev& m, long long x, long long y, long long z) {
    if (!key_ok(x, y, z)) return kValPending;
    unsigned long long k = pack_key(x, y, z);
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (key[i] == k) return val[i];
    int s = lookup_slot(m.slots, m.slot_mask, k);
    uint32_t v = s >= 0 ? m.slots[s].val : kValPending;
    key[next] = k;
    val[next] = v;
    next = (next + 1) % N;
    return v;
  }
};

__device__ inline float read_D(const MapDev& m, const uint8_t* blk, int i) {
  return m.fp16 ? __half2float(reinterpret_cast<const __half*>(blk)[i]) : reinterpret_cast<const float*>(blk)[i];
}

// trilinear field at x on the level-l grid; false when a corner is unallocated or unobserved
__device__ bool field(const MapDev& m, BlockCache& bc, const float x[3], int l, float* out) {
  const float inv = 1.0f / m.v[l];
  long long j0[3];
  float fr[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float g = x[a] * inv - 0.5f;
    float fl = floorf(g);
    j0[a] = (long long)fl;
    fr[a] = g - fl;
  }
  const int nl = kFineDim >> l;
  float acc = 0.0f;
  for (int k = 0; k < 8; ++k) {
    const int ax = k & 1, ay = (k >> 1) & 1, az = k >> 2;
    const long long j[3] = {j0[0] + ax, j0[1] + ay, j0[2] + az};
    const long long bk[3] = {floor_div(j[0], nl), floor_div(j[1], nl), floor_div(j[2], nl)};
    const uint32_t val = bc.get(m, bk[0], bk[1], bk[2]);
    if (val == kValPending) return false;
    const int lb = (int)((val >> 28) & 3u);
    const int nb = kFineDim >> lb;
    const uint8_t* blk = m.heap[lb] + (size_t)(val & kPtrMask) * m.block_bytes[lb];
    int idx;
    if (lb == l) {
      idx = (int)(j[0] - bk[0] * nl) + nl * ((int)(j[1] - bk[1] * nl) + nl * (int)(j[2] - bk[2] * nl));
    } else {
      long long cf[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) cf[a] = l == 0 ? j[a] : j[a] * (1LL << l) + (1LL << (l - 1));
      idx = (int)(floor_div(cf[0], 1LL << lb) - bk[0] * nb) +
            nb * ((int)(floor_div(cf[1], 1LL << lb) - bk[1] * nb) + nb * (int)(floor_div(cf[2], 1LL << lb) - bk[2] * nb));
    }
    const int nvb = nb * nb * nb;
    const float w = reinterpret_cast<const float*>(blk + off_W(nvb, m.fp16, m.color))[idx];
    if (!(w > 0.0f)) return false;
    const float wx = ax ? fr[0] : 1.0f - fr[0];
    const float wy = ay ? fr[1] : 1.0f - fr[1];
    const float wz = az ? fr[2] : 1.0f - fr[2];
    acc = acc + wx * wy * wz * read_D(m, blk, idx);
  }
  *out = acc;
  return true;
}

// sample at t: false when the sample's block is not allocated
__device__ inline bool sample(const MapDev& m, BlockCache& bc, const float o[3], const float r[3], float t, float invE,
                              int* level, bool* valid, float* F) {
  const float x[3] = {o[0] + t * r[0], o[1] + t * r[1], o[2] + t * r[2]};
  const uint32_t val = bc.get(m, (long long)floorf(x[0] * invE), (long long)floorf(x[1] * invE),
                              (long long)floorf(x[2] * invE));
  if (val == kValPending) return false;
  *level = (int)((val >> 28) & 3u);
  *valid = field(m, bc, x, *level, F);
  return true;
}

__global__ void __launch_bounds__(128) k_raycast(MapDev m, CamArgs c, float* __restrict__ out) {
  // 16 x 8 pixel tiles: neighbouring threads march through the same blocks
  const int u = blockIdx.x * 16 + (threadIdx.x & 15);
  const int v = blockIdx.y * 8 + (threadIdx.x >> 4);
  if (u >= c.width || v >= c.height) return;
  BlockCache bc;
  const float qx = ((float)u - c.cx) / c.fx, qy = ((float)v - c.cy) / c.fy;
  const float nq = sqrtf(qx * qx + qy * qy + 1.0f);
  const float rc[3] = {qx / nq, qy / nq, 1.0f / nq};
  float r[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) r[a] = c.R[3 * a + 0] * rc[0] + c.R[3 * a + 1] * rc[1] + c.R[3 * a + 2] * rc[2];
  const float o[3] = {c.t[0], c.t[1], c.t[2]};
  const float E = m.E, invE = 1.0f / E, half_tau = m.tau * 0.5f;
  float t = c.min_depth * nq;
  const float t_far = c.max_depth * nq;
  bool have_prev = false;
  float t_prev = 0.0f, F_prev = 0.0f, hit = 0.0f;
  for (int it = 0; it < kRaycastMaxIter && t <= t_far; ++it) {
    int l = 0;
    bool valid = false;
    float F = 0.0f;
    if (!sample(m, bc, o, r, t, invE, &l, &valid, &F)) {
      // jump to the exit face of the empty block
      const float x[3] = {o[0] + t * r[0], o[1] + t * r[1], o[2] + t * r[2]};
      float t_exit = t_far + 1.0f;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (r[a] == 0.0f) continue;
        const float bf = floorf(x[a] * invE);
        const float face = (r[a] > 0.0f ? bf + 1.0f : bf) * E;
        const float ta = (face - o[a]) / r[a];
        if (ta < t_exit) t_exit = ta;
      }
      const float step_min = t + 1e-4f * E;
      const float tn = t_exit + 1e-4f * E;
      t = tn > step_min ? tn : step_min;
      have_prev = false;
      continue;
    }
    if (valid && have_prev && F_prev > 0.0f && !(F > 0.0f)) {
      float ta = t_prev, Fa = F_prev, tb = t, Fb = F;
      float ts = ta + (tb - ta) * (Fa / (Fa - Fb));
      int l2 = 0;
      bool v2 = false;
      float F2 = 0.0f;
      if (sample(m, bc, o, r, ts, invE, &l2, &v2, &F2) && v2) {
        if (F2 > 0.0f) { ta = ts; Fa = F2; } else { tb = ts; Fb = F2; }
        if (Fa - Fb > 0.0f) ts = ta + (tb - ta) * (Fa / (Fa - Fb));
      }
      hit = ts * rc[2];
      break;
    }
    have_prev = valid;
    if (valid) {
      t_prev = t;
      F_prev = F;
    }
    const float s = m.v[l] < half_tau ? m.v[l] : half_tau;
    t = t + s;
  }
  out[(size_t)v * c.width + u] = hit;
}

}  // namespace

void launch_raycast(const MapDev& m, const CamArgs& c, float* out, cudaStream_t s) {
  dim3 grid((c.width + 15) / 16, (c.height + 7) / 8);
  k_raycast<<<grid, 128, 0, s>>>(m, c, out);
}

}  // namespace mrh
