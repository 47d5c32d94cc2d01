// Raycast of the adaptive grid (the rendering branch of Fig. 2): one thread per pixel.
//
// The ray marches from min_depth to max_depth (as z-depth). A sample in an empty brick (4 x 4 x 4 blocks, looked up
// in a small insert-only set filled when blocks are created) jumps to the brick's exit face; a sample in an
// unallocated block of a non-empty brick jumps to the block's exit face; so empty space costs one probe per 32 cm
// instead of one per voxel. Inside an allocated block of level l the field is the trilinear interpolation over the
// 8 nearest voxel centres of that level's grid; a corner in a neighbouring block reads that block's voxel containing
// the corner centre, whatever its level, so coarse and fine blocks blend across resolution boundaries. A sample is
// valid only when all 8 corners are observed (W > 0). The next sample lies min(v_l, tau / 2) ahead, or 0.75 F ahead
// when the sample is valid and F is larger (F <= tau underestimates the distance to the surface, so the step stays
// in front of it). At the first valid + -> - sign change the linear root is taken, evaluated once more, and one
// secant step refines it. Output is z-depth, 0 where nothing was hit.
//
// Every step follows the oracle's float operation order (this file is compiled without multiply-add contraction),
// so depths agree with the oracle to rounding and hit/miss decisions agree except at exact ties.
#include <cuda_fp16.h>

#include "mrh_internal.cuh"

namespace mrh {
namespace {

// Block coordinates fit in 32 bits (|key| < 2^20, voxel indices < 2^23), so all index math here is 32-bit: divisions
// by the power-of-two block side are arithmetic shifts (floor for negatives) and remainders are masks. (64-bit
// integer division and float -> int64 conversion run on the B300's small FP64 path and dominated an earlier
// version of this kernel.)
__device__ inline bool key_ok32(int x, int y, int z) {
  const int lim = (int)kKeyLimit;
  return x >= -lim && x <= lim && y >= -lim && y <= lim && z >= -lim && z <= lim;
}

// float -> int floor, out-of-range values map to an invalid key
__device__ inline int ifloor(float v) {
  const float f = floorf(v);
  return fabsf(f) < 1073741824.0f ? (int)f : 0x7FFFFFFF;
}

// Small per-thread cache of the last looked-up blocks: the 8 corners of a sample almost always fall in 1-2 blocks.
// Kept in registers (static indices only; replacement shifts the entries), never in local memory.
struct BlockCache {
  unsigned long long k0 = kEmptyKey, k1 = kEmptyKey, k2 = kEmptyKey, k3 = kEmptyKey;
  uint32_t v0 = 0, v1 = 0, v2 = 0, v3 = 0;
  // heap value of block (x, y, z), or kValPending when the block is not allocated or has no storage
  __device__ inline uint32_t get(const MapDev& m, int x, int y, int z) {
    if (!key_ok32(x, y, z)) return kValPending;
    const unsigned long long k = pack_key(x, y, z);
    if (k == k0) return v0;
    if (k == k1) return v1;
    if (k == k2) return v2;
    if (k == k3) return v3;
    const int s = lookup_slot(m.slots, m.slot_mask, k);
    const uint32_t v = s >= 0 ? m.slots[s].val : kValPending;
    k3 = k2; v3 = v2;
    k2 = k1; v2 = v1;
    k1 = k0; v1 = v0;
    k0 = k; v0 = v;
    return v;
  }
};

__device__ inline const uint8_t* block_ptr(const MapDev& m, uint32_t val) {
  const int lb = (int)((val >> 28) & 3u);
  return m.heap[lb] + (size_t)(val & kPtrMask) * m.block_bytes[lb];
}

__device__ inline float read_D(const MapDev& m, const uint8_t* blk, int i) {
  return m.fp16 ? __half2float(reinterpret_cast<const __half*>(blk)[i]) : reinterpret_cast<const float*>(blk)[i];
}
__device__ inline float read_W(const MapDev& m, const uint8_t* blk, int nv, int i) {
  return reinterpret_cast<const float*>(blk + off_W(nv, m.fp16, m.color))[i];
}

// Brick membership with a one-entry register cache.
struct BrickCache {
  unsigned long long key = kEmptyKey;
  bool present = false;
  __device__ inline bool get(const MapDev& m, int bx, int by, int bz) {
    if (!key_ok32(bx, by, bz)) return false;
    const unsigned long long k = pack_key(bx, by, bz);
    if (k == key) return present;
    const uint32_t h = hash_xyz(bx, by, bz, m.brick_mask);
    bool found = false;
    for (int p = 0; p < kMaxProbes; ++p) {
      const unsigned long long c = m.brick_keys[(h + (uint32_t)p) & m.brick_mask];
      if (c == k) {
        found = true;
        break;
      }
      if (c == kEmptyKey) break;
    }
    key = k;
    present = found;
    return found;
  }
};

// trilinear field at x on the level-l grid; false when a corner is unallocated or unobserved
__device__ bool field(const MapDev& m, BlockCache& bc, const float x[3], int l, float* out) {
  const float inv = m.inv_v[l];
  int j0[3];
  float fr[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float g = x[a] * inv - 0.5f;
    const float fl = floorf(g);
    j0[a] = (int)fl;
    fr[a] = g - fl;
  }
  const int sh = 3 - l, nl = 1 << sh, mask = nl - 1;
  float acc = 0.0f;
  const int b0[3] = {j0[0] >> sh, j0[1] >> sh, j0[2] >> sh};
  const int r0[3] = {j0[0] & mask, j0[1] & mask, j0[2] & mask};
  if (r0[0] < mask && r0[1] < mask && r0[2] < mask) {
    // all 8 corners inside one block
    const uint32_t val = bc.get(m, b0[0], b0[1], b0[2]);
    if (val == kValPending) return false;
    const int lb = (int)((val >> 28) & 3u);
    if (lb == l) {
      const uint8_t* blk = block_ptr(m, val);
      const int nv = nl * nl * nl;
      const int base = r0[0] + nl * (r0[1] + nl * r0[2]);
      for (int k = 0; k < 8; ++k) {
        const int ax = k & 1, ay = (k >> 1) & 1, az = k >> 2;
        const int idx = base + ax + nl * (ay + nl * az);
        if (!(read_W(m, blk, nv, idx) > 0.0f)) return false;
        const float wx = ax ? fr[0] : 1.0f - fr[0];
        const float wy = ay ? fr[1] : 1.0f - fr[1];
        const float wz = az ? fr[2] : 1.0f - fr[2];
        acc = acc + wx * wy * wz * read_D(m, blk, idx);
      }
      *out = acc;
      return true;
    }
  }
  for (int k = 0; k < 8; ++k) {
    const int ax = k & 1, ay = (k >> 1) & 1, az = k >> 2;
    const int j[3] = {j0[0] + ax, j0[1] + ay, j0[2] + az};
    const int bk[3] = {j[0] >> sh, j[1] >> sh, j[2] >> sh};
    const uint32_t val = bc.get(m, bk[0], bk[1], bk[2]);
    if (val == kValPending) return false;
    const int lb = (int)((val >> 28) & 3u);
    const int nb = kFineDim >> lb;
    const uint8_t* blk = block_ptr(m, val);
    int idx;
    if (lb == l) {
      idx = (j[0] & mask) + nl * ((j[1] & mask) + nl * (j[2] & mask));
    } else {
      // the finest-level cell holding the corner centre, then block bk's voxel (at its own level) containing it
      int c[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) c[a] = (l == 0 ? j[a] : (j[a] << l) + (1 << (l - 1))) >> lb;
      idx = (c[0] & (nb - 1)) + nb * ((c[1] & (nb - 1)) + nb * (c[2] & (nb - 1)));
    }
    if (!(read_W(m, blk, nb * nb * nb, idx) > 0.0f)) return false;
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
  const uint32_t val = bc.get(m, ifloor(x[0] * invE), ifloor(x[1] * invE), ifloor(x[2] * invE));
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
  BrickCache brc;
  const float qx = ((float)u - c.cx) / c.fx, qy = ((float)v - c.cy) / c.fy;
  const float nq = sqrtf(qx * qx + qy * qy + 1.0f);
  const float rc[3] = {qx / nq, qy / nq, 1.0f / nq};
  float r[3], inv_r[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    r[a] = c.R[3 * a + 0] * rc[0] + c.R[3 * a + 1] * rc[1] + c.R[3 * a + 2] * rc[2];
    inv_r[a] = r[a] != 0.0f ? 1.0f / r[a] : 0.0f;
  }
  const float o[3] = {c.t[0], c.t[1], c.t[2]};
  const float E = m.E, invE = 1.0f / E, half_tau = m.tau * 0.5f, eps = 1e-4f * E;
  float t = c.min_depth * nq;
  const float t_far = c.max_depth * nq;
  bool have_prev = false;
  float t_prev = 0.0f, F_prev = 0.0f, hit = 0.0f;
  for (int it = 0; it < kRaycastMaxIter && t <= t_far; ++it) {
    const float x[3] = {o[0] + t * r[0], o[1] + t * r[1], o[2] + t * r[2]};
    const int bk[3] = {ifloor(x[0] * invE), ifloor(x[1] * invE), ifloor(x[2] * invE)};
    const int br[3] = {bk[0] >> kBrickShift, bk[1] >> kBrickShift, bk[2] >> kBrickShift};
    const bool brick = brc.get(m, br[0], br[1], br[2]);
    const uint32_t val = brick ? bc.get(m, bk[0], bk[1], bk[2]) : kValPending;
    if (val == kValPending) {
      // jump to the exit face of the empty brick, or of the empty block
      const int span = brick ? 1 : (1 << kBrickShift);
      float t_exit = t_far + 1.0f;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (r[a] == 0.0f) continue;
        const int cell = brick ? bk[a] : br[a];
        const float face = (float)((r[a] > 0.0f ? cell + 1 : cell) * span) * E;
        const float ta = (face - o[a]) * inv_r[a];
        if (ta < t_exit) t_exit = ta;
      }
      const float step_min = t + eps;
      const float tn = t_exit + eps;
      t = tn > step_min ? tn : step_min;
      have_prev = false;
      continue;
    }
    const int l = (int)((val >> 28) & 3u);
    float F = 0.0f;
    const bool valid = field(m, bc, x, l, &F);
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
    float s = m.v[l] < half_tau ? m.v[l] : half_tau;
    if (valid && F > 0.0f) {
      const float sF = 0.75f * F;
      if (sF > s) s = sF;
    }
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
