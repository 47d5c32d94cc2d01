// Raycast of the adaptive grid (the rendering branch of Fig. 2): one thread per pixel.
//
// The ray is searched from min_depth to max_depth (as z-depth) for the first + -> - crossing of the trilinear TSDF on
// the sample grid t_j = t_min + j h, h = min(v_0, tau / 2) (cast_ray states which samples the march leaves out and
// why none of them can change the result). Brick and block occupancy come from two small insert-only sets filled when blocks are created
// (super-bricks of 4 x 4 x 4 bricks with a 64-bit mask of non-empty bricks; bricks with a 64-bit mask of created
// blocks), cached in registers, so a sample in empty space costs a memory probe only when the ray enters a new
// super-brick or non-empty brick. Inside an allocated block of level l the field is the trilinear interpolation over
// the 8 nearest voxel centres of that level's grid; a corner in a neighbouring block reads that block's voxel
// containing the corner centre, whatever its level, so coarse and fine blocks blend across resolution boundaries. A
// sample has a field only when all 8 corners are observed (W > 0). Output is z-depth, 0 where nothing was hit;
// optionally the unit normal (the normalised gradient of the same trilinear interpolant at the hit) and the colour
// (its trilinear mean of the stored colour, rounded to u8), zero where the hit's block or one of its 8 corners is
// missing or unobserved.
//
// Positions, trilinear sums and the root use fused multiply-adds where they save instructions: the raycast is
// compared with the CPU oracle's double-precision definition within a stated tolerance, not bit for bit.
#pragma once
#include <cuda_fp16.h>

#include <cstddef>

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

// heap value of block (x, y, z), or kValPending when the block is not allocated or has no storage. Not inlined:
// the probe loop is the cache-miss path of several call sites, and one copy keeps the kernel's code small.
static_assert(sizeof(Slot) == 16 && offsetof(Slot, val) == 8, "find_block reads a slot as one ulonglong2");

// Linear probing as lookup_slot, each probe one 16-byte load of the whole slot (key and heap value together, so a
// hit costs no second dependent load).
__device__ __noinline__ uint32_t find_block(const Slot* __restrict__ slots, uint32_t slot_mask, int x, int y, int z) {
  if (!key_ok32(x, y, z)) return kValPending;
  const unsigned long long key = pack_key(x, y, z);
  const uint32_t h = hash_key(key, slot_mask);
  const ulonglong2* sl = reinterpret_cast<const ulonglong2*>(slots);
  for (int p = 0; p < kMaxProbes; ++p) {
    const ulonglong2 e = sl[(h + (uint32_t)p) & slot_mask];
    if (e.x == key) return (uint32_t)e.y;  // Slot::val: the low word after the key
    if (e.x == kEmptyKey) return kValPending;
  }
  return kValPending;
}

// occupancy_bits with the mask word loaded next to each probed key (no second dependent load on a hit)
__device__ __noinline__ unsigned long long find_bits(const unsigned long long* __restrict__ keys,
                                                     const unsigned long long* __restrict__ vals, uint32_t mask,
                                                     int x, int y, int z) {
  if (!key_ok32(x, y, z)) return 0ull;
  const unsigned long long key = pack_key(x, y, z);
  const uint32_t h = hash_xyz(x, y, z, mask);
  for (int p = 0; p < kMaxProbes; ++p) {
    const uint32_t s = (h + (uint32_t)p) & mask;
    const unsigned long long c = keys[s], b = vals[s];
    if (c == key) return b;
    if (c == kEmptyKey) return 0ull;
  }
  return 0ull;
}

// Two most recent block lookups, keyed by coordinates, in registers (static indices only).
struct BlockCache {
  int x0 = 0x7FFFFFFF, y0 = 0, z0 = 0, x1 = 0x7FFFFFFF, y1 = 0, z1 = 0;
  uint32_t v0 = 0, v1 = 0;
  __device__ inline uint32_t get(const MapDev& m, int x, int y, int z) {
    if (x == x0 && y == y0 && z == z0) return v0;
    if (x == x1 && y == y1 && z == z1) {
      // promote
      const int tx = x0, ty = y0, tz = z0;
      const uint32_t tv = v0;
      x0 = x1; y0 = y1; z0 = z1; v0 = v1;
      x1 = tx; y1 = ty; z1 = tz; v1 = tv;
      return v0;
    }
    const uint32_t v = find_block(m.slots, m.slot_mask, x, y, z);
    x1 = x0; y1 = y0; z1 = z0; v1 = v0;
    x0 = x; y0 = y; z0 = z; v0 = v;
    return v;
  }
};

// Occupancy mask of one set (bricks or super-bricks) with a one-entry register cache.
struct OccCache {
  int x = 0x7FFFFFFF, y = 0, z = 0;
  unsigned long long bits = 0;
  __device__ inline unsigned long long get(const unsigned long long* keys, const unsigned long long* vals,
                                           uint32_t mask, int cx, int cy, int cz) {
    if (cx == x && cy == y && cz == z) return bits;
    x = cx;
    y = cy;
    z = cz;
    bits = find_bits(keys, vals, mask, cx, cy, cz);
    return bits;
  }
};

__device__ inline const uint8_t* block_ptr(const MapDev& m, uint32_t val) {
  const int lb = (int)((val >> 28) & 3u);
  return m.heap[lb] + (size_t)(val & kPtrMask) * m.block_bytes[lb];
}

// Storage format (FP16 / colour) is a template parameter of the raycaster, so field reads carry no format branches.
template <bool FP16>
__device__ inline float read_D(const uint8_t* blk, int i) {
  if (FP16) return __half2float(reinterpret_cast<const __half*>(blk)[i]);
  return reinterpret_cast<const float*>(blk)[i];
}
template <bool FP16, bool COLOR>
__device__ inline float read_W(const uint8_t* blk, int nv, int i) {
  return reinterpret_cast<const float*>(blk + off_W(nv, FP16, COLOR))[i];
}
template <bool FP16>
__device__ inline float read_C(const uint8_t* blk, int nv, int i, int q) {
  if (FP16) return __half2float(reinterpret_cast<const __half*>(blk + off_C(nv, 1, q))[i]);
  return reinterpret_cast<const float*>(blk + off_C(nv, 0, q))[i];
}

// Destination of one raycast: z-depth, and optionally normals (3 floats per pixel) and colours (3 bytes per pixel).
struct RayOut {
  float* depth;
  float* normal;
  uint8_t* rgb;
};

// trilinear field at x on the level-l grid; false when a corner is unallocated or unobserved. Each distinct block
// among the 8 corners is looked up once (usually there is only one); the corner sum runs in corner order 0..7.
template <bool FP16, bool COLOR>
__device__ bool field(const MapDev& m, BlockCache& bc, const float x[3], int l, float* out) {
  const float inv = m.inv_v[l];
  int j0[3];
  float fr[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float g = fmaf(x[a], inv, -0.5f);
    const float fl = floorf(g);
    j0[a] = (int)fl;
    fr[a] = g - fl;
  }
  const int sh = 3 - l, nl = 1 << sh, mask = nl - 1;
  const int b0[3] = {j0[0] >> sh, j0[1] >> sh, j0[2] >> sh};
  // corners with offset 1 along axis a fall in the next block iff j0 sits on the block's last voxel along a
  const bool sx = (j0[0] & mask) == mask, sy = (j0[1] & mask) == mask, sz = (j0[2] & mask) == mask;
  // distinct blocks of the corners, in registers: v<zyx> for the block offset (x, y, z) in {0, 1}^3
  uint32_t v000, v100 = 0, v010 = 0, v110 = 0, v001 = 0, v101 = 0, v011 = 0, v111 = 0;
  // every needed block is looked up before any is tested (a missing one only ends the sample afterwards)
  v000 = bc.get(m, b0[0], b0[1], b0[2]);
  if (sx) v100 = bc.get(m, b0[0] + 1, b0[1], b0[2]);
  if (sy) v010 = bc.get(m, b0[0], b0[1] + 1, b0[2]);
  if (sx && sy) v110 = bc.get(m, b0[0] + 1, b0[1] + 1, b0[2]);
  if (sz) v001 = bc.get(m, b0[0], b0[1], b0[2] + 1);
  if (sx && sz) v101 = bc.get(m, b0[0] + 1, b0[1], b0[2] + 1);
  if (sy && sz) v011 = bc.get(m, b0[0], b0[1] + 1, b0[2] + 1);
  if (sx && sy && sz) v111 = bc.get(m, b0[0] + 1, b0[1] + 1, b0[2] + 1);
  const bool ok = v000 != kValPending && (!sx || v100 != kValPending) && (!sy || v010 != kValPending) &&
                  (!(sx && sy) || v110 != kValPending) && (!sz || v001 != kValPending) &&
                  (!(sx && sz) || v101 != kValPending) && (!(sy && sz) || v011 != kValPending) &&
                  (!(sx && sy && sz) || v111 != kValPending);
  if (!ok) return false;
  const uint32_t lvl = (uint32_t)l;
  const bool same = ((v000 >> 28) & 3u) == lvl && (!sx || ((v100 >> 28) & 3u) == lvl) &&
                    (!sy || ((v010 >> 28) & 3u) == lvl) && (!(sx && sy) || ((v110 >> 28) & 3u) == lvl) &&
                    (!sz || ((v001 >> 28) & 3u) == lvl) && (!(sx && sz) || ((v101 >> 28) & 3u) == lvl) &&
                    (!(sy && sz) || ((v011 >> 28) & 3u) == lvl) && (!(sx && sy && sz) || ((v111 >> 28) & 3u) == lvl);
  if (same) {
    // the corners span 1 to 8 blocks (one in most samples), all of level l: a 32-bit word offset per block offset (a missing offset reuses
    // the block the corner falls in), the index of each corner from per-axis terms, the 16 loads issued together
    const uint8_t* hl = m.heap[l];
    const uint32_t bw = m.block_bytes[l] >> 2;
    uint32_t q[8];
    q[0] = (v000 & kPtrMask) * bw;
    q[1] = sx ? (v100 & kPtrMask) * bw : q[0];
    q[2] = sy ? (v010 & kPtrMask) * bw : q[0];
    q[3] = sx && sy ? (v110 & kPtrMask) * bw : (sx ? q[1] : q[2]);
    q[4] = sz ? (v001 & kPtrMask) * bw : q[0];
    q[5] = sx && sz ? (v101 & kPtrMask) * bw : (sx ? q[1] : q[4]);
    q[6] = sy && sz ? (v011 & kPtrMask) * bw : (sy ? q[2] : q[4]);
    q[7] = sx && sy && sz ? (v111 & kPtrMask) * bw
           : sx && sy ? q[3]
           : sx && sz ? q[5]
           : sy && sz ? q[6]
           : sx       ? q[1]
           : sy       ? q[2]
                      : q[4];
    const int nv = nl * nl * nl;
    const uint32_t wo = off_W(nv, FP16, COLOR) >> 2;
    const int ix0 = j0[0] & mask, ix1 = (j0[0] + 1) & mask;
    const int iy0 = (j0[1] & mask) * nl, iy1 = ((j0[1] + 1) & mask) * nl;
    const int iz0 = (j0[2] & mask) * nl * nl, iz1 = ((j0[2] + 1) & mask) * nl * nl;
    float w[8], d[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint32_t idx = (uint32_t)((k & 1 ? ix1 : ix0) + ((k >> 1) & 1 ? iy1 : iy0) + (k >> 2 ? iz1 : iz0));
      w[k] = reinterpret_cast<const float*>(hl)[q[k] + wo + idx];
      if (FP16) d[k] = __half2float(reinterpret_cast<const __half*>(hl)[2 * q[k] + idx]);
      else d[k] = reinterpret_cast<const float*>(hl)[q[k] + idx];
    }
    bool all = true;
#pragma unroll
    for (int k = 0; k < 8; ++k) all = all && w[k] > 0.0f;
    if (!all) return false;
    float acc = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float wx = (k & 1) ? fr[0] : 1.0f - fr[0];
      const float wy = ((k >> 1) & 1) ? fr[1] : 1.0f - fr[1];
      const float wz = (k >> 2) ? fr[2] : 1.0f - fr[2];
      acc = fmaf(wx * wy * wz, d[k], acc);
    }
    *out = acc;
    return true;
  }
  // corners in blocks of different levels: every corner's block and voxel first, the 16 loads issued together (no
  // early exit between them), then the observed test and the sum in corner order
  float w[8], d[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int ax = k & 1, ay = (k >> 1) & 1, az = k >> 2;
    const bool bx = ax && sx, by = ay && sy, bz = az && sz;
    const uint32_t val = bz ? (by ? (bx ? v111 : v011) : (bx ? v101 : v001))
                            : (by ? (bx ? v110 : v010) : (bx ? v100 : v000));
    const int lb = (int)((val >> 28) & 3u);
    const int nb = kFineDim >> lb;
    const uint8_t* blk = block_ptr(m, val);
    const int j[3] = {j0[0] + ax, j0[1] + ay, j0[2] + az};
    int idx;
    if (lb == l) {
      idx = (j[0] & mask) + nl * ((j[1] & mask) + nl * (j[2] & mask));
    } else {
      // the finest-level cell holding the corner centre, then the block's voxel (at its own level) containing it
      int cc[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) cc[a] = (l == 0 ? j[a] : (j[a] << l) + (1 << (l - 1))) >> lb;
      idx = (cc[0] & (nb - 1)) + nb * ((cc[1] & (nb - 1)) + nb * (cc[2] & (nb - 1)));
    }
    w[k] = read_W<FP16, COLOR>(blk, nb * nb * nb, idx);
    d[k] = read_D<FP16>(blk, idx);
  }
  bool all = true;
#pragma unroll
  for (int k = 0; k < 8; ++k) all = all && w[k] > 0.0f;
  if (!all) return false;
  float acc = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float wx = (k & 1) ? fr[0] : 1.0f - fr[0];
    const float wy = ((k >> 1) & 1) ? fr[1] : 1.0f - fr[1];
    const float wz = (k >> 2) ? fr[2] : 1.0f - fr[2];
    acc = fmaf(wx * wy * wz, d[k], acc);
  }
  *out = acc;
  return true;
}

// Surface attributes at a hit x in a block of level l, over the 8 corners field() uses (each corner's block and voxel
// found the same way): g = the interpolant's gradient times v_l (the x weight's derivative is +1 for the upper
// corner, -1 for the lower), col = the trilinear mean of the stored colour, both summed in corner order. False when a
// corner's block is unallocated or a corner is unobserved. Runs once per hit pixel; the corners' weights and
// distances are loaded together before they are tested.
template <bool FP16, bool COLOR>
__device__ __noinline__ bool shade(const MapDev& m, const float x[3], int l, float g[3], float col[3]) {
  const float inv = m.inv_v[l];
  int j0[3];
  float fr[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float gg = x[a] * inv - 0.5f;
    const float fl = floorf(gg);
    j0[a] = (int)fl;
    fr[a] = gg - fl;
    g[a] = 0.0f;
    col[a] = 0.0f;
  }
  const int sh = 3 - l, nl = 1 << sh, mask = nl - 1;
  const uint8_t* blk[8];
  int nvs[8], idx[8];
  int lb0 = 0x7FFFFFFF, lb1 = 0, lb2 = 0;  // the last corner's block and its heap value (corners share blocks)
  uint32_t lval = kValPending;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int ax = k & 1, ay = (k >> 1) & 1, az = k >> 2;
    const int j[3] = {j0[0] + ax, j0[1] + ay, j0[2] + az};
    const int c0 = j[0] >> sh, c1 = j[1] >> sh, c2 = j[2] >> sh;
    if (c0 != lb0 || c1 != lb1 || c2 != lb2) {
      lb0 = c0;
      lb1 = c1;
      lb2 = c2;
      lval = find_block(m.slots, m.slot_mask, c0, c1, c2);
    }
    if (lval == kValPending) return false;
    const int lb = (int)((lval >> 28) & 3u);
    const int nb = kFineDim >> lb;
    blk[k] = block_ptr(m, lval);
    nvs[k] = nb * nb * nb;
    if (lb == l) {
      idx[k] = (j[0] & mask) + nl * ((j[1] & mask) + nl * (j[2] & mask));
    } else {
      int cc[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) cc[a] = (l == 0 ? j[a] : (j[a] << l) + (1 << (l - 1))) >> lb;
      idx[k] = (cc[0] & (nb - 1)) + nb * ((cc[1] & (nb - 1)) + nb * (cc[2] & (nb - 1)));
    }
  }
  float w[8], d[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    w[k] = read_W<FP16, COLOR>(blk[k], nvs[k], idx[k]);
    d[k] = read_D<FP16>(blk[k], idx[k]);
  }
  bool ok = true;
#pragma unroll
  for (int k = 0; k < 8; ++k) ok = ok && w[k] > 0.0f;
  if (!ok) return false;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int ax = k & 1, ay = (k >> 1) & 1, az = k >> 2;
    const float wx = ax ? fr[0] : 1.0f - fr[0];
    const float wy = ay ? fr[1] : 1.0f - fr[1];
    const float wz = az ? fr[2] : 1.0f - fr[2];
    const float tx = (wy * wz) * d[k], ty = (wx * wz) * d[k], tz = (wx * wy) * d[k];
    g[0] = ax ? g[0] + tx : g[0] - tx;
    g[1] = ay ? g[1] + ty : g[1] - ty;
    g[2] = az ? g[2] + tz : g[2] - tz;
    if (COLOR) {
      const float wt = (wx * wy) * wz;
#pragma unroll
      for (int q = 0; q < 3; ++q) col[q] = col[q] + wt * read_C<FP16>(blk[k], nvs[k], idx[k], q);
    }
  }
  return true;
}

// One ray: march, find the first zero crossing, write its z-depth (0 = none) and the requested surface attributes.
//
// The crossing searched is the one of the definition: samples on the grid t_j = t_min + j h, h = min(v_0, tau / 2),
// the first two consecutive samples that both have a field with F_j > 0 >= F_j+1, narrowed inside that bracket. The
// march visits the grid samples in order and leaves out only samples that cannot end such a bracket:
//   - a level-l block is sampled at its own voxel pitch (the definition's min(v_l, tau / 2)): every 2^l-th grid sample
//     from its first one, then the first grid sample past its exit face;
//   - a sample in an empty brick or unallocated block has no field, nor has any other sample of that cell: the march
//     continues at the first grid sample past the cell's exit face;
//   - in a block whose observed voxels all hold D > 0 (dmin, kept by the fusion epilogue), every sample whose 8
//     corners lie in the block (the block shrunk by half a voxel, and by a further 1e-3 voxel so that float rounding
//     of the position cannot move a sample across) has F > 0 or no field: after the first such sample the march
//     continues at the last grid sample of that interior (of the block's pitch), which it evaluates, since it may
//     begin a bracket;
//   - the bracket (1 to 4 grid steps wide) is narrowed by bisections (the definition's own first steps) down to h / 8
//     and the linear root of the last bracket: the result lies within h / 8 of the fully converged crossing of the
//     same bracket.
template <bool FP16, bool COLOR>
__device__ inline void cast_ray(const MapDev& m, const CamArgs& c, int u, int v, const RayOut& out) {
  BlockCache bc;
  OccCache super_c, brick_c;
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
  const float E = m.E, invE = 1.0f / E;
  const float h = fminf(m.v[0], 0.5f * m.tau), inv_h = 1.0f / h;
  const float t0 = c.min_depth * nq, t_far = c.max_depth * nq;
  int j = 0;           // grid index of the current sample
  bool pv = false;     // the previous sample (index jp, parameter tp) was evaluated, with nothing skipped since, and
  float Fp = 0.0f;     // has a field of value Fp
  int jp = 0;
  float tp = 0.0f;
  int cb0 = 0x7FFFFFFF, cb1 = 0, cb2 = 0, jb = 0;  // the allocated block of the last sample and its first sample
  float dmin_b = 0.0f;                              // and its least stored D
  int jn_b = 0;                                     // and, at a coarse level, the first sample beyond its exit face
  // refine > 0: the loop evaluates the bracket's midpoint tm (the same code path as every grid sample, so the field
  // evaluation exists once in the kernel)
  int refine = 0;
  float ta = 0.0f, Fa = 0.0f, tb = 0.0f, Fb = 0.0f, tm = 0.0f, t_hit = 0.0f;
  bool hit = false;
  for (int it = 0; it < kRaycastMaxIter; ++it) {
    const float t = refine ? tm : fmaf((float)j, h, t0);
    if (!refine && t > t_far) break;
    const float x[3] = {fmaf(t, r[0], o[0]), fmaf(t, r[1], o[1]), fmaf(t, r[2], o[2])};
    const int bk[3] = {ifloor(x[0] * invE), ifloor(x[1] * invE), ifloor(x[2] * invE)};
    const int br[3] = {bk[0] >> kBrickShift, bk[1] >> kBrickShift, bk[2] >> kBrickShift};
    // occupancy: super-brick mask (probed when the super-brick changes) -> brick non-empty? -> brick mask (probed
    // when the brick changes) -> block created? -> block lookup. Empty cells cost register work only.
    const unsigned long long sbits = super_c.get(m.super_keys, m.super_bits, m.super_mask, br[0] >> kSuperShift,
                                                 br[1] >> kSuperShift, br[2] >> kSuperShift);
    const bool brick = (sbits & cell_bit(br[0], br[1], br[2])) != 0;
    bool block = false;
    if (brick) {
      const unsigned long long bbits = brick_c.get(m.brick_keys, m.brick_bits, m.brick_mask, br[0], br[1], br[2]);
      block = (bbits & cell_bit(bk[0], bk[1], bk[2])) != 0;
    }
    const uint32_t val = block ? bc.get(m, bk[0], bk[1], bk[2]) : kValPending;
    if (val == kValPending) {
      if (refine) {  // a midpoint without a field: the crossing is taken there
        t_hit = tm;
        hit = true;
        break;
      }
      // continue at the first grid sample past the exit face of the empty super-brick, brick, or block
      const bool sempty = sbits == 0ull;
      const int span = brick ? 1 : sempty ? (1 << (kBrickShift + kSuperShift)) : (1 << kBrickShift);
      float t_exit = t_far + 1.0f;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (r[a] == 0.0f) continue;
        const int cell = brick ? bk[a] : sempty ? (br[a] >> kSuperShift) : br[a];
        const float face = (float)((r[a] > 0.0f ? cell + 1 : cell) * span) * E;
        const float tf = (face - o[a]) * inv_r[a];
        if (tf < t_exit) t_exit = tf;
      }
      const float jf = ceilf((t_exit - t0) * inv_h);
      const int jn = jf < 1073741824.0f ? (int)jf : 1073741824;
      j = jn > j ? jn : j + 1;
      pv = false;
      continue;
    }
    const int l = (int)((val >> 28) & 3u);
    if (!refine && (bk[0] != cb0 || bk[1] != cb1 || bk[2] != cb2)) {
      cb0 = bk[0];
      cb1 = bk[1];
      cb2 = bk[2];
      jb = j;
      dmin_b = m.dmin[l][val & kPtrMask];  // read once per block: the samples of a block test a register
      if (l > 0) {
        // a coarse block's samples stop at the first grid sample beyond its exit face (also computed once)
        float t_exit = t_far + 1.0f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          if (r[a] == 0.0f) continue;
          const float face = (float)(r[a] > 0.0f ? bk[a] + 1 : bk[a]) * E;
          const float tf = (face - o[a]) * inv_r[a];
          if (tf < t_exit) t_exit = tf;
        }
        const float jf = ceilf((t_exit - t0) * inv_h);
        jn_b = jf < 1073741824.0f ? (int)jf : 1073741824;
      }
    }
    int j_skip = -1;  // the interior's last grid sample, when this sample lies in a positive block's interior
    if (!refine && dmin_b > 0.0f) {
      // inside the block's interior (every corner in the block)? then the march continues at the interior's last
      // grid sample after this one (evaluated first, so that the least-D load overlaps the corner loads)
      const float vl = m.v[l], in = (0.5f + 1e-3f) * vl;
      float t_out = t_far + 1.0f;
      bool inside = true;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float lo = fmaf((float)bk[a], E, in), hi = fmaf((float)(bk[a] + 1), E, -in);
        inside = inside && x[a] >= lo && x[a] <= hi;
        if (r[a] != 0.0f) {
          const float tf = ((r[a] > 0.0f ? hi : lo) - o[a]) * inv_r[a];
          if (tf < t_out) t_out = tf;
        }
      }
      if (inside) {
        const float jf = floorf((t_out - t0) * inv_h);
        int jl = jf < 1073741824.0f ? (int)jf : 1073741824;
        jl = jb + (((jl - jb) >> l) << l);  // a sample of the block's pitch
        if (jl > j) j_skip = jl;
      }
    }
    float F = 0.0f;
    const bool valid = field<FP16, COLOR>(m, bc, x, l, &F);
    if (refine) {
      if (!valid) {
        t_hit = tm;
        hit = true;
        break;
      }
      if (F > 0.0f) {
        ta = tm;
        Fa = F;
      } else {
        tb = tm;
        Fb = F;
      }
      if (--refine == 0) {
        t_hit = ta + (tb - ta) * (Fa / (Fa - Fb));
        hit = true;
        break;
      }
      tm = 0.5f * (ta + tb);
      continue;
    }
    if (valid && pv && Fp > 0.0f && !(F > 0.0f)) {
      ta = tp;
      Fa = Fp;
      tb = t;
      Fb = F;
      const int steps = j - jp;  // bisections down to h / 8
      refine = 3 + (steps > 1 ? 1 : 0) + (steps > 2 ? 1 : 0);
      tm = 0.5f * (ta + tb);
      continue;
    }
    pv = valid;
    Fp = F;
    jp = j;
    tp = t;
    // the block's pitch, but not past the first grid sample beyond its exit face
    const int step = l > 0 ? min(1 << l, jn_b > j ? jn_b - j : 1) : 1;
    if (j_skip > j + step) {
      j = j_skip;
      pv = false;  // the samples left out were positive or had no field: none can end a bracket at sample j_skip
    } else {
      j += step;
    }
  }
  const size_t px = (size_t)v * c.width + u;
  out.depth[px] = hit ? t_hit * rc[2] : 0.0f;
  if (out.normal || out.rgb) {
    float g[3], col[3];
    bool ok = false;
    if (hit) {
      const float xh[3] = {fmaf(t_hit, r[0], o[0]), fmaf(t_hit, r[1], o[1]), fmaf(t_hit, r[2], o[2])};
      const uint32_t val = bc.get(m, ifloor(xh[0] * invE), ifloor(xh[1] * invE), ifloor(xh[2] * invE));
      ok = val != kValPending && shade<FP16, COLOR>(m, xh, (int)((val >> 28) & 3u), g, col);
    }
    if (out.normal) {
      const float nn = ok ? sqrtf(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]) : 0.0f;
#pragma unroll
      for (int a = 0; a < 3; ++a) out.normal[3 * px + a] = nn > 0.0f ? g[a] / nn : 0.0f;
    }
    if (out.rgb) {
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float cv = ok && COLOR ? col[q] + 0.5f : 0.0f;
        out.rgb[3 * px + q] = (uint8_t)(cv <= 0.0f ? 0 : cv >= 255.0f ? 255 : (int)cv);
      }
    }
  }
}

// cast_ray with the storage format chosen at run time (one branch per ray)
__device__ inline void cast_ray_any(const MapDev& m, const CamArgs& c, int u, int v, const RayOut& out) {
  if (m.fp16) {
    if (m.color) cast_ray<true, true>(m, c, u, v, out);
    else cast_ray<true, false>(m, c, u, v, out);
  } else {
    if (m.color) cast_ray<false, true>(m, c, u, v, out);
    else cast_ray<false, false>(m, c, u, v, out);
  }
}

}  // namespace
}  // namespace mrh
