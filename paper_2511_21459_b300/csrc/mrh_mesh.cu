// Multi-resolution Marching Cubes over every allocated block of a map (Sec. 3.4, Figs. 5 and 6).
//
// Positions are integers in units of half a finest voxel: a block edge is 16 units and a level-l voxel centre lies at
// an odd multiple of 2^l. Every voxel is the low corner of one cell that runs, along each axis, to the next voxel
// centre: one voxel further inside its block; from the block's last voxel, to the first centre of the neighbouring
// block, half a voxel of each level away. A coarse cell next to a finer block is therefore cut short (the truncated
// coarse voxels of Fig. 6) and the cells of neighbouring blocks tile space without overlap; there is no cell where
// that neighbour is missing. A cell corner takes the trilinear field of the block that contains it, on that block's
// grid, each of the 8 nearest centres read from the voxel that contains it whatever its block's level (coarse and fine
// values blend across the boundary, Fig. 5); corners of zero weight are not read, and a cell with an unallocated or
// unobserved read emits nothing. The surface crosses a cell edge where it is linear between the corner values.
//
// One warp per allocated block, in two passes: the interior cells (all 8 corners are voxel centres of the block) read
// their corners straight from the payload; the shell of cells at the block's upper faces (the last voxel along some
// axis) evaluates the field with hash lookups. Each warp reserves its triangles with one atomic per 32 cells. Compiled without multiply-add contraction, so
// every vertex is the float result of the same operations the oracle performs.
#include <cuda_fp16.h>

#include <cstring>
#include <mutex>

#include "mrh_internal.cuh"

namespace mrh {
namespace {

// ---- case table: triangles per case (at most 5) as edge triples; corner c sits at (c & 1, c >> 1 & 1, c >> 2 & 1)
// and is inside when its value is below zero; edge 4a + r joins the r-th corner (ascending) with bit a clear to its
// neighbour along a.
__constant__ uint8_t c_ntri[256];
__constant__ int8_t c_tri[256][15];
__constant__ int8_t c_edge_end[12][2];

struct CaseTable {
  uint8_t ntri[256];
  int8_t tri[256][15];
  int8_t edge_end[12][2];
  bool ok = true;
};

// Built on the host from the definition: each face's corners are walked counter-clockwise as seen from outside the
// cell; a crossing where the walk enters the inside is joined to the next crossing where it leaves (so two diagonal
// inside corners of a face are cut off separately); the joined segments of the six faces close into loops, taken in
// order of their lowest edge and fanned into triangles from it.
CaseTable make_case_table() {
  CaseTable t;
  int edge_id[8][8];
  for (int i = 0; i < 8; ++i)
    for (int j = 0; j < 8; ++j) edge_id[i][j] = -1;
  int ne = 0;
  for (int axis = 0; axis < 3; ++axis)
    for (int lo = 0; lo < 8; ++lo) {
      if (lo & (1 << axis)) continue;
      const int hi = lo | (1 << axis);
      t.edge_end[ne][0] = (int8_t)lo;
      t.edge_end[ne][1] = (int8_t)hi;
      edge_id[lo][hi] = edge_id[hi][lo] = ne;
      ++ne;
    }
  // the 6 faces as corner cycles, counter-clockwise seen from outside: for the face at coordinate `side` of axis a,
  // with p = a + 1 and q = a + 2 (mod 3), the cycle (0,0) (1,0) (1,1) (0,1) in (p, q) faces +a, its reverse -a
  int face[6][4];
  for (int a = 0; a < 3; ++a) {
    const int p = (a + 1) % 3, q = (a + 2) % 3;
    const int pq[4][2] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}};
    for (int side = 0; side < 2; ++side)
      for (int k = 0; k < 4; ++k) {
        const int* c = pq[side ? k : (4 - k) & 3];
        face[2 * a + side][k] = (side << a) | (c[0] << p) | (c[1] << q);
      }
  }
  for (int cs = 0; cs < 256; ++cs) {
    int link[12];
    for (int e = 0; e < 12; ++e) link[e] = -1;
    for (int f = 0; f < 6; ++f) {
      int at[4], into[4], n = 0;
      for (int k = 0; k < 4; ++k) {
        const int c0 = face[f][k], c1 = face[f][(k + 1) & 3];
        const bool in0 = (cs >> c0) & 1, in1 = (cs >> c1) & 1;
        if (in0 == in1) continue;
        at[n] = edge_id[c0][c1];
        into[n] = in1 ? 1 : 0;
        ++n;
      }
      for (int k = 0; k < n; ++k)
        if (into[k]) link[at[k]] = at[(k + 1) % n];
    }
    int nt = 0;
    bool used[12] = {};
    for (int e0 = 0; e0 < 12; ++e0) {
      if (link[e0] < 0 || used[e0]) continue;
      int ring[12], len = 0;
      for (int e = e0; !used[e]; e = link[e]) {
        used[e] = true;
        ring[len++] = e;
        if (link[e] < 0) {
          t.ok = false;
          break;
        }
      }
      for (int k = 1; k + 1 < len; ++k) {
        if (nt >= 5) {
          t.ok = false;
          break;
        }
        t.tri[cs][3 * nt] = (int8_t)ring[0];
        t.tri[cs][3 * nt + 1] = (int8_t)ring[k];
        t.tri[cs][3 * nt + 2] = (int8_t)ring[k + 1];
        ++nt;
      }
    }
    for (int k = 3 * nt; k < 15; ++k) t.tri[cs][k] = -1;
    t.ntri[cs] = (uint8_t)nt;
  }
  return t;
}

// ---- device side

__device__ inline uint32_t block_val(const MapDev& m, int x, int y, int z) {
  const int lim = (int)kKeyLimit;
  if (x < -lim || x > lim || y < -lim || y > lim || z < -lim || z > lim) return kValPending;
  const int s = lookup_slot(m.slots, m.slot_mask, pack_key(x, y, z));
  return s >= 0 ? m.slots[s].val : kValPending;
}

__device__ inline const uint8_t* payload(const MapDev& m, uint32_t val) {
  const int l = (int)((val >> 28) & 3u);
  return m.heap[l] + (size_t)(val & kPtrMask) * m.block_bytes[l];
}

template <bool FP16>
__device__ inline float voxel_D(const uint8_t* blk, int i) {
  if (FP16) return __half2float(reinterpret_cast<const __half*>(blk)[i]);
  return reinterpret_cast<const float*>(blk)[i];
}

// The values of the 3 x 3 x 3 blocks around the block a warp meshes (looked up once, one lane each, into shared
// memory); a lookup outside the neighbourhood goes to the hash table.
struct Neighbourhood {
  const uint32_t* val;  // 27 entries, index (dx + 1) + 3 (dy + 1) + 9 (dz + 1)
  int K[3];
  __device__ inline uint32_t get(const MapDev& m, int x, int y, int z) const {
    const int dx = x - K[0] + 1, dy = y - K[1] + 1, dz = z - K[2] + 1;
    if ((unsigned)dx < 3u && (unsigned)dy < 3u && (unsigned)dz < 3u) return val[dx + 3 * dy + 9 * dz];
    return block_val(m, x, y, z);
  }
};

// trilinear field at the unit point P on the grid of the block containing it (see the file comment)
template <bool FP16, bool COLOR>
__device__ __noinline__ bool corner_value(const MapDev& m, const Neighbourhood& nb, const int P[3], float* out) {
  const uint32_t v = nb.get(m, P[0] >> 4, P[1] >> 4, P[2] >> 4);
  if (v == kValPending) return false;
  const int lp = (int)((v >> 28) & 3u);
  const int s = 1 << lp, s2 = 2 * s;
  int j0[3];
  float fr[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int g = P[a] - s;
    j0[a] = g >> (lp + 1);
    fr[a] = (float)(g - j0[a] * s2) / (float)s2;
  }
  float acc = 0.0f;
  int cx = 0x7FFFFFFF, cy = 0, cz = 0;  // last block looked up, and its value
  uint32_t cv = kValPending;
  for (int k = 0; k < 8; ++k) {
    const int ax = k & 1, ay = (k >> 1) & 1, az = k >> 2;
    const float wx = ax ? fr[0] : 1.0f - fr[0];
    const float wy = ay ? fr[1] : 1.0f - fr[1];
    const float wz = az ? fr[2] : 1.0f - fr[2];
    const float w = (wx * wy) * wz;
    if (w == 0.0f) continue;
    const int C[3] = {(2 * (j0[0] + ax) + 1) * s, (2 * (j0[1] + ay) + 1) * s, (2 * (j0[2] + az) + 1) * s};
    const int kx = C[0] >> 4, ky = C[1] >> 4, kz = C[2] >> 4;
    if (kx != cx || ky != cy || kz != cz) {
      cx = kx;
      cy = ky;
      cz = kz;
      cv = nb.get(m, kx, ky, kz);
    }
    if (cv == kValPending) return false;
    const int lb = (int)((cv >> 28) & 3u), nbs = kFineDim >> lb, sh = lb + 1;
    const int idx = ((C[0] - kx * 16) >> sh) + nbs * (((C[1] - ky * 16) >> sh) + nbs * ((C[2] - kz * 16) >> sh));
    const uint8_t* blk = payload(m, cv);
    if (!(reinterpret_cast<const float*>(blk + off_W(nbs * nbs * nbs, FP16, COLOR))[idx] > 0.0f)) return false;
    acc = acc + w * voxel_D<FP16>(blk, idx);
  }
  *out = acc;
  return true;
}

struct MeshOut {
  float* tris;
  unsigned long long cap;
  unsigned long long* count;
  uint32_t* next;  // chunks of 32 hash slots are handed out from this counter (zero at launch)
};

// One pass of 32 cells (warp-collective): reserve the pass's triangles with one atomic, then each lane writes its
// cell's triangles; vertex = low corner + f (high - low), f = F_low / (F_low - F_high), per coordinate in metres.
__device__ inline void emit_cell(const MeshOut& o, int lane, bool ok, int cs, const float F[8], const int c[3],
                                 const int h[3], float unit) {
  const int nt = ok ? (int)c_ntri[cs] : 0;
  int incl = nt;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int y = __shfl_up_sync(~0u, incl, d);
    if (lane >= d) incl += y;
  }
  unsigned long long first = 0;
  if (lane == 31 && incl > 0) first = atomicAdd(o.count, (unsigned long long)incl);
  first = __shfl_sync(~0u, first, 31) + (unsigned long long)(incl - nt);
  for (int t = 0; t < nt; ++t) {
    if (first + t >= o.cap) break;
    float* dst = o.tris + 9 * (first + t);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int e = c_tri[cs][3 * t + q];
      const int ca = c_edge_end[e][0], cb = c_edge_end[e][1];
      const float f = F[ca] / (F[ca] - F[cb]);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float pa = (float)(c[a] + ((ca >> a) & 1) * h[a]) * unit;
        const float pb = (float)(c[a] + ((cb >> a) & 1) * h[a]) * unit;
        dst[3 * q + a] = pa + f * (pb - pa);
      }
    }
  }
}

template <bool FP16, bool COLOR>
__global__ void __launch_bounds__(256) k_mesh(MapDev m, MeshOut o) {
  __shared__ uint32_t s_nbr[8][27];
  const int lane = threadIdx.x & 31;
  const uint32_t nslots = m.slot_mask + 1;
  const float unit = m.E / 16.0f;
  for (;;) {
    // blocks cost very different amounts (surface crossings, shell lookups): warps take chunks as they finish
    uint32_t chunk = 0;
    if (lane == 0) chunk = atomicAdd(o.next, 1u);
    const uint32_t base = __shfl_sync(~0u, chunk, 0) * 32u;
    if (base >= nslots) break;
    const uint32_t sl = base + lane;
    const unsigned long long key_l = sl < nslots ? m.slots[sl].key : kEmptyKey;
    const uint32_t val_l = sl < nslots ? m.slots[sl].val : kValPending;
    unsigned live = __ballot_sync(~0u, key_l != kEmptyKey && val_l != kValPending);
    while (live) {
      const int src = __ffs(live) - 1;
      live &= live - 1;
      const unsigned long long key = __shfl_sync(~0u, key_l, src);
      const uint32_t val = __shfl_sync(~0u, val_l, src);
      int K[3];
      unpack_key(key, &K[0], &K[1], &K[2]);
      const int l = (int)((val >> 28) & 3u), nl = kFineDim >> l, nv = nl * nl * nl, s = 1 << l;
      const uint8_t* blk = payload(m, val);
      const float* Wb = reinterpret_cast<const float*>(blk + off_W(nv, FP16, COLOR));
      uint32_t* s_nb = s_nbr[threadIdx.x >> 5];
      __syncwarp();  // the previous block's shell is done with the table
      if (lane < 27) s_nb[lane] = lane == 13 ? val : block_val(m, K[0] + lane % 3 - 1, K[1] + (lane / 3) % 3 - 1,
                                                               K[2] + lane / 9 - 1);
      __syncwarp();
      const Neighbourhood nb{s_nb, {K[0], K[1], K[2]}};
      // extent of the cells of the last voxel along each axis: to the first centre of the neighbouring block
      int hl[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const uint32_t nvl = s_nb[13 + (a == 0 ? 1 : a == 1 ? 3 : 9)];
        hl[a] = nvl == kValPending ? 0 : s + (1 << ((nvl >> 28) & 3u));
      }
      // interior cells: (nl - 1)^3 of them, corners read from the payload
      const int ni = nl - 1, n_in = ni * ni * ni;
      for (int b0 = 0; b0 < n_in; b0 += 32) {
        const int cell = b0 + lane;
        const bool in = cell < n_in;
        const int i[3] = {cell % ni, (cell / ni) % ni, cell / (ni * ni)};
        int c[3], h[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          c[a] = K[a] * 16 + (2 * i[a] + 1) * s;
          h[a] = 2 * s;
        }
        // the 16 loads of the cell's corners are independent (all in the block for an interior cell) and issued
        // together; the observed test and the case index follow
        float F[8], Wq[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int idx = (i[0] + (q & 1)) + nl * ((i[1] + ((q >> 1) & 1)) + nl * (i[2] + (q >> 2)));
          F[q] = in ? voxel_D<FP16>(blk, idx) : 0.0f;
          Wq[q] = in ? Wb[idx] : 0.0f;
        }
        bool ok = in;
        int cs = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          ok = ok && Wq[q] > 0.0f;
          if (F[q] < 0.0f) cs |= 1 << q;
        }
        emit_cell(o, lane, ok, cs, F, c, h, unit);
      }
      // the shell at the upper faces: z = last slab (nl^2), then y = last (nl (nl - 1)), then x = last ((nl - 1)^2)
      const int n_sh = nv - n_in;
      for (int b0 = 0; b0 < n_sh; b0 += 32) {
        const int b = b0 + lane;
        bool ok = b < n_sh;
        int i[3];
        if (b < nl * nl) {
          i[0] = b % nl;
          i[1] = b / nl;
          i[2] = nl - 1;
        } else if (b < nl * nl + nl * ni) {
          const int r = b - nl * nl;
          i[0] = r % nl;
          i[1] = nl - 1;
          i[2] = r / nl;
        } else {
          const int r = b - nl * nl - nl * ni;
          i[0] = nl - 1;
          i[1] = r % (ni > 0 ? ni : 1);
          i[2] = r / (ni > 0 ? ni : 1);
        }
        int c[3], h[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          c[a] = K[a] * 16 + (2 * i[a] + 1) * s;
          h[a] = i[a] < nl - 1 ? 2 * s : hl[a];
          ok = ok && h[a] > 0;
        }
        float F[8];
        int cs = 0;
#pragma unroll 1
        for (int q = 0; q < 8 && ok; ++q) {
          const int P[3] = {c[0] + (q & 1) * h[0], c[1] + ((q >> 1) & 1) * h[1], c[2] + (q >> 2) * h[2]};
          ok = corner_value<FP16, COLOR>(m, nb, P, &F[q]);
          if (ok && F[q] < 0.0f) cs |= 1 << q;
        }
        emit_cell(o, lane, ok, cs, F, c, h, unit);
      }
    }
  }
}

// ---- vertex collapse (see mrh_weld_mesh in the C ABI)

// order-preserving encoding of a float as an unsigned integer (and back)
__device__ inline uint32_t ord_f(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ inline float unord_f(uint32_t u) { return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u); }

// grid cell of a vertex, packed so that the integer order is the (x, then y, then z) order; false when out of range
__device__ inline bool weld_key(const float* p, float inv, unsigned long long* key) {
  unsigned long long k = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float q = floorf(p[a] * inv);
    if (!(fabsf(q) < 1048576.0f)) return false;
    k = (k << 21) | (unsigned long long)((long long)q + (1ll << 20));
  }
  *key = k;
  return true;
}

__device__ inline uint32_t weld_hash(unsigned long long k, uint32_t mask) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  return (uint32_t)k & mask;
}

__global__ void k_weld_init(WeldScratch w) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < w.table; i += gridDim.x * blockDim.x) {
    w.keys[i] = kEmptyKey;
    w.mn[3 * i] = w.mn[3 * i + 1] = w.mn[3 * i + 2] = 0xFFFFFFFFu;
  }
  if (blockIdx.x == 0 && threadIdx.x < 4) w.counters[threadIdx.x] = 0;
}

__global__ void k_weld_insert(WeldScratch w, const float* tris, uint32_t nv, float inv) {
  const uint32_t mask = w.table - 1;
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
    const float* p = tris + 3ull * v;
    unsigned long long key;
    if (!weld_key(p, inv, &key)) {
      w.vslot[v] = 0xFFFFFFFFu;
      atomicOr(&w.counters[1], 1u);
      continue;
    }
    uint32_t sl = weld_hash(key, mask);
    for (uint32_t probe = 0; probe < w.table; ++probe, sl = (sl + 1) & mask) {
      const unsigned long long cur = w.keys[sl];
      if (cur == key) break;
      if (cur == kEmptyKey) {
        const unsigned long long old = atomicCAS(&w.keys[sl], kEmptyKey, key);
        if (old == kEmptyKey) {
          atomicAdd(&w.counters[0], 1u);
          break;
        }
        if (old == key) break;
      }
    }
    w.vslot[v] = sl;
    atomicMin(&w.mn[3 * sl], ord_f(p[0]));
  }
}

// the smallest member: y among the members with the smallest x, then z among those with the smallest x and y
template <int AXIS>
__global__ void k_weld_min(WeldScratch w, const float* tris, uint32_t nv) {
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
    const uint32_t sl = w.vslot[v];
    if (sl == 0xFFFFFFFFu) continue;
    const float* p = tris + 3ull * v;
    bool lead = ord_f(p[0]) == w.mn[3 * sl];
    if (AXIS == 2) lead = lead && ord_f(p[1]) == w.mn[3 * sl + 1];
    if (lead) atomicMin(&w.mn[3 * sl + AXIS], ord_f(p[AXIS]));
  }
}

__global__ void k_weld_compact(WeldScratch w) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < w.table; i += gridDim.x * blockDim.x) {
    const unsigned long long k = w.keys[i];
    if (k == kEmptyKey) continue;
    const uint32_t j = atomicAdd(&w.counters[3], 1u);
    w.ckeys[j] = k;
    w.cslots[j] = i;
  }
}

// vertex i = the i-th cluster in key order
__global__ void k_weld_number(WeldScratch w, uint32_t n, float* verts, uint64_t cap) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t sl = w.cslots[i];
    w.vidx[sl] = i;
    if (i < cap)
#pragma unroll
      for (int a = 0; a < 3; ++a) verts[3ull * i + a] = unord_f(w.mn[3 * sl + a]);
  }
}

__device__ inline bool weld_face(const WeldScratch& w, uint64_t t, uint32_t* i0, uint32_t* i1, uint32_t* i2) {
  *i0 = w.vidx[w.vslot[3 * t]];
  *i1 = w.vidx[w.vslot[3 * t + 1]];
  *i2 = w.vidx[w.vslot[3 * t + 2]];
  return *i0 != *i1 && *i1 != *i2 && *i0 != *i2;
}

// faces keep their soup order: count the kept faces of each block of kWeldScanBlock, scan the counts, write
__global__ void __launch_bounds__(kWeldScanBlock) k_weld_count(WeldScratch w, uint64_t n_tris) {
  const uint64_t t = (uint64_t)blockIdx.x * kWeldScanBlock + threadIdx.x;
  uint32_t a, b, c;
  const int keep = t < n_tris && weld_face(w, t, &a, &b, &c);
  const int n = __syncthreads_count(keep);
  if (threadIdx.x == 0) w.blk[blockIdx.x] = (uint32_t)n;
}

__global__ void __launch_bounds__(1024) k_weld_scan(WeldScratch w, uint32_t nblk) {
  __shared__ uint32_t part[1024];
  const uint32_t per = (nblk + 1023) / 1024, lo = threadIdx.x * per;
  uint32_t sum = 0;
  for (uint32_t i = lo; i < lo + per && i < nblk; ++i) sum += w.blk[i];
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int d = 1; d < 1024; d <<= 1) {
    const uint32_t y = threadIdx.x >= (uint32_t)d ? part[threadIdx.x - d] : 0u;
    __syncthreads();
    part[threadIdx.x] += y;
    __syncthreads();
  }
  uint32_t run = part[threadIdx.x] - sum;
  for (uint32_t i = lo; i < lo + per && i < nblk; ++i) {
    const uint32_t c = w.blk[i];
    w.blk[i] = run;
    run += c;
  }
  if (threadIdx.x == 1023) w.counters[2] = part[1023];
}

__global__ void __launch_bounds__(kWeldScanBlock) k_weld_faces(WeldScratch w, uint64_t n_tris, int32_t* faces,
                                                               uint64_t cap) {
  __shared__ uint32_t warp_base[kWeldScanBlock / 32];
  const uint64_t t = (uint64_t)blockIdx.x * kWeldScanBlock + threadIdx.x;
  uint32_t a = 0, b = 0, c = 0;
  const bool keep = t < n_tris && weld_face(w, t, &a, &b, &c);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned bal = __ballot_sync(~0u, keep);
  if (lane == 0) warp_base[warp] = __popc(bal);
  __syncthreads();
  if (warp == 0) {
    uint32_t x = warp_base[lane], incl = x;
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(~0u, incl, d);
      if (lane >= d) incl += y;
    }
    warp_base[lane] = incl - x;
  }
  __syncthreads();
  if (keep) {
    const uint64_t pos = (uint64_t)w.blk[blockIdx.x] + warp_base[warp] + __popc(bal & ((1u << lane) - 1u));
    if (pos < cap) {
      faces[3 * pos] = (int32_t)a;
      faces[3 * pos + 1] = (int32_t)b;
      faces[3 * pos + 2] = (int32_t)c;
    }
  }
}

std::mutex g_table_mutex;
bool g_table_on[64] = {};

}  // namespace

cudaError_t mesh_table_ready(int device) {
  std::lock_guard<std::mutex> lock(g_table_mutex);
  if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
  if (g_table_on[device]) return cudaSuccess;
  static const CaseTable t = make_case_table();
  if (!t.ok) return cudaErrorUnknown;
  cudaError_t e = cudaMemcpyToSymbol(c_ntri, t.ntri, sizeof(t.ntri));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_tri, t.tri, sizeof(t.tri));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_edge_end, t.edge_end, sizeof(t.edge_end));
  if (e == cudaSuccess) g_table_on[device] = true;
  return e;
}

void host_case_table(uint8_t* ntri, int8_t* tri, int8_t* edge_end) {
  static const CaseTable t = make_case_table();
  std::memcpy(ntri, t.ntri, sizeof(t.ntri));
  std::memcpy(tri, t.tri, sizeof(t.tri));
  std::memcpy(edge_end, t.edge_end, sizeof(t.edge_end));
}

cudaError_t weld_clusters(const WeldScratch& w, const float* tris, uint32_t nv, float delta, cudaStream_t s, int sms) {
  const float inv = 1.0f / delta;
  k_weld_init<<<sms * 4, 256, 0, s>>>(w);
  k_weld_insert<<<sms * 8, 256, 0, s>>>(w, tris, nv, inv);
  k_weld_min<1><<<sms * 8, 256, 0, s>>>(w, tris, nv);
  k_weld_min<2><<<sms * 8, 256, 0, s>>>(w, tris, nv);
  k_weld_compact<<<sms * 8, 256, 0, s>>>(w);
  return cudaGetLastError();
}

cudaError_t weld_output(const WeldScratch& w, const float* tris, uint32_t n_clusters, float* verts, uint64_t cap_verts,
                        int32_t* faces, uint64_t cap_faces, uint64_t n_tris, size_t nblk, cudaStream_t s, int sms) {
  (void)tris;
  k_weld_number<<<sms * 8, 256, 0, s>>>(w, n_clusters, verts, cap_verts);
  k_weld_count<<<(unsigned)nblk, kWeldScanBlock, 0, s>>>(w, n_tris);
  k_weld_scan<<<1, 1024, 0, s>>>(w, (uint32_t)nblk);
  k_weld_faces<<<(unsigned)nblk, kWeldScanBlock, 0, s>>>(w, n_tris, faces, cap_faces);
  return cudaGetLastError();
}

void launch_mesh(const MapDev& m, float* tris, uint64_t cap, unsigned long long* count, cudaStream_t s, int sms) {
  const MeshOut o{tris, (unsigned long long)cap, count, &m.st->mesh_next};
  cudaMemsetAsync(o.next, 0, sizeof(uint32_t), s);
  const int grid = sms * 4;  // resident at once; the warps take slot chunks until none are left
  if (m.fp16) {
    if (m.color) k_mesh<true, true><<<grid, 256, 0, s>>>(m, o);
    else k_mesh<true, false><<<grid, 256, 0, s>>>(m, o);
  } else {
    if (m.color) k_mesh<false, true><<<grid, 256, 0, s>>>(m, o);
    else k_mesh<false, false><<<grid, 256, 0, s>>>(m, o);
  }
}

}  // namespace mrh
