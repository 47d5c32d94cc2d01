// Fusion of one frame into the touched blocks, the block variance and re-levelling, in one pass.
//
//   camera  (Sec. 3.1 "Cameras", Eq. 2): every voxel of a touched block projects to its nearest pixel; the signed
//           distance is the pixel's range minus the voxel's distance, occluded voxels (more than tau behind) are
//           skipped, the rest clipped to tau.
//   LiDAR   (Sec. 3.1 "3D Point Cloud", Eq. 1): each ray walks the voxels of its truncation band (a DDA over
//           finest-level cells, one observation per voxel of the block's own level); d = clip((p - x) . n, tau).
//           One walk per point stages its observations and counts them per block; each fusion item gets one
//           segment of the observation buffer and the staged runs are scattered into it; inside a block they are
//           binned per voxel and each voxel applies its observations in ascending point index, so the result does
//           not depend on scheduling.
//   both    running mean (Eq. 3, w_k = 1) in Welford's incremental form and S2 += (d - D_old)(d - D_new)
//           (Sec. 3.2.1); then the mean voxel variance of the block over observed voxels; then merge to the next
//           coarser level below theta_l (Sec. 3.2.1, Fig. 4a) or split to the next finer level above h theta_{l-1}.
//
// Work decomposition: one warp per work item, with no CTA-wide barrier anywhere. An item is one level-0 block (8^3
// voxels, 32 lanes), two level-1 blocks (4^3, 16 lanes each) or sixteen level-2 blocks (2^3, 2 lanes each). A lane
// owns 4 consecutive voxels per chunk of 4 G voxels (G = lanes per block) and moves each field of them with one
// 16-byte (fp32) or 8-byte (fp16) access: the fields of a block stream fully coalesced. The block's mean variance is
// a butterfly shuffle reduction that leaves the sum in every lane of the block's group, so every lane takes the same
// decision without communication. Re-levelled blocks (a small fraction per frame) are resampled from their just-
// written payload into a heap block popped from the other level's free stack.
//
// The block variance decides in float; a value within 1e-5 (relative) of a threshold is recomputed in double, in
// voxel order, exactly as the CPU oracle computes it, so level decisions match the oracle bit for bit. (The float
// estimate's relative error is below 24 ulp = 1.5e-6: 15 sequential + 5 shuffle additions of non-negative terms, the
// per-voxel approximate quotient S2 / W (__fdividef, within 2 ulp) and the final division.)
//
// This file is compiled without multiply-add contraction: float expressions round in source order, like the oracle.
#pragma once
#include <cuda_fp16.h>

#include "mrh_internal.cuh"

namespace mrh {
namespace {

constexpr float kBandF = 1e-5f;
constexpr uint32_t kInvalidPtr = 0xFFFFFFFFu;
enum { kActNone = 0, kActMerge = 1, kActSplit = 2 };

template <bool FP16>
struct Field {
  static __device__ inline void load4(const uint8_t* p, int i4, float out[4]) {
    if constexpr (FP16) {
      uint2 u = reinterpret_cast<const uint2*>(p)[i4];
      __half2 a = *reinterpret_cast<__half2*>(&u.x), b = *reinterpret_cast<__half2*>(&u.y);
      float2 fa = __half22float2(a), fb = __half22float2(b);
      out[0] = fa.x; out[1] = fa.y; out[2] = fb.x; out[3] = fb.y;
    } else {
      float4 f = reinterpret_cast<const float4*>(p)[i4];
      out[0] = f.x; out[1] = f.y; out[2] = f.z; out[3] = f.w;
    }
  }
  static __device__ inline void store4(uint8_t* p, int i4, const float in[4]) {
    if constexpr (FP16) {
      __half2 a = __floats2half2_rn(in[0], in[1]), b = __floats2half2_rn(in[2], in[3]);
      uint2 u;
      u.x = *reinterpret_cast<uint32_t*>(&a);
      u.y = *reinterpret_cast<uint32_t*>(&b);
      reinterpret_cast<uint2*>(p)[i4] = u;
    } else {
      reinterpret_cast<float4*>(p)[i4] = make_float4(in[0], in[1], in[2], in[3]);
    }
  }
  static __device__ inline float get1(const uint8_t* p, int i) {
    if constexpr (FP16) return __half2float(reinterpret_cast<const __half*>(p)[i]);
    else return reinterpret_cast<const float*>(p)[i];
  }
  static __device__ inline void store1(uint8_t* p, int i, float x) {
    if constexpr (FP16) reinterpret_cast<__half*>(p)[i] = __float2half_rn(x);
    else reinterpret_cast<float*>(p)[i] = x;
  }
  // the value a later read of the stored field returns
  static __device__ inline float kept(float x) {
    if constexpr (FP16) return __half2float(__float2half_rn(x));
    else return x;
  }
};

// One Welford step (Eq. 3 incremental form + S2 update of Sec. 3.2.1); the division by W + 1 is a multiplication by
// its correctly rounded reciprocal (the oracle's reading of the arithmetic).
template <bool FP16>
__device__ inline void welford(float d, float& D, float& W, float& S2, float& Wn) {
  Wn = W + 1.0f;
  const float inv = __frcp_rn(Wn);
  float e = d - D;
  float Dn = D + e * inv;
  S2 = S2 + e * (d - Dn);
  D = Field<FP16>::kept(Dn);
  W = Wn;
}

// 4 consecutive voxels of one lane
struct Chunk {
  float D[4], W[4], S2[4], C[3][4];
};

// What a lane knows about the block its group works on.
struct Ctx {
  int l, nl, nv, G, g, li;
  bool active;
  uint32_t P;        // position in the level-concatenated list (LiDAR buffers)
  uint32_t P_first;  // P of the item's first group
  int kx, ky, kz;    // block key
};

// -------------------------------------------------------------------------------------------- camera observer

// Reads the frame's range image (rho = z |K^-1 [u v 1]|, written by the allocation kernel with the same float
// expression, -1 where the depth is invalid) and its colour packed as one 32-bit word per pixel, so a voxel costs one
// 4-byte gather per image instead of recomputing the pixel ray. CamT: the camera held by value (a kernel parameter)
// or by reference (a copy in shared memory, batched path).
template <bool FP16, bool COLOR, class CamT = CamArgs>
struct CameraObs {
  CamT c;
  const float* rho_img;
  const uint32_t* rgb_img;  // null when the frame has no colour

  static constexpr bool kDefers = false;
  __device__ inline void collect(const MapDev&, const Ctx&, int) {}
  __device__ inline int take_deferred(const Ctx&, int) const { return 0; }

  // voxels vi0 .. vi0 + 3 of the block. Written without early exits: all four voxels are computed side by side and
  // an update is kept only where the voxel is observed, so the four independent chains can overlap.
  __device__ inline int apply(const MapDev& m, const Ctx& x, int vi0, Chunk& ch, int& n_vox, int&) const {
    const float vl = m.v[x.l];
    const float ob0 = (float)x.kx * m.E - c.t[0];
    const float ob1 = (float)x.ky * m.E - c.t[1];
    const float ob2 = (float)x.kz * m.E - c.t[2];
    const int sh = 3 - x.l, msk = x.nl - 1;
    const float fw = (float)c.width, fh = (float)c.height;
    int n_upd = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int vi = vi0 + k;
      const int xi = vi & msk, yi = (vi >> sh) & msk, zi = vi >> (2 * sh);
      const float w0 = ob0 + ((float)xi + 0.5f) * vl;
      const float w1 = ob1 + ((float)yi + 0.5f) * vl;
      const float w2 = ob2 + ((float)zi + 0.5f) * vl;
      const float xc = c.R[0] * w0 + c.R[3] * w1 + c.R[6] * w2;
      const float yc = c.R[1] * w0 + c.R[4] * w1 + c.R[7] * w2;
      const float zc = c.R[2] * w0 + c.R[5] * w1 + c.R[8] * w2;
      const float iz = __frcp_rn(zc);  // both quotients by z use its correctly rounded reciprocal
      const float uf = c.fx * xc * iz + c.cx + 0.5f;
      const float vf = c.fy * yc * iz + c.cy + 0.5f;
      bool ok = zc > 0.0f && uf >= 0.0f && uf < fw && vf >= 0.0f && vf < fh;
      const int u = ok ? (int)floorf(uf) : 0, v = ok ? (int)floorf(vf) : 0;
      const int pix = v * c.width + u;
      const float rho = __ldg(rho_img + pix);
      const float dist = sqrtf(xc * xc + yc * yc + zc * zc);
      const float eta = rho - dist;
      ok = ok && rho >= 0.0f && !(eta < -m.tau);  // valid depth; not occluded (more than tau behind the surface)
      const float d = eta < m.tau ? eta : m.tau;
      const float Wn = ch.W[k] + 1.0f;
      const float inv = __frcp_rn(Wn);  // 1 / (W + 1), shared by D and the colour channels
      const float e = d - ch.D[k];
      const float Dn = ch.D[k] + e * inv;
      const float S2n = ch.S2[k] + e * (d - Dn);
      if (ok) {
        ch.D[k] = Field<FP16>::kept(Dn);
        ch.W[k] = Wn;
        ch.S2[k] = S2n;
        ++n_upd;
      }
      if constexpr (COLOR) {
        if (rgb_img) {
          const uint32_t packed = __ldg(rgb_img + pix);
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            const float col = (float)((packed >> (8 * q)) & 255u);
            const float Cn = ch.C[q][k] + (col - ch.C[q][k]) * inv;
            if (ok) ch.C[q][k] = Cn;  // rounded to the storage format by the store (nothing reads it before)
          }
        }
      }
    }
    n_vox = n_upd;  // a camera frame observes a voxel at most once
    return n_upd;
  }
};

// -------------------------------------------------------------------------------------------- LiDAR observer

// Per warp, in shared memory: 512 voxel bins (the item's voxels) as exclusive offsets (entry 512 = total) and fill
// cursors. The item's observation records are regrouped per voxel in global memory (obs_bin, the item's range of it).
constexpr int kLidarWarps = 4;
constexpr int kLocalSort = 16;

struct LidarSmem {
  uint32_t off[kLidarWarps][513];
  uint32_t fill[kLidarWarps][512];  // fill cursors while regrouping; then the queue of deferred voxels
  uint32_t n_deferred[kLidarWarps];
};

template <bool FP16>
struct LidarObs {
  LidarSmem* sm;
  uint2* recs;  // this warp's regrouped records: obs_bin + item base
  mutable uint32_t vmax = 0;  // the most observations one of this lane's voxels received

  // warp-collective: regroup the item's observations per voxel (bin = group * nv + voxel), keeping for each voxel
  // its records contiguous
  __device__ inline void collect(const MapDev& m, const Ctx& x, int warp) {
    const int lane = threadIdx.x & 31;
    uint32_t* off = sm->off[warp];
    uint32_t* fill = sm->fill[warp];
    for (int i = lane; i < 512; i += 32) {
      off[i] = 0;
      fill[i] = 0;
    }
    __syncwarp();
    uint32_t r0 = 0, r1 = 0;
    if (x.active) {
      r0 = m.blk_off[x.P];
      r1 = r0 + m.blk_count[x.P];
      if (r1 > m.max_obs) r0 = r1 = 0;  // observations were not stored (status already set)
    }
    {
      // four independent record loads in flight before their shared-memory counts
      const uint32_t base = (uint32_t)(x.g * x.nv);
      uint32_t r = r0 + x.li;
      for (; r + 3u * x.G < r1; r += 4u * x.G) {
        uint32_t v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = m.obs_rec[r + k * x.G].x;
#pragma unroll
        for (int k = 0; k < 4; ++k) atomicAdd(&off[base + (v[k] & 511u)], 1u);
      }
      for (; r < r1; r += x.G) atomicAdd(&off[base + (m.obs_rec[r].x & 511u)], 1u);
    }
    __syncwarp();
    // counts -> exclusive offsets (16 consecutive bins per lane)
    uint32_t local[16], sum = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      local[k] = off[16 * lane + k];
      sum += local[k];
    }
    uint32_t incl = sum;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(~0u, incl, o);
      if (lane >= o) incl += t;
    }
    uint32_t run = incl - sum;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      off[16 * lane + k] = run;
      run += local[k];
    }
    if (lane == 31) off[512] = incl;
    recs = m.obs_bin + m.blk_off[x.P_first];
    __syncwarp();
    {
      const uint32_t base = (uint32_t)(x.g * x.nv);
      uint32_t r = r0 + x.li;
      for (; r + 3u * x.G < r1; r += 4u * x.G) {
        uint2 q[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) q[k] = m.obs_rec[r + k * x.G];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint32_t bin = base + (q[k].x & 511u);
          recs[off[bin] + atomicAdd(&fill[bin], 1u)] = q[k];
        }
      }
      for (; r < r1; r += x.G) {
        const uint2 rec = m.obs_rec[r];
        const uint32_t bin = base + (rec.x & 511u);
        recs[off[bin] + atomicAdd(&fill[bin], 1u)] = rec;
      }
    }
    if (lane == 0) sm->n_deferred[warp] = 0;
    __syncwarp();
  }

  // Level-0 items defer the voxels with three or more observations (about 10 % of observed voxels in a street scan):
  // they are applied afterwards with one voxel per lane, so that the whole warp does not run the long path whenever
  // one lane needs it. Returns the number of deferred voxels (queued in fill[]).
  static constexpr bool kDefers = true;
  __device__ inline int take_deferred(const Ctx&, int warp) const {
    __syncwarp();
    return (int)sm->n_deferred[warp];
  }
  __device__ inline uint32_t deferred(int warp, int q) const { return sm->fill[warp][q]; }
  __device__ inline uint32_t range(int warp, uint32_t bin, uint32_t* cnt) const {
    const uint32_t o0 = sm->off[warp][bin];
    *cnt = sm->off[warp][bin + 1] - o0;
    return o0;
  }

  // Sorting network on N keys in registers (bitonic, ascending; N a power of two; all indices compile-time).
  template <int N>
  __device__ static void bitonic_sort(unsigned long long (&e)[N]) {
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
      for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
          const int p = i ^ j;
          if (p > i) {
            const unsigned long long a = e[i], b = e[p];
            const bool up = (i & k) == 0;
            const bool swap = up ? a > b : a < b;
            e[i] = swap ? b : a;
            e[p] = swap ? a : b;
          }
        }
      }
    }
  }

  // The observations of one voxel with three to N of them: all records loaded with independent loads, sorted by
  // key in registers (padding keys sort last), applied in point order.
  template <int N>
  __device__ static void apply_sorted(const uint2* rec, uint32_t cnt, float& D, float& W, float& S2) {
    unsigned long long e[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const uint2 q = (uint32_t)i < cnt ? rec[i] : make_uint2(0xFFFFFFFFu, 0u);
      e[i] = ((unsigned long long)q.x << 32) | q.y;
    }
    bitonic_sort<N>(e);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      if ((uint32_t)i < cnt) {
        float Wn;
        welford<FP16>(__uint_as_float((uint32_t)e[i]), D, W, S2, Wn);
      }
    }
  }

  // the observations of one voxel with three or more, in point order (about 10 % of observed voxels in a street
  // scan, 93 % of them with at most 8; coarse voxels can hold hundreds)
  __device__ static void apply_long(const uint2* rec, uint32_t cnt, float& D, float& W, float& S2) {
    if (cnt <= 8) {
      apply_sorted<8>(rec, cnt, D, W, S2);
    } else if (cnt <= (uint32_t)kLocalSort) {
      apply_sorted<kLocalSort>(rec, cnt, D, W, S2);
    } else {
      // the observations in point order without moving them: each pass over the voxel's records keeps the 8
      // smallest keys above the last one applied in a sorted register array, then applies them (a voxel's keys are
      // distinct: one observation per ray); reads only, so the records stay in L1
      uint32_t last = 0;
      bool started = false;
      for (uint32_t done = 0; done < cnt;) {
        uint32_t a[8], d[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          a[j] = 0xFFFFFFFFu;
          d[j] = 0u;
        }
        for (uint32_t i = 0; i < cnt; ++i) {
          const uint2 r = rec[i];
          uint32_t kk = r.x, dd = r.y;
          if (started && kk <= last) continue;
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            if (kk < a[j]) {
              const uint32_t tk = a[j], td = d[j];
              a[j] = kk;
              d[j] = dd;
              kk = tk;
              dd = td;
            }
          }
        }
        const uint32_t take = cnt - done < 8u ? cnt - done : 8u;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if ((uint32_t)j < take) {
            float Wn;
            welford<FP16>(__uint_as_float(d[j]), D, W, S2, Wn);
            last = a[j];
          }
        }
        started = true;
        done += take;
      }
    }
  }

  // The lane's 4 voxels: the observations of one voxel are applied in point order (each ray observes a voxel at most
  // once, so the keys of one voxel are distinct). One or two observations (90 % of observed voxels in a street scan)
  // are handled with the first two records of all 4 voxels loaded up front and the order decided in registers.
  __device__ inline int apply(const MapDev&, const Ctx& x, int vi0, Chunk& ch, int& n_vox, int& n_def) const {
    const int warp = threadIdx.x >> 5;
    const uint32_t* off = sm->off[warp];
    const int bin0 = x.g * x.nv + vi0;
    uint32_t o[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) o[k] = off[bin0 + k];
    uint2 a[4], b[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t cnt = o[k + 1] - o[k];
      a[k] = cnt >= 1 ? recs[o[k]] : make_uint2(0u, 0u);
      b[k] = cnt >= 2 ? recs[o[k] + 1] : make_uint2(0u, 0u);
    }
    int n_upd = 0;
    n_vox = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t cnt = o[k + 1] - o[k];
      n_upd += (int)cnt;
      n_vox += cnt > 0 ? 1 : 0;
      vmax = max(vmax, cnt);
      if (cnt <= 2) {
        const bool sw = cnt == 2 && a[k].x > b[k].x;
        const uint32_t d1 = sw ? b[k].y : a[k].y, d2 = sw ? a[k].y : b[k].y;
        float Wn;
        if (cnt >= 1) welford<FP16>(__uint_as_float(d1), ch.D[k], ch.W[k], ch.S2[k], Wn);
        if (cnt == 2) welford<FP16>(__uint_as_float(d2), ch.D[k], ch.W[k], ch.S2[k], Wn);
      } else if (x.l == 0) {
        // deferred: counted when applied
        const uint32_t q = atomicAdd(&sm->n_deferred[warp], 1u);
        sm->fill[warp][q] = (uint32_t)(bin0 + k);
        n_upd -= (int)cnt;
        n_vox -= 1;
        ++n_def;
      } else {
        apply_long(recs + o[k], cnt, ch.D[k], ch.W[k], ch.S2[k]);
      }
    }
    return n_upd;
  }
};

// -------------------------------------------------------------------------------------------- warp fusion body

template <bool FP16, bool COLOR>
struct BlockIO {
  uint8_t* blk;
  int nv;
  __device__ inline void load(int i4, Chunk& ch) const {
    Field<FP16>::load4(blk, i4, ch.D);
    Field<false>::load4(blk + off_W(nv, FP16, COLOR), i4, ch.W);
    Field<false>::load4(blk + off_S2(nv, FP16, COLOR), i4, ch.S2);
    if constexpr (COLOR) {
#pragma unroll
      for (int q = 0; q < 3; ++q) Field<FP16>::load4(blk + off_C(nv, FP16, q), i4, ch.C[q]);
    }
  }
  __device__ inline void store(int i4, const Chunk& ch) const {
    Field<FP16>::store4(blk, i4, ch.D);
    Field<false>::store4(blk + off_W(nv, FP16, COLOR), i4, ch.W);
    Field<false>::store4(blk + off_S2(nv, FP16, COLOR), i4, ch.S2);
    if constexpr (COLOR) {
#pragma unroll
      for (int q = 0; q < 3; ++q) Field<FP16>::store4(blk + off_C(nv, FP16, q), i4, ch.C[q]);
    }
  }
};

__device__ inline void zero_chunk(Chunk& ch) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    ch.D[k] = ch.W[k] = ch.S2[k] = 0.0f;
    ch.C[0][k] = ch.C[1][k] = ch.C[2][k] = 0.0f;
  }
}

// merge (Sec. 3.2.1, Fig. 4a): coarse voxel = W-weighted pool of its observed 2x2x2 children of block `src`;
// W = max child weight; S2 = pooled variance times W. Lanes li, li + G, ... of the group write coarse voxels.
template <bool FP16, bool COLOR>
__device__ void merge_block(const uint8_t* src, int nl, uint8_t* dst, int li, int G) {
  using F = Field<FP16>;
  const int nv = nl * nl * nl, nc = nl / 2, nvc = nc * nc * nc;
  const float* sW = reinterpret_cast<const float*>(src + off_W(nv, FP16, COLOR));
  const float* sS = reinterpret_cast<const float*>(src + off_S2(nv, FP16, COLOR));
  for (int ci = li; ci < nvc; ci += G) {
    const int cx = ci % nc, cy = (ci / nc) % nc, cz = ci / (nc * nc);
    float sw = 0.f, swd = 0.f, ss2 = 0.f, wmax = 0.f, swc[3] = {0.f, 0.f, 0.f};
    for (int q = 0; q < 8; ++q) {
      const int ch = (2 * cx + (q & 1)) + nl * ((2 * cy + ((q >> 1) & 1)) + nl * (2 * cz + (q >> 2)));
      const float Wi = sW[ch];
      if (!(Wi > 0.0f)) continue;
      sw = sw + Wi;
      swd = swd + Wi * F::get1(src, ch);
      ss2 = ss2 + sS[ch];
      if (Wi > wmax) wmax = Wi;
      if constexpr (COLOR) {
#pragma unroll
        for (int c = 0; c < 3; ++c) swc[c] = swc[c] + Wi * F::get1(src + off_C(nv, FP16, c), ch);
      }
    }
    float oD = 0.f, oW = 0.f, oS = 0.f, oC[3] = {0.f, 0.f, 0.f};
    if (sw > 0.0f) {
      const float var = ss2 / sw;
      oD = swd / sw;
      oW = wmax;
      oS = var * wmax;
      if constexpr (COLOR) {
#pragma unroll
        for (int c = 0; c < 3; ++c) oC[c] = swc[c] / sw;
      }
    }
    F::store1(dst, ci, oD);
    reinterpret_cast<float*>(dst + off_W(nvc, FP16, COLOR))[ci] = oW;
    reinterpret_cast<float*>(dst + off_S2(nvc, FP16, COLOR))[ci] = oS;
    if constexpr (COLOR) {
#pragma unroll
      for (int c = 0; c < 3; ++c) F::store1(dst + off_C(nvc, FP16, c), ci, oC[c]);
    }
  }
}

// split (extension): fine voxel = trilinear interpolation of the observed coarse voxels at its centre (clamped to
// the block); W and S2 from the coarse voxel that contains it.
template <bool FP16, bool COLOR>
__device__ void split_block(const uint8_t* src, int nc, uint8_t* dst, int li, int G) {
  using F = Field<FP16>;
  const int nv = nc * nc * nc, nf = 2 * nc, nvf = nf * nf * nf;
  const float* sW = reinterpret_cast<const float*>(src + off_W(nv, FP16, COLOR));
  const float* sS = reinterpret_cast<const float*>(src + off_S2(nv, FP16, COLOR));
  for (int fi = li; fi < nvf; fi += G) {
    const int f[3] = {fi % nf, (fi / nf) % nf, fi / (nf * nf)};
    int i0[3];
    float fr[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float p = (float)f[a] * 0.5f - 0.25f;
      if (p < 0.0f) p = 0.0f;
      if (p > (float)(nc - 1)) p = (float)(nc - 1);
      int i = (int)floorf(p);
      if (i > nc - 2) i = nc - 2;
      i0[a] = i;
      fr[a] = p - (float)i;
    }
    float sw = 0.f, sd = 0.f, sc[3] = {0.f, 0.f, 0.f};
    for (int q = 0; q < 8; ++q) {
      const int ax = q & 1, ay = (q >> 1) & 1, az = q >> 2;
      const int cv = (i0[0] + ax) + nc * ((i0[1] + ay) + nc * (i0[2] + az));
      if (!(sW[cv] > 0.0f)) continue;
      const float wx = ax ? fr[0] : 1.0f - fr[0];
      const float wy = ay ? fr[1] : 1.0f - fr[1];
      const float wz = az ? fr[2] : 1.0f - fr[2];
      const float w = wx * wy * wz;
      sw = sw + w;
      sd = sd + w * F::get1(src, cv);
      if constexpr (COLOR) {
#pragma unroll
        for (int c = 0; c < 3; ++c) sc[c] = sc[c] + w * F::get1(src + off_C(nv, FP16, c), cv);
      }
    }
    const int own = (f[0] >> 1) + nc * ((f[1] >> 1) + nc * (f[2] >> 1));
    float oD, oC[3] = {0.f, 0.f, 0.f};
    if (sw > 0.0f) {
      oD = sd / sw;
      if constexpr (COLOR) {
#pragma unroll
        for (int c = 0; c < 3; ++c) oC[c] = sc[c] / sw;
      }
    } else {
      oD = F::get1(src, own);
      if constexpr (COLOR) {
#pragma unroll
        for (int c = 0; c < 3; ++c) oC[c] = F::get1(src + off_C(nv, FP16, c), own);
      }
    }
    F::store1(dst, fi, oD);
    reinterpret_cast<float*>(dst + off_W(nvf, FP16, COLOR))[fi] = sW[own];
    reinterpret_cast<float*>(dst + off_S2(nvf, FP16, COLOR))[fi] = sS[own];
    if constexpr (COLOR) {
#pragma unroll
      for (int c = 0; c < 3; ++c) F::store1(dst + off_C(nvf, FP16, c), fi, oC[c]);
    }
  }
}

// Work items of this frame: one per level-0 block, one per two level-1 blocks, one per sixteen level-2 blocks.
struct ItemCounts {
  uint32_t n0, n1, n2, it0, it1, it2;
  __device__ inline uint32_t items() const { return it0 + it1 + it2; }
};

__device__ inline ItemCounts item_counts(const MapDev& m) {
  ItemCounts c;
  c.n0 = min(m.st->touched_count[0], m.max_touched);
  c.n1 = m.L > 1 ? min(m.st->touched_count[1], m.max_touched) : 0;
  c.n2 = m.L > 2 ? min(m.st->touched_count[2], m.max_touched) : 0;
  c.it0 = c.n0;
  c.it1 = (c.n1 + 1) / 2;
  c.it2 = (c.n2 + 15) / 16;
  return c;
}

// One work item, processed by the whole warp (warp-uniform control flow). my_obs / my_vox: the lane's running
// counts of observations and updated voxels (Acc: 32 bits where a caller flushes them per map and frame).
template <bool FP16, bool COLOR, class Obs, class Acc = unsigned long long>
__device__ inline void fuse_item(const MapDev& m, Obs& obs, int warp_in_cta, const ItemCounts& ic, uint32_t item,
                                 Acc& my_obs, Acc& my_vox) {
  const int lane = threadIdx.x & 31;
  const uint32_t n0 = ic.n0, n1 = ic.n1, n2 = ic.n2, it0 = ic.it0, it1 = ic.it1;
  {
    Ctx x;
    uint32_t first, count, pbase;
    if (item < it0) { x.l = 0; first = item; count = n0; pbase = 0; }
    else if (item < it0 + it1) { x.l = 1; first = (item - it0) * 2; count = n1; pbase = n0; }
    else { x.l = 2; first = (item - it0 - it1) * 16; count = n2; pbase = n0 + n1; }
    x.nl = kFineDim >> x.l;
    x.nv = x.nl * x.nl * x.nl;
    x.G = x.nv < 128 ? x.nv / 4 : 32;  // lanes per block: 32, 16, 2
    x.g = lane / x.G;
    x.li = lane % x.G;
    const uint32_t idx = first + x.g;
    x.active = idx < count;
    x.P = pbase + idx;
    x.P_first = pbase + first;
    const int l = x.l, nl = x.nl, nv = x.nv, G = x.G, li = x.li;
    const int chunks = nv / (4 * G);  // 4, 1, 1

    BlockMeta bm;
    bm.key = 0;
    bm.val = 0;
    bm.slot = 0;
    if (x.active) bm = m.meta[l][idx];
    const bool isnew = (bm.val & kValNew) != 0;
    const uint32_t ptr = bm.val & kPtrMask;
    unpack_key(bm.key, &x.kx, &x.ky, &x.kz);
    const BlockIO<FP16, COLOR> io{m.heap[l] + (size_t)ptr * m.block_bytes[l], nv};
    const bool load = x.active && !isnew;

    obs.collect(m, x, warp_in_cta);

    // ---- chunks: load, update, write back (when changed), accumulate block statistics
    float vsum = 0.f;
    int nobs = 0;
    uint32_t sumw32 = 0;  // at most 16 voxels per lane, each W < 2^24
    float dmn = __int_as_float(0x7f800000);  // least stored D over observed voxels (+inf: none)
    // one chunk in registers at a time: at 64 registers a thread, 4 CTAs of 8 warps share an SM and their
    // interleaving hides the load latency better than a register double buffer at 3 CTAs (measured)
    Chunk cur;
    for (int c = 0; c < chunks; ++c) {
      if (load) io.load(c * G + li, cur);
      else zero_chunk(cur);
      int n_def = 0;
      if (x.active) {
        int n_vox = 0;
        my_obs += (Acc)obs.apply(m, x, 4 * (c * G + li), cur, n_vox, n_def);
        my_vox += (Acc)n_vox;
        // a chunk without an update is unchanged in memory, unless the block is new (zero state to write)
        if (n_vox > 0 || isnew) io.store(c * G + li, cur);
      }
      // (a deferred voxel still holds its value before this frame here: a value it can only lower the least D by,
      // and its final value joins when it is applied)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (cur.W[q] > 0.0f) dmn = fminf(dmn, cur.D[q]);
      bool counted = false;
      if constexpr (Obs::kDefers) {
        if (n_def) {
          // a chunk with deferred voxels: the others are counted now, the deferred ones once applied
          const int vi0 = 4 * (c * G + li);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            uint32_t cnt = 0;
            obs.range(warp_in_cta, (uint32_t)(x.g * nv + vi0 + q), &cnt);
            if (cnt < 3 && cur.W[q] > 0.0f) {
              vsum = vsum + __fdividef(cur.S2[q], cur.W[q]);
              nobs += 1;
              sumw32 += (uint32_t)cur.W[q];
            }
          }
          counted = true;
        }
      }
      if (!counted) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (cur.W[q] > 0.0f) {
            vsum = vsum + __fdividef(cur.S2[q], cur.W[q]);  // estimate only (see the error bound above)
            nobs += 1;
            sumw32 += (uint32_t)cur.W[q];
          }
        }
      }
    }
    if constexpr (Obs::kDefers) {
      // deferred voxels of a level-0 item: one voxel per lane, state read from and written back to the block
      const int n_deferred = obs.take_deferred(x, warp_in_cta);
      for (int q = li; q < n_deferred; q += G) {
        const uint32_t bin = obs.deferred(warp_in_cta, q);
        uint32_t cnt = 0;
        const uint32_t o0 = obs.range(warp_in_cta, bin, &cnt);
        float* Wp = reinterpret_cast<float*>(io.blk + off_W(nv, FP16, COLOR)) + bin;
        float* Sp = reinterpret_cast<float*>(io.blk + off_S2(nv, FP16, COLOR)) + bin;
        float D = Field<FP16>::get1(io.blk, (int)bin), W = *Wp, S2 = *Sp;
        Obs::apply_long(obs.recs + o0, cnt, D, W, S2);
        obs.vmax = max(obs.vmax, cnt);
        Field<FP16>::store1(io.blk, (int)bin, D);
        *Wp = W;
        *Sp = S2;
        my_obs += cnt;
        my_vox += 1;
        vsum = vsum + __fdividef(S2, W);
        nobs += 1;
        sumw32 += (uint32_t)W;
        dmn = fminf(dmn, D);
      }
    }
    long long sumw = sumw32;
    for (int o = G / 2; o > 0; o >>= 1) {
      vsum = vsum + __shfl_xor_sync(~0u, vsum, o);
      nobs += __shfl_xor_sync(~0u, nobs, o);
      sumw += __shfl_xor_sync(~0u, sumw, o);
      dmn = fminf(dmn, __shfl_xor_sync(~0u, dmn, o));
    }
    if (x.active && li == 0) m.dmin[l][ptr] = dmn;

    // ---- decision (every lane of the group computes the same one)
    // Outside the band the float estimate and the float threshold are on the same side as the exact values (the
    // estimate is within 1.5e-6 and the float threshold within 6e-8, relative), so the float comparison decides.
    int act = kActNone;
    bool recheck = false;
    const float vb = nobs > 0 ? vsum / (float)nobs : 0.0f;
    const bool eligible = x.active && nobs > 0 && sumw >= (long long)m.min_obs * nobs;
    const bool can_merge = eligible && l < m.L - 1;
    const bool can_split = eligible && m.split_h > 0.0 && l > 0;
    const float thr_mf = m.thr_merge_f[l], thr_sf = m.thr_split_f[l];
    if (can_merge) recheck |= fabsf(vb - thr_mf) <= kBandF * fabsf(thr_mf);
    if (can_split) recheck |= fabsf(vb - thr_sf) <= kBandF * fabsf(thr_sf);
    double exact = 0.0;
    const int leader = lane - li;
    if (__any_sync(~0u, recheck)) {
      __syncwarp();  // the group's payload writes are visible to its leader
      if (recheck && li == 0) {
        const float* W = reinterpret_cast<const float*>(io.blk + off_W(nv, FP16, COLOR));
        const float* S = reinterpret_cast<const float*>(io.blk + off_S2(nv, FP16, COLOR));
        double acc = 0.0;
        for (int i = 0; i < nv; ++i) {
          const float w = W[i];
          if (w > 0.0f) acc = acc + (double)S[i] / (double)w;
        }
        exact = acc / (double)nobs;
        atomicAdd(&m.st->rechecks, 1u);
      }
      exact = __shfl_sync(~0u, exact, leader);
    }
    if (can_merge && (recheck ? exact < m.thr_merge[l] : vb < thr_mf)) act = kActMerge;
    else if (can_split && (recheck ? exact > m.thr_split[l] : vb > thr_sf)) act = kActSplit;

    // ---- re-level (rare): pop a heap block of the target level, resample into it, retire the old block
    if (__any_sync(~0u, act != kActNone)) {
      uint32_t newptr = 0;
      if (act != kActNone && li == 0) {
        const int lt = act == kActMerge ? l + 1 : l - 1;
        const int t = atomicSub(&m.st->free_top[lt], 1);
        if (t <= 0) {
          atomicAdd(&m.st->free_top[lt], 1);
          set_status(m.st, kStPoolEmpty);
          newptr = kInvalidPtr;
        } else {
          newptr = m.free_stack[lt][t - 1];
        }
      }
      newptr = __shfl_sync(~0u, newptr, leader);
      if (newptr == kInvalidPtr) act = kActNone;
      __syncwarp();  // the group's payload writes are visible to every lane that resamples them
      if (act == kActMerge) {
        merge_block<FP16, COLOR>(io.blk, nl, m.heap[l + 1] + (size_t)newptr * m.block_bytes[l + 1], li, G);
      } else if (act == kActSplit) {
        split_block<FP16, COLOR>(io.blk, nl, m.heap[l - 1] + (size_t)newptr * m.block_bytes[l - 1], li, G);
      }
      if (act != kActNone && li == 0) {
        const int lt = act == kActMerge ? l + 1 : l - 1;
        // the resampled payload holds weighted means of the observed voxels: its least D is at least this one
        m.dmin[lt][newptr] = dmn;
        m.slots[bm.slot].val = newptr | ((uint32_t)lt << 28);
        const uint32_t r = atomicAdd(&m.st->retire_count, 1u);
        m.retire[r] = ptr | ((uint32_t)l << 28);
        atomicAdd(act == kActMerge ? &m.st->merged : &m.st->split, 1u);
      }
    }
    if (act == kActNone && isnew && x.active && li == 0) m.slots[bm.slot].val = bm.val & ~kValNew;
  }
}

// A warp's share of the items of one map (grid-strided), then the observation counter.
template <bool FP16, bool COLOR, class Obs>
__device__ inline void fuse_warp_body(const MapDev& m, Obs& obs, int warp_in_cta, uint32_t warp_id, uint32_t nwarps) {
  const int lane = threadIdx.x & 31;
  const ItemCounts ic = item_counts(m);
  const uint32_t items = ic.items();
  unsigned long long my_obs = 0, my_vox = 0;
  for (uint32_t item = warp_id; item < items; item += nwarps)
    fuse_item<FP16, COLOR>(m, obs, warp_in_cta, ic, item, my_obs, my_vox);
  for (int o = 16; o > 0; o >>= 1) {
    my_obs += __shfl_xor_sync(~0u, my_obs, o);
    my_vox += __shfl_xor_sync(~0u, my_vox, o);
  }
  if (lane == 0 && my_obs) atomicAdd(&m.st->observations, my_obs);
  if (lane == 0 && my_vox) atomicAdd(&m.st->updated_voxels, my_vox);
}

}  // namespace
}  // namespace mrh
