// Fusion of one frame into the touched blocks, the block variance and re-levelling, in one pass.
//
//   camera  (Sec. 3.1 "Cameras", Eq. 2): every voxel of a touched block projects to its nearest pixel; the signed
//           distance is the pixel's range minus the voxel's distance, occluded voxels (more than tau behind) are
//           skipped, the rest clipped to tau.
//   LiDAR   (Sec. 3.1 "3D Point Cloud", Eq. 1): each ray walks the voxels of its truncation band (a DDA over
//           finest-level cells, one observation per voxel of the block's own level); d = clip((p - x) . n, tau).
//           Observations are counted per block, prefix-summed and scattered; inside a block they are binned per
//           voxel and each voxel applies its observations in ascending point index, so the result does not depend on
//           scheduling.
//   both    running mean (Eq. 3, w_k = 1) in Welford's incremental form and S2 += (d - D_old)(d - D_new)
//           (Sec. 3.2.1); then the mean voxel variance of the block over observed voxels; then merge to the next
//           coarser level below theta_l (Sec. 3.2.1, Fig. 4a) or split to the next finer level above h theta_{l-1}.
//
// Work decomposition: a CTA of 128 threads takes 512 voxels per step: one level-0 block (8^3), eight level-1
// blocks (4^3) or sixty-four level-2 blocks (2^3). Each thread owns 4 consecutive voxels and moves each field of
// them with one 16-byte (fp32) or 8-byte (fp16) access, so a block's fields stream fully coalesced. The updated state
// is staged in shared memory, the block variance is reduced with warp shuffles, and a block that changes level is
// resampled from shared memory straight into a block popped from the other level's heap (a merged block never
// writes its fine payload back).
//
// The block variance decides in float; a value within 4e-6 (relative) of a threshold is recomputed in double, in
// voxel order, exactly as the CPU oracle computes it, so level decisions match the oracle bit for bit. (The float
// sum's relative error is below 13 ulp: <= 3 sequential + 5 shuffle + 3 cross-warp additions of non-negative terms,
// the per-voxel division and the final division.)
//
// This file is compiled without multiply-add contraction: float expressions round in source order, like the oracle.
#include <cuda_fp16.h>

#include "mrh_internal.cuh"

namespace mrh {
namespace {

constexpr int kThreads = 128;
constexpr double kBand = 4e-6;
constexpr int kLocalSort = 16;
enum { kActNone = 0, kActMerge = 1, kActSplit = 2 };

template <bool FP16>
struct Field {
  static __device__ inline void load4(const uint8_t* p, int li, float out[4]) {
    if constexpr (FP16) {
      uint2 u = reinterpret_cast<const uint2*>(p)[li];
      __half2 a = *reinterpret_cast<__half2*>(&u.x), b = *reinterpret_cast<__half2*>(&u.y);
      float2 fa = __half22float2(a), fb = __half22float2(b);
      out[0] = fa.x; out[1] = fa.y; out[2] = fb.x; out[3] = fb.y;
    } else {
      float4 f = reinterpret_cast<const float4*>(p)[li];
      out[0] = f.x; out[1] = f.y; out[2] = f.z; out[3] = f.w;
    }
  }
  static __device__ inline void store4(uint8_t* p, int li, const float in[4]) {
    if constexpr (FP16) {
      __half2 a = __floats2half2_rn(in[0], in[1]), b = __floats2half2_rn(in[2], in[3]);
      uint2 u;
      u.x = *reinterpret_cast<uint32_t*>(&a);
      u.y = *reinterpret_cast<uint32_t*>(&b);
      reinterpret_cast<uint2*>(p)[li] = u;
    } else {
      reinterpret_cast<float4*>(p)[li] = make_float4(in[0], in[1], in[2], in[3]);
    }
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

// What one CTA step knows about the block its thread group works on.
struct Ctx {
  int l, nl, nv, G, g, li;
  bool active;
  uint32_t idx;         // position in touched[l]
  uint32_t P;           // position in the level-concatenated list (LiDAR buffers)
  uint32_t P_first;     // P of the CTA step's first group
  int kx, ky, kz;       // block key
};

// One Welford step (Eq. 3 incremental form + S2 update of Sec. 3.2.1).
template <bool FP16>
__device__ inline void welford(float d, float& D, float& W, float& S2, float& Wn) {
  Wn = W + 1.0f;
  float e = d - D;
  float Dn = D + e / Wn;
  S2 = S2 + e * (d - Dn);
  D = Field<FP16>::kept(Dn);
  W = Wn;
}

// -------------------------------------------------------------------------------------------- camera observer

template <bool FP16, bool COLOR>
struct CameraObs {
  CamArgs c;
  const float* depth;
  const uint8_t* rgb;

  __device__ inline void collect(const MapDev&, const Ctx&) {}

  __device__ inline int apply(const MapDev& m, const Ctx& x, float D[4], float W[4], float S2[4], float C[3][4]) {
    if (!x.active) return 0;
    const float vl = m.v[x.l];
    const float ob0 = (float)x.kx * m.E - c.t[0];
    const float ob1 = (float)x.ky * m.E - c.t[1];
    const float ob2 = (float)x.kz * m.E - c.t[2];
    int n_upd = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int vi = 4 * x.li + k;
      const int xi = vi % x.nl, yi = (vi / x.nl) % x.nl, zi = vi / (x.nl * x.nl);
      float w0 = ob0 + ((float)xi + 0.5f) * vl;
      float w1 = ob1 + ((float)yi + 0.5f) * vl;
      float w2 = ob2 + ((float)zi + 0.5f) * vl;
      float xc = c.R[0] * w0 + c.R[3] * w1 + c.R[6] * w2;
      float yc = c.R[1] * w0 + c.R[4] * w1 + c.R[7] * w2;
      float zc = c.R[2] * w0 + c.R[5] * w1 + c.R[8] * w2;
      if (!(zc > 0.0f)) continue;
      float uf = c.fx * xc / zc + c.cx + 0.5f;
      float vf = c.fy * yc / zc + c.cy + 0.5f;
      if (!(uf >= 0.0f && uf < (float)c.width && vf >= 0.0f && vf < (float)c.height)) continue;
      int u = (int)floorf(uf), v = (int)floorf(vf);
      size_t pix = (size_t)v * c.width + u;
      float zm = __ldg(depth + pix);
      if (!(zm >= c.min_depth && zm <= c.max_depth)) continue;
      float qx = ((float)u - c.cx) / c.fx, qy = ((float)v - c.cy) / c.fy;
      float rho = zm * sqrtf(qx * qx + qy * qy + 1.0f);
      float dist = sqrtf(xc * xc + yc * yc + zc * zc);
      float eta = rho - dist;
      if (eta < -m.tau) continue;  // occluded: more than tau behind the measured surface
      float d = eta < m.tau ? eta : m.tau;
      float Wn;
      welford<FP16>(d, D[k], W[k], S2[k], Wn);
      if constexpr (COLOR) {
        if (rgb) {
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            float col = (float)__ldg(rgb + 3 * pix + q);
            float ec = col - C[q][k];
            C[q][k] = Field<FP16>::kept(C[q][k] + ec / Wn);
          }
        }
      }
      ++n_upd;
    }
    return n_upd;
  }
};

// -------------------------------------------------------------------------------------------- LiDAR observer

template <bool FP16>
struct LidarObs {
  uint32_t* s_cnt;
  uint32_t* s_off;
  uint32_t item_base;

  // CTA-collective: bin this step's observations per voxel (bins are the step's 512 voxels).
  __device__ inline void collect(const MapDev& m, const Ctx& x) {
    uint32_t* s_fill = s_off + 512;
    for (int i = threadIdx.x; i < 512; i += kThreads) {
      s_cnt[i] = 0;
      s_fill[i] = 0;
    }
    __syncthreads();
    uint32_t r0 = 0, r1 = 0;
    if (x.active) {
      r0 = m.blk_off[x.P];
      r1 = m.blk_off[x.P + 1];
      if (r1 > m.max_obs) r0 = r1 = 0;  // observations were not stored (status already set)
    }
    for (uint32_t r = r0 + x.li; r < r1; r += x.G) atomicAdd(&s_cnt[x.g * x.nv + (m.obs_key[r] & 511u)], 1u);
    __syncthreads();
    // exclusive scan of the 512 bin counts: 4 per thread, warp shuffle, then across the 4 warps
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t c4[4], sum = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      c4[k] = s_cnt[4 * tid + k];
      sum += c4[k];
    }
    uint32_t incl = sum;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(~0u, incl, o);
      if (lane >= o) incl += t;
    }
    __shared__ uint32_t s_w[4];
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    uint32_t base = 0;
    for (int w = 0; w < warp; ++w) base += s_w[w];
    uint32_t run = base + incl - sum;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      s_off[4 * tid + k] = run;
      run += c4[k];
    }
    item_base = m.blk_off[x.P_first];
    __syncthreads();
    for (uint32_t r = r0 + x.li; r < r1; r += x.G) {
      uint32_t bin = x.g * x.nv + (m.obs_key[r] & 511u);
      uint32_t pos = s_off[bin] + atomicAdd(&s_fill[bin], 1u);
      m.obs_idx[item_base + pos] = r;
    }
    __syncthreads();
  }

  __device__ inline int apply(const MapDev& m, const Ctx& x, float D[4], float W[4], float S2[4], float (*)[4]) {
    if (!x.active) return 0;
    int n_upd = 0;
#pragma unroll 1
    for (int k = 0; k < 4; ++k) {
      const int bin = 4 * threadIdx.x + k;
      const uint32_t cnt = s_cnt[bin];
      if (cnt == 0) continue;
      uint32_t* idx = m.obs_idx + item_base + s_off[bin];
      // order the voxel's observations by point index (each ray observes a voxel at most once)
      if (cnt <= kLocalSort) {
        unsigned long long e[kLocalSort];
        for (uint32_t i = 0; i < cnt; ++i) {
          uint32_t r = idx[i];
          unsigned long long key = ((unsigned long long)(m.obs_key[r] >> 9) << 32) | r;
          uint32_t j = i;
          while (j > 0 && e[j - 1] > key) {
            e[j] = e[j - 1];
            --j;
          }
          e[j] = key;
        }
        for (uint32_t i = 0; i < cnt; ++i) {
          float Wn;
          welford<FP16>(m.obs_d[(uint32_t)e[i]], D[k], W[k], S2[k], Wn);
        }
      } else {
        for (uint32_t i = 1; i < cnt; ++i) {
          uint32_t r = idx[i];
          uint32_t kr = m.obs_key[r] >> 9;
          uint32_t j = i;
          while (j > 0 && (m.obs_key[idx[j - 1]] >> 9) > kr) {
            idx[j] = idx[j - 1];
            --j;
          }
          idx[j] = r;
        }
        for (uint32_t i = 0; i < cnt; ++i) {
          float Wn;
          welford<FP16>(m.obs_d[idx[i]], D[k], W[k], S2[k], Wn);
        }
      }
      n_upd += (int)cnt;
    }
    return n_upd;
  }
};

// -------------------------------------------------------------------------------------------- generic fusion kernel

template <bool FP16, bool COLOR, class Obs>
__device__ inline void fuse_body(const MapDev& m, Obs& obs) {
  using F = Field<FP16>;
  __shared__ float sD[512], sW[512], sS2[512];
  __shared__ float sC[COLOR ? 3 : 1][COLOR ? 512 : 1];
  __shared__ int s_act[64];
  __shared__ uint32_t s_ptr[64];
  __shared__ float s_rv[4];
  __shared__ int s_rn[4];
  __shared__ long long s_rw[4];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t n0 = min(m.st->touched_count[0], m.max_touched);
  const uint32_t n1 = m.L > 1 ? min(m.st->touched_count[1], m.max_touched) : 0;
  const uint32_t n2 = m.L > 2 ? min(m.st->touched_count[2], m.max_touched) : 0;
  const uint32_t it0 = n0, it1 = (n1 + 7) / 8, it2 = (n2 + 63) / 64;
  const uint32_t items = it0 + it1 + it2;
  unsigned long long my_obs = 0;

  for (uint32_t item = blockIdx.x; item < items; item += gridDim.x) {
    Ctx x;
    uint32_t first, count, pbase;
    if (item < it0) { x.l = 0; first = item; count = n0; pbase = 0; }
    else if (item < it0 + it1) { x.l = 1; first = (item - it0) * 8; count = n1; pbase = n0; }
    else { x.l = 2; first = (item - it0 - it1) * 64; count = n2; pbase = n0 + n1; }
    x.nl = kFineDim >> x.l;
    x.nv = x.nl * x.nl * x.nl;
    x.G = x.nv / 4;
    x.g = tid / x.G;
    x.li = tid % x.G;
    x.idx = first + x.g;
    x.active = x.idx < count;
    x.P = pbase + x.idx;
    x.P_first = pbase + first;
    const int l = x.l, nl = x.nl, nv = x.nv, G = x.G, g = x.g, li = x.li;
    const bool active = x.active;

    uint32_t slot = 0, val = 0, ptr = 0;
    bool isnew = true;
    x.kx = x.ky = x.kz = 0;
    if (active) {
      slot = m.touched[l][x.idx];
      val = m.slots[slot].val;
      ptr = val & kPtrMask;
      isnew = (val & kValNew) != 0;
      unpack_key(m.slots[slot].key, &x.kx, &x.ky, &x.kz);
    }
    uint8_t* blk = m.heap[l] + (size_t)ptr * m.block_bytes[l];
    uint8_t* pW = blk + off_W(nv, FP16, COLOR);
    uint8_t* pS = blk + off_S2(nv, FP16, COLOR);

    float D[4] = {0, 0, 0, 0}, W[4] = {0, 0, 0, 0}, S2[4] = {0, 0, 0, 0};
    float C[3][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}};
    if (active && !isnew) {
      F::load4(blk, li, D);
      Field<false>::load4(pW, li, W);
      Field<false>::load4(pS, li, S2);
      if constexpr (COLOR) {
#pragma unroll
        for (int q = 0; q < 3; ++q) F::load4(blk + off_C(nv, FP16, q), li, C[q]);
      }
    }

    obs.collect(m, x);
    my_obs += (unsigned long long)obs.apply(m, x, D, W, S2, C);

    // ---- stage in shared memory, block statistics (Sec. 3.2.1: mean voxel variance of the block)
    float vsum = 0.f;
    int nobs = 0;
    long long sumw = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int si = 4 * tid + k;  // == g * nv + 4 li + k
      sD[si] = D[k];
      sW[si] = W[k];
      sS2[si] = S2[k];
      if constexpr (COLOR) {
#pragma unroll
        for (int q = 0; q < 3; ++q) sC[q][si] = C[q][k];
      }
      if (W[k] > 0.0f) {
        vsum = vsum + S2[k] / W[k];
        nobs += 1;
        sumw += (long long)W[k];
      }
    }
    const int width = G < 32 ? G : 32;
    for (int off = width / 2; off > 0; off >>= 1) {
      vsum = vsum + __shfl_xor_sync(~0u, vsum, off);
      nobs += __shfl_xor_sync(~0u, nobs, off);
      sumw += __shfl_xor_sync(~0u, sumw, off);
    }
    if (G == 128 && lane == 0) {
      s_rv[warp] = vsum;
      s_rn[warp] = nobs;
      s_rw[warp] = sumw;
    }
    __syncthreads();
    if (li == 0) {
      if (G == 128) {
        vsum = s_rv[0] + s_rv[1] + s_rv[2] + s_rv[3];
        nobs = s_rn[0] + s_rn[1] + s_rn[2] + s_rn[3];
        sumw = s_rw[0] + s_rw[1] + s_rw[2] + s_rw[3];
      }
      int act = kActNone;
      uint32_t newptr = 0;
      // eligibility: observed, mean weight >= k_min over observed voxels
      if (active && nobs > 0 && sumw >= (long long)m.min_obs * nobs) {
        const double vb32 = (double)(vsum / (float)nobs);
        bool have_exact = false;
        double vexact = 0.0;
        auto vbar_near = [&](double thr) -> double {
          if (fabs(vb32 - thr) <= kBand * fabs(thr)) {
            if (!have_exact) {
              double acc = 0.0;
              for (int i = 0; i < nv; ++i) {
                float w = sW[g * nv + i];
                if (w > 0.0f) acc = acc + (double)sS2[g * nv + i] / (double)w;
              }
              vexact = acc / (double)nobs;
              have_exact = true;
              atomicAdd(&m.st->rechecks, 1u);
            }
            return vexact;
          }
          return vb32;
        };
        if (l < m.L - 1 && vbar_near(m.theta[l]) < m.theta[l]) {
          act = kActMerge;
        } else if (m.split_h > 0.0 && l > 0) {
          const double thr = m.split_h * m.theta[l - 1];
          if (vbar_near(thr) > thr) act = kActSplit;
        }
        if (act != kActNone) {
          const int lt = act == kActMerge ? l + 1 : l - 1;
          int t = atomicSub(&m.st->free_top[lt], 1);
          if (t <= 0) {
            atomicAdd(&m.st->free_top[lt], 1);
            set_status(m.st, kStPoolEmpty);
            act = kActNone;
          } else {
            newptr = m.free_stack[lt][t - 1];
          }
        }
      }
      s_act[g] = act;
      s_ptr[g] = newptr;
    }
    __syncthreads();

    const int act = active ? s_act[g] : kActNone;
    if (active && act == kActNone) {
      F::store4(blk, li, D);
      Field<false>::store4(pW, li, W);
      Field<false>::store4(pS, li, S2);
      if constexpr (COLOR) {
#pragma unroll
        for (int q = 0; q < 3; ++q) F::store4(blk + off_C(nv, FP16, q), li, C[q]);
      }
    } else if (act == kActMerge) {
      // coarse voxel = W-weighted pool of its observed 2x2x2 children; W = max child weight; S2 = pooled
      // variance times W
      const int nc = nl / 2, nvc = nc * nc * nc;
      uint8_t* nb = m.heap[l + 1] + (size_t)s_ptr[g] * m.block_bytes[l + 1];
      for (int ci = li; ci < nvc; ci += G) {
        const int cx = ci % nc, cy = (ci / nc) % nc, cz = ci / (nc * nc);
        float sw = 0.f, swd = 0.f, ss2 = 0.f, wmax = 0.f, swc[3] = {0.f, 0.f, 0.f};
        for (int k = 0; k < 8; ++k) {
          const int ch = g * nv + (2 * cx + (k & 1)) + nl * ((2 * cy + ((k >> 1) & 1)) + nl * (2 * cz + (k >> 2)));
          const float Wi = sW[ch];
          if (!(Wi > 0.0f)) continue;
          sw = sw + Wi;
          swd = swd + Wi * sD[ch];
          ss2 = ss2 + sS2[ch];
          if (Wi > wmax) wmax = Wi;
          if constexpr (COLOR) {
#pragma unroll
            for (int q = 0; q < 3; ++q) swc[q] = swc[q] + Wi * sC[q][ch];
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
            for (int q = 0; q < 3; ++q) oC[q] = swc[q] / sw;
          }
        }
        F::store1(nb, ci, oD);
        reinterpret_cast<float*>(nb + off_W(nvc, FP16, COLOR))[ci] = oW;
        reinterpret_cast<float*>(nb + off_S2(nvc, FP16, COLOR))[ci] = oS;
        if constexpr (COLOR) {
#pragma unroll
          for (int q = 0; q < 3; ++q) F::store1(nb + off_C(nvc, FP16, q), ci, oC[q]);
        }
      }
    } else if (act == kActSplit) {
      // fine voxel = trilinear interpolation of the observed coarse voxels at its centre (clamped to the block);
      // W and S2 from the coarse voxel that contains it
      const int nc = nl, nf = 2 * nl, nvf = nf * nf * nf;
      uint8_t* nb = m.heap[l - 1] + (size_t)s_ptr[g] * m.block_bytes[l - 1];
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
        for (int k = 0; k < 8; ++k) {
          const int ax = k & 1, ay = (k >> 1) & 1, az = k >> 2;
          const int cv = g * nv + (i0[0] + ax) + nc * ((i0[1] + ay) + nc * (i0[2] + az));
          if (!(sW[cv] > 0.0f)) continue;
          const float wx = ax ? fr[0] : 1.0f - fr[0];
          const float wy = ay ? fr[1] : 1.0f - fr[1];
          const float wz = az ? fr[2] : 1.0f - fr[2];
          const float w = wx * wy * wz;
          sw = sw + w;
          sd = sd + w * sD[cv];
          if constexpr (COLOR) {
#pragma unroll
            for (int q = 0; q < 3; ++q) sc[q] = sc[q] + w * sC[q][cv];
          }
        }
        const int own = g * nv + (f[0] >> 1) + nc * ((f[1] >> 1) + nc * (f[2] >> 1));
        float oD, oC[3] = {0.f, 0.f, 0.f};
        if (sw > 0.0f) {
          oD = sd / sw;
          if constexpr (COLOR) {
#pragma unroll
            for (int q = 0; q < 3; ++q) oC[q] = sc[q] / sw;
          }
        } else {
          oD = sD[own];
          if constexpr (COLOR) {
#pragma unroll
            for (int q = 0; q < 3; ++q) oC[q] = sC[q][own];
          }
        }
        F::store1(nb, fi, oD);
        reinterpret_cast<float*>(nb + off_W(nvf, FP16, COLOR))[fi] = sW[own];
        reinterpret_cast<float*>(nb + off_S2(nvf, FP16, COLOR))[fi] = sS2[own];
        if constexpr (COLOR) {
#pragma unroll
          for (int q = 0; q < 3; ++q) F::store1(nb + off_C(nvf, FP16, q), fi, oC[q]);
        }
      }
    }
    if (active && li == 0) {
      if (act != kActNone) {
        const int lt = act == kActMerge ? l + 1 : l - 1;
        m.slots[slot].val = s_ptr[g] | ((uint32_t)lt << 28);
        uint32_t r = atomicAdd(&m.st->retire_count, 1u);
        m.retire[r] = ptr | ((uint32_t)l << 28);
        atomicAdd(act == kActMerge ? &m.st->merged : &m.st->split, 1u);
      } else if (isnew) {
        m.slots[slot].val = val & ~kValNew;
      }
    }
    __syncthreads();
  }
  for (int off = 16; off > 0; off >>= 1) my_obs += __shfl_xor_sync(~0u, my_obs, off);
  if (lane == 0 && my_obs) atomicAdd(&m.st->observations, my_obs);
}

template <bool FP16, bool COLOR>
__global__ void __launch_bounds__(kThreads) k_fuse_depth(MapDev m, CamArgs c, const float* __restrict__ depth,
                                                         const uint8_t* __restrict__ rgb) {
  CameraObs<FP16, COLOR> obs{c, depth, rgb};
  fuse_body<FP16, COLOR>(m, obs);
}

template <bool FP16, bool COLOR>
__global__ void __launch_bounds__(kThreads) k_fuse_points(MapDev m) {
  __shared__ uint32_t s_cnt[512], s_off[1024];
  LidarObs<FP16> obs{s_cnt, s_off, 0};
  fuse_body<FP16, COLOR>(m, obs);
}

// -------------------------------------------------------------------------------------------- LiDAR observation passes

// FILL = false: count each block's observations; FILL = true: write them (point index, voxel, d).
template <bool FILL>
__global__ void __launch_bounds__(128) k_lidar_walk(MapDev m, PoseD P, const float* __restrict__ xyz, uint64_t n) {
  const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  long long A[3], B[3];
  double rho;
  double rhat[3];
  if (!lidar_ray(m, P, xyz, j, A, B, &rho, rhat)) return;
  const uint32_t n0 = min(m.st->touched_count[0], m.max_touched);
  const uint32_t n1 = min(m.st->touched_count[1], m.max_touched);
  const float rho_f = (float)rho;
  const float rh[3] = {(float)rhat[0], (float)rhat[1], (float)rhat[2]};
  const float o_f[3] = {(float)P.T[3], (float)P.T[7], (float)P.T[11]};

  long long cb[3] = {0, 0, 0}, lg[3] = {0, 0, 0};
  bool have_block = false, cur_ok = false, have_last = false;
  int cl = 0;
  uint32_t cur_P = 0, run = 0;
  float ob[3] = {0.f, 0.f, 0.f};
  constexpr int kRunCap = 32;
  uint32_t rk[FILL ? kRunCap : 1];
  float rd[FILL ? kRunCap : 1];

  auto flush = [&]() {
    if (!cur_ok || run == 0) return;
    if constexpr (!FILL) {
      atomicAdd(&m.blk_count[cur_P], run);
    } else {
      uint32_t base = m.blk_off[cur_P] + atomicAdd(&m.blk_fill[cur_P], run);
      if (base + run <= m.max_obs) {
        for (uint32_t i = 0; i < run; ++i) {
          m.obs_key[base + i] = rk[i];
          m.obs_d[base + i] = rd[i];
        }
      } else {
        set_status(m.st, kStObsFull);
      }
    }
    run = 0;
  };

  bool ok = walk_cells(A, B, kVoxelUnit, kMaxVoxelCells, [&](const long long* f) {
    long long bk[3] = {floor_div(f[0], kFineDim), floor_div(f[1], kFineDim), floor_div(f[2], kFineDim)};
    if (!have_block || bk[0] != cb[0] || bk[1] != cb[1] || bk[2] != cb[2]) {
      flush();
      have_block = true;
      cb[0] = bk[0]; cb[1] = bk[1]; cb[2] = bk[2];
      have_last = false;
      cur_ok = false;
      int s = lookup_slot(m.slots, m.slot_mask, pack_key(bk[0], bk[1], bk[2]));
      if (s >= 0) {
        uint32_t val = m.slots[s].val;
        if (val != kValPending) {
          uint32_t sp = m.slot_pos[s];
          uint32_t lv = sp >> 28, jj = sp & kPtrMask;
          // the position is this frame's only if the level list points back at the slot
          const uint32_t cnt_lv = min(m.st->touched_count[lv], m.max_touched);
          if (lv == ((val >> 28) & 3u) && (int)lv < m.L && jj < cnt_lv && m.touched[lv][jj] == (uint32_t)s) {
            cl = (int)lv;
            cur_P = jj + (lv >= 1 ? n0 : 0) + (lv >= 2 ? n1 : 0);
            cur_ok = true;
            ob[0] = (float)bk[0] * m.E - o_f[0];
            ob[1] = (float)bk[1] * m.E - o_f[1];
            ob[2] = (float)bk[2] * m.E - o_f[2];
          }
        }
      }
    }
    if (!cur_ok) return;
    long long g[3] = {floor_div(f[0], 1LL << cl), floor_div(f[1], 1LL << cl), floor_div(f[2], 1LL << cl)};
    if (have_last && g[0] == lg[0] && g[1] == lg[1] && g[2] == lg[2]) return;
    have_last = true;
    lg[0] = g[0]; lg[1] = g[1]; lg[2] = g[2];
    const int nl = kFineDim >> cl;
    const int li[3] = {(int)(g[0] - cb[0] * nl), (int)(g[1] - cb[1] * nl), (int)(g[2] - cb[2] * nl)};
    if constexpr (FILL) {
      if (run == kRunCap) flush();  // cannot happen at level 0 (<= 22 voxels of one block per ray), kept as a guard
      const float vl = m.v[cl];
      float xr0 = ob[0] + ((float)li[0] + 0.5f) * vl;
      float xr1 = ob[1] + ((float)li[1] + 0.5f) * vl;
      float xr2 = ob[2] + ((float)li[2] + 0.5f) * vl;
      float d = rho_f - (xr0 * rh[0] + xr1 * rh[1] + xr2 * rh[2]);
      if (d < -m.tau) d = -m.tau;
      if (d > m.tau) d = m.tau;
      rk[run] = ((uint32_t)j << 9) | (uint32_t)(li[0] + nl * (li[1] + nl * li[2]));
      rd[run] = d;
    }
    ++run;
  });
  flush();
  if (!ok) set_status(m.st, kStSegment);
}

__global__ void k_zero_obs_counts(MapDev m) {
  const uint32_t total = min(m.st->touched_count[0], m.max_touched) + min(m.st->touched_count[1], m.max_touched) +
                         min(m.st->touched_count[2], m.max_touched);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    m.blk_count[i] = 0;
    m.blk_fill[i] = 0;
  }
}

// exclusive prefix sum of the per-block observation counts (one CTA, 16 consecutive entries per thread)
__global__ void __launch_bounds__(1024) k_scan_obs(MapDev m) {
  __shared__ uint32_t s_w[32];
  __shared__ uint32_t s_carry;
  const uint32_t total = min(m.st->touched_count[0], m.max_touched) + min(m.st->touched_count[1], m.max_touched) +
                         min(m.st->touched_count[2], m.max_touched);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_carry = 0;
  __syncthreads();
  for (uint32_t base = 0; base < total; base += 1024u * 16u) {
    uint32_t v[16], sum = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      uint32_t i = base + (uint32_t)tid * 16u + k;
      v[k] = i < total ? m.blk_count[i] : 0u;
      sum += v[k];
    }
    uint32_t incl = sum;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(~0u, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      uint32_t w = s_w[lane];
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(~0u, w, o);
        if (lane >= o) w += t;
      }
      s_w[lane] = w;
    }
    __syncthreads();
    uint32_t run = s_carry + (warp > 0 ? s_w[warp - 1] : 0u) + incl - sum;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      uint32_t i = base + (uint32_t)tid * 16u + k;
      if (i < total) m.blk_off[i] = run;
      run += v[k];
    }
    __syncthreads();
    if (tid == 0) s_carry += s_w[31];
    __syncthreads();
  }
  if (tid == 0) m.blk_off[total] = s_carry;
}

}  // namespace

void launch_fuse_depth(const MapDev& m, const CamArgs& c, const float* depth, const uint8_t* rgb, cudaStream_t s,
                       int sms) {
  const int grid = sms * 16;
  if (m.fp16) {
    if (m.color) k_fuse_depth<true, true><<<grid, kThreads, 0, s>>>(m, c, depth, rgb);
    else k_fuse_depth<true, false><<<grid, kThreads, 0, s>>>(m, c, depth, rgb);
  } else {
    if (m.color) k_fuse_depth<false, true><<<grid, kThreads, 0, s>>>(m, c, depth, rgb);
    else k_fuse_depth<false, false><<<grid, kThreads, 0, s>>>(m, c, depth, rgb);
  }
}

void launch_lidar_observations(const MapDev& m, const double* T, const float* xyz, uint64_t n, cudaStream_t s,
                               int sms) {
  PoseD P;
  for (int i = 0; i < 16; ++i) P.T[i] = T[i];
  k_zero_obs_counts<<<sms * 2, 256, 0, s>>>(m);
  if (n == 0) {
    k_scan_obs<<<1, 1024, 0, s>>>(m);
    return;
  }
  const unsigned blocks = (unsigned)((n + 127) / 128);
  k_lidar_walk<false><<<blocks, 128, 0, s>>>(m, P, xyz, n);
  k_scan_obs<<<1, 1024, 0, s>>>(m);
  k_lidar_walk<true><<<blocks, 128, 0, s>>>(m, P, xyz, n);
}

void launch_fuse_points(const MapDev& m, const double*, const float*, uint64_t, cudaStream_t s, int sms) {
  const int grid = sms * 12;
  if (m.fp16) {
    if (m.color) k_fuse_points<true, true><<<grid, kThreads, 0, s>>>(m);
    else k_fuse_points<true, false><<<grid, kThreads, 0, s>>>(m);
  } else {
    if (m.color) k_fuse_points<false, true><<<grid, kThreads, 0, s>>>(m);
    else k_fuse_points<false, false><<<grid, kThreads, 0, s>>>(m);
  }
}

}  // namespace mrh
