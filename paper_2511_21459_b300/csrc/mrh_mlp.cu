// Training and batch inference of the learned level predictor (see mrh_mlp.cuh for the network and its arithmetic).
//
// k_mlp_grad: the gradient of the mean softmax cross-entropy over a batch, with the products of the forward and
// backward passes on the tensor cores (mma.sync, BF16 operands, FP32 accumulation; see the kernel). The network sees
// BF16 weights; gradients update FP32 master weights.
// k_mlp_adam: Adam on the master weights (beta1 0.9, beta2 0.999, eps 1e-8), then the BF16 copy, then zero gradients.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "mrh_mlp.cuh"

namespace mrh {
namespace {

// -------------------------------------------------------------------------------------------- training on tensor cores
//
// k_mlp_grad: persistent CTAs of 4 warps take tiles of 64 samples. Every product of the forward and backward passes
// is a small matrix product run by mma.sync.m16n8k16 (BF16 operands, FP32 accumulation) on the tensor cores:
//   forward   A1 = X W1 + b1, A2 = H1 W2 + b2, Z = H2 W3 + b3 (X, H1, H2 and the weights are BF16 values, so these
//             products are exact before the FP32 sums); H = BF16(GELU(A)) as in inference;
//   backward  dW3 += H2^T dZ, dW2 += H1^T dA2, dH1 = dA2 W2^T, dW1 += X^T dA1; the FP32 gradient operand is split into
//             a BF16 high part and a BF16 remainder, two products each, which carries 16 of its 24 mantissa bits;
//             dH2 = dZ W3^T (three terms) and the bias sums run on the CUDA cores.
// The weight gradients of a CTA stay in its warps' accumulator registers over all its tiles and reach the global
// gradient with one atomic add per parameter per CTA.

constexpr int kTcTile = 64;    // samples per tile
constexpr int kTcThreads = 128;

struct TcSmem {
  uint16_t w[kMlpParams + 5];           // BF16 weights (bit patterns)
  uint16_t x[kTcTile][kMlpIn];          // BF16 inputs
  float a1[kTcTile][kMlpH];             // pre-activations, then their gradients
  float a2[kTcTile][kMlpH];
  uint16_t h1[kTcTile][kMlpH];          // BF16 activations
  uint16_t h2[kTcTile][kMlpH];
  float dz[kTcTile][4];                 // d loss / d logits (column 3 zero)
  float loss[kTcTile];
};

__device__ __forceinline__ uint32_t pack_bf16(uint16_t lo, uint16_t hi) { return (uint32_t)lo | ((uint32_t)hi << 16); }

// the BF16 high part of x and the BF16 rounding of the remainder x - high
__device__ __forceinline__ void split_bf16(float x, uint16_t& hi, uint16_t& lo) {
  hi = float_to_bf16(x);
  lo = float_to_bf16(x - bf16_to_float(hi));
}

// D += A B for one m16n8k16 tile: a[4], b[2] hold BF16 pairs in the standard fragment layout
// (lane = 4 g + t: a0 = A[g][2t, 2t+1], a1 = A[g+8][2t, 2t+1], a2 = A[g][2t+8, 2t+9], a3 = A[g+8][2t+8, 2t+9];
//  b0 = B[2t, 2t+1][g], b1 = B[2t+8, 2t+9][g]; c0, c1 = C[g][2t, 2t+1], c2, c3 = C[g+8][2t, 2t+1])
__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(kTcThreads) k_mlp_grad(const uint16_t* __restrict__ w, const float* __restrict__ x,
                                                       const int32_t* __restrict__ y, uint32_t n, float inv_n,
                                                       float* __restrict__ grad, float* __restrict__ loss) {
  extern __shared__ __align__(16) unsigned char s_raw[];
  TcSmem& sm = *reinterpret_cast<TcSmem*>(s_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  for (int p = tid; p < kMlpParams; p += kTcThreads) sm.w[p] = w[p];
  const uint16_t* W1 = sm.w + kOffW1;  // [in][h]
  const uint16_t* W2 = sm.w + kOffW2;  // [h][h]
  const uint16_t* W3 = sm.w + kOffW3;  // [h][out]
  // weight-gradient accumulators, kept over all tiles of this CTA:
  //   dW1 (16 x 64): m-tile 0, n-tiles 2 warp, 2 warp + 1;  dW2 (64 x 64): m-tile warp, n-tiles 0..7;
  //   dW3 (64 x 8, columns 3..7 padding): m-tile warp
  float g1[2][4], g2[8][4], g3[4];
  #pragma unroll
  for (int i = 0; i < 4; ++i) {
    g1[0][i] = g1[1][i] = g3[i] = 0.0f;
    for (int j = 0; j < 8; ++j) g2[j][i] = 0.0f;
  }
  float gb = 0.0f, gb3 = 0.0f;  // bias sums: thread j < 64 column j of dA1, 64 <= j < 128 column j - 64 of dA2
  float my_loss = 0.0f;
  const uint32_t tiles = (n + kTcTile - 1) / kTcTile;
  __syncthreads();
  for (uint32_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const uint32_t base = tile * kTcTile;
    for (int e = tid; e < kTcTile * kMlpIn; e += kTcThreads) {
      const int i = e / kMlpIn, k = e % kMlpIn;
      sm.x[i][k] = base + i < n ? float_to_bf16(x[(size_t)(base + i) * kMlpIn + k]) : (uint16_t)0;
    }
    __syncthreads();
    const int r0 = 16 * warp;  // this warp's 16 samples of the tile in the forward pass
    // ---- layer 1: A1 = X W1 + b1 (K = 16)
    {
      uint32_t a[4];
      a[0] = pack_bf16(sm.x[r0 + g][2 * t], sm.x[r0 + g][2 * t + 1]);
      a[1] = pack_bf16(sm.x[r0 + g + 8][2 * t], sm.x[r0 + g + 8][2 * t + 1]);
      a[2] = pack_bf16(sm.x[r0 + g][2 * t + 8], sm.x[r0 + g][2 * t + 9]);
      a[3] = pack_bf16(sm.x[r0 + g + 8][2 * t + 8], sm.x[r0 + g + 8][2 * t + 9]);
      #pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const int col = 8 * nt + g;
        uint32_t b[2];
        b[0] = pack_bf16(W1[(2 * t) * kMlpH + col], W1[(2 * t + 1) * kMlpH + col]);
        b[1] = pack_bf16(W1[(2 * t + 8) * kMlpH + col], W1[(2 * t + 9) * kMlpH + col]);
        float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        mma16816(c, a, b);
        #pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int row = r0 + g + (q >> 1) * 8, cc = 8 * nt + 2 * t + (q & 1);
          const float v = c[q] + bf16_to_float(sm.w[kOffB1 + cc]);
          sm.a1[row][cc] = v;
          sm.h1[row][cc] = float_to_bf16(mlp_gelu(v));
        }
      }
    }
    __syncwarp();
    // ---- layer 2: A2 = H1 W2 + b2 (K = 64), this warp's rows only
    {
      float c[8][4];
      #pragma unroll
      for (int nt = 0; nt < 8; ++nt)
        #pragma unroll
        for (int q = 0; q < 4; ++q) c[nt][q] = 0.0f;
      #pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        const int k0 = 16 * ks;
        uint32_t a[4];
        a[0] = pack_bf16(sm.h1[r0 + g][k0 + 2 * t], sm.h1[r0 + g][k0 + 2 * t + 1]);
        a[1] = pack_bf16(sm.h1[r0 + g + 8][k0 + 2 * t], sm.h1[r0 + g + 8][k0 + 2 * t + 1]);
        a[2] = pack_bf16(sm.h1[r0 + g][k0 + 2 * t + 8], sm.h1[r0 + g][k0 + 2 * t + 9]);
        a[3] = pack_bf16(sm.h1[r0 + g + 8][k0 + 2 * t + 8], sm.h1[r0 + g + 8][k0 + 2 * t + 9]);
        #pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
          const int col = 8 * nt + g;
          uint32_t b[2];
          b[0] = pack_bf16(W2[(k0 + 2 * t) * kMlpH + col], W2[(k0 + 2 * t + 1) * kMlpH + col]);
          b[1] = pack_bf16(W2[(k0 + 2 * t + 8) * kMlpH + col], W2[(k0 + 2 * t + 9) * kMlpH + col]);
          mma16816(c[nt], a, b);
        }
      }
      #pragma unroll
      for (int nt = 0; nt < 8; ++nt)
        #pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int row = r0 + g + (q >> 1) * 8, cc = 8 * nt + 2 * t + (q & 1);
          const float v = c[nt][q] + bf16_to_float(sm.w[kOffB2 + cc]);
          sm.a2[row][cc] = v;
          sm.h2[row][cc] = float_to_bf16(mlp_gelu(v));
        }
    }
    __syncwarp();
    // ---- logits Z = H2 W3 + b3 (N = 3, padded to 8), into dz[][] of this warp's rows
    {
      float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      #pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        const int k0 = 16 * ks;
        uint32_t a[4], b[2];
        a[0] = pack_bf16(sm.h2[r0 + g][k0 + 2 * t], sm.h2[r0 + g][k0 + 2 * t + 1]);
        a[1] = pack_bf16(sm.h2[r0 + g + 8][k0 + 2 * t], sm.h2[r0 + g + 8][k0 + 2 * t + 1]);
        a[2] = pack_bf16(sm.h2[r0 + g][k0 + 2 * t + 8], sm.h2[r0 + g][k0 + 2 * t + 9]);
        a[3] = pack_bf16(sm.h2[r0 + g + 8][k0 + 2 * t + 8], sm.h2[r0 + g + 8][k0 + 2 * t + 9]);
        const bool col = g < kMlpOut;
        b[0] = col ? pack_bf16(W3[(k0 + 2 * t) * kMlpOut + g], W3[(k0 + 2 * t + 1) * kMlpOut + g]) : 0u;
        b[1] = col ? pack_bf16(W3[(k0 + 2 * t + 8) * kMlpOut + g], W3[(k0 + 2 * t + 9) * kMlpOut + g]) : 0u;
        mma16816(c, a, b);
      }
      if (t < 2)
        #pragma unroll
        for (int q = 0; q < 4; ++q) sm.dz[r0 + g + (q >> 1) * 8][2 * t + (q & 1)] = c[q];
    }
    __syncwarp();
    // ---- softmax cross-entropy and d loss / d logits, one lane per sample of this warp
    if (lane < 16) {
      const int row = r0 + lane;
      float z[kMlpOut];
      #pragma unroll
      for (int cc = 0; cc < kMlpOut; ++cc) z[cc] = sm.dz[row][cc] + bf16_to_float(sm.w[kOffB3 + cc]);
      float zmax = z[0];
      for (int cc = 1; cc < kMlpOut; ++cc) zmax = z[cc] > zmax ? z[cc] : zmax;
      float se = 0.0f, p[kMlpOut];
      #pragma unroll
      for (int cc = 0; cc < kMlpOut; ++cc) {
        p[cc] = expf(z[cc] - zmax);
        se = se + p[cc];
      }
      const int yi = base + row < n ? y[base + row] : -1;
      if (yi >= 0 && yi < kMlpOut) {  // a label outside [0, 3) contributes nothing
        my_loss += -(z[yi] - zmax - logf(se));
        #pragma unroll
        for (int cc = 0; cc < kMlpOut; ++cc) sm.dz[row][cc] = (p[cc] / se - (cc == yi ? 1.0f : 0.0f)) * inv_n;
      } else {
        #pragma unroll
        for (int cc = 0; cc < kMlpOut; ++cc) sm.dz[row][cc] = 0.0f;
      }
      sm.dz[row][3] = 0.0f;
    }
    __syncthreads();
    // ---- dW3 += H2^T dZ (M = 64 hidden: m-tile warp; K = the tile's samples)
    #pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
      const int s0 = 16 * ks, m0 = 16 * warp;
      uint32_t a[4];
      a[0] = pack_bf16(sm.h2[s0 + 2 * t][m0 + g], sm.h2[s0 + 2 * t + 1][m0 + g]);
      a[1] = pack_bf16(sm.h2[s0 + 2 * t][m0 + g + 8], sm.h2[s0 + 2 * t + 1][m0 + g + 8]);
      a[2] = pack_bf16(sm.h2[s0 + 2 * t + 8][m0 + g], sm.h2[s0 + 2 * t + 9][m0 + g]);
      a[3] = pack_bf16(sm.h2[s0 + 2 * t + 8][m0 + g + 8], sm.h2[s0 + 2 * t + 9][m0 + g + 8]);
      uint16_t h[4], l[4];
      const bool col = g < 4;
      split_bf16(col ? sm.dz[s0 + 2 * t][g] : 0.0f, h[0], l[0]);
      split_bf16(col ? sm.dz[s0 + 2 * t + 1][g] : 0.0f, h[1], l[1]);
      split_bf16(col ? sm.dz[s0 + 2 * t + 8][g] : 0.0f, h[2], l[2]);
      split_bf16(col ? sm.dz[s0 + 2 * t + 9][g] : 0.0f, h[3], l[3]);
      const uint32_t bh[2] = {pack_bf16(h[0], h[1]), pack_bf16(h[2], h[3])};
      const uint32_t bl[2] = {pack_bf16(l[0], l[1]), pack_bf16(l[2], l[3])};
      mma16816(g3, a, bh);
      mma16816(g3, a, bl);
    }
    if (tid < kMlpOut)
      for (int s = 0; s < kTcTile; ++s) gb3 += sm.dz[s][tid];
    // ---- dA2 = (dZ W3^T) * GELU'(A2), in place of A2 (three terms per element, CUDA cores)
    for (int e = tid; e < kTcTile * kMlpH; e += kTcThreads) {
      const int s = e / kMlpH, k = e % kMlpH;
      float d = 0.0f;
      #pragma unroll
      for (int cc = 0; cc < kMlpOut; ++cc) d = d + sm.dz[s][cc] * bf16_to_float(W3[k * kMlpOut + cc]);
      sm.a2[s][k] = d * mlp_gelu_grad(sm.a2[s][k]);
    }
    __syncthreads();
    // ---- dW2 += H1^T dA2 (m-tile warp, n-tiles 0..7; K = the tile's samples)
    #pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
      const int s0 = 16 * ks, m0 = 16 * warp;
      uint32_t a[4];
      a[0] = pack_bf16(sm.h1[s0 + 2 * t][m0 + g], sm.h1[s0 + 2 * t + 1][m0 + g]);
      a[1] = pack_bf16(sm.h1[s0 + 2 * t][m0 + g + 8], sm.h1[s0 + 2 * t + 1][m0 + g + 8]);
      a[2] = pack_bf16(sm.h1[s0 + 2 * t + 8][m0 + g], sm.h1[s0 + 2 * t + 9][m0 + g]);
      a[3] = pack_bf16(sm.h1[s0 + 2 * t + 8][m0 + g + 8], sm.h1[s0 + 2 * t + 9][m0 + g + 8]);
      #pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const int col = 8 * nt + g;
        uint16_t h[4], l[4];
        split_bf16(sm.a2[s0 + 2 * t][col], h[0], l[0]);
        split_bf16(sm.a2[s0 + 2 * t + 1][col], h[1], l[1]);
        split_bf16(sm.a2[s0 + 2 * t + 8][col], h[2], l[2]);
        split_bf16(sm.a2[s0 + 2 * t + 9][col], h[3], l[3]);
        const uint32_t bh[2] = {pack_bf16(h[0], h[1]), pack_bf16(h[2], h[3])};
        const uint32_t bl[2] = {pack_bf16(l[0], l[1]), pack_bf16(l[2], l[3])};
        mma16816(g2[nt], a, bh);
        mma16816(g2[nt], a, bl);
      }
    }
    if (tid >= kMlpH)
      for (int s = 0; s < kTcTile; ++s) gb += sm.a2[s][tid - kMlpH];
    // ---- dA1 = (dA2 W2^T) * GELU'(A1), this warp's rows, in place of A1
    {
      float c[8][4];
      #pragma unroll
      for (int nt = 0; nt < 8; ++nt)
        #pragma unroll
        for (int q = 0; q < 4; ++q) c[nt][q] = 0.0f;
      #pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        const int k0 = 16 * ks;
        uint16_t h[8], l[8];
        split_bf16(sm.a2[r0 + g][k0 + 2 * t], h[0], l[0]);
        split_bf16(sm.a2[r0 + g][k0 + 2 * t + 1], h[1], l[1]);
        split_bf16(sm.a2[r0 + g + 8][k0 + 2 * t], h[2], l[2]);
        split_bf16(sm.a2[r0 + g + 8][k0 + 2 * t + 1], h[3], l[3]);
        split_bf16(sm.a2[r0 + g][k0 + 2 * t + 8], h[4], l[4]);
        split_bf16(sm.a2[r0 + g][k0 + 2 * t + 9], h[5], l[5]);
        split_bf16(sm.a2[r0 + g + 8][k0 + 2 * t + 8], h[6], l[6]);
        split_bf16(sm.a2[r0 + g + 8][k0 + 2 * t + 9], h[7], l[7]);
        const uint32_t ah[4] = {pack_bf16(h[0], h[1]), pack_bf16(h[2], h[3]), pack_bf16(h[4], h[5]),
                                pack_bf16(h[6], h[7])};
        const uint32_t al[4] = {pack_bf16(l[0], l[1]), pack_bf16(l[2], l[3]), pack_bf16(l[4], l[5]),
                                pack_bf16(l[6], l[7])};
        #pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
          const int row = 8 * nt + g;  // W2 row: the H1 index this column of dH1 belongs to
          uint32_t b[2];
          b[0] = pack_bf16(W2[row * kMlpH + k0 + 2 * t], W2[row * kMlpH + k0 + 2 * t + 1]);
          b[1] = pack_bf16(W2[row * kMlpH + k0 + 2 * t + 8], W2[row * kMlpH + k0 + 2 * t + 9]);
          mma16816(c[nt], ah, b);
          mma16816(c[nt], al, b);
        }
      }
      #pragma unroll
      for (int nt = 0; nt < 8; ++nt)
        #pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int row = r0 + g + (q >> 1) * 8, cc = 8 * nt + 2 * t + (q & 1);
          sm.a1[row][cc] = c[nt][q] * mlp_gelu_grad(sm.a1[row][cc]);
        }
    }
    __syncthreads();
    // ---- dW1 += X^T dA1 (M = 16 inputs; n-tiles 2 warp, 2 warp + 1; K = the tile's samples)
    #pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
      const int s0 = 16 * ks;
      uint32_t a[4];
      a[0] = pack_bf16(sm.x[s0 + 2 * t][g], sm.x[s0 + 2 * t + 1][g]);
      a[1] = pack_bf16(sm.x[s0 + 2 * t][g + 8], sm.x[s0 + 2 * t + 1][g + 8]);
      a[2] = pack_bf16(sm.x[s0 + 2 * t + 8][g], sm.x[s0 + 2 * t + 9][g]);
      a[3] = pack_bf16(sm.x[s0 + 2 * t + 8][g + 8], sm.x[s0 + 2 * t + 9][g + 8]);
      #pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int col = 8 * (2 * warp + i) + g;
        uint16_t h[4], l[4];
        split_bf16(sm.a1[s0 + 2 * t][col], h[0], l[0]);
        split_bf16(sm.a1[s0 + 2 * t + 1][col], h[1], l[1]);
        split_bf16(sm.a1[s0 + 2 * t + 8][col], h[2], l[2]);
        split_bf16(sm.a1[s0 + 2 * t + 9][col], h[3], l[3]);
        const uint32_t bh[2] = {pack_bf16(h[0], h[1]), pack_bf16(h[2], h[3])};
        const uint32_t bl[2] = {pack_bf16(l[0], l[1]), pack_bf16(l[2], l[3])};
        mma16816(g1[i], a, bh);
        mma16816(g1[i], a, bl);
      }
    }
    if (tid < kMlpH)
      for (int s = 0; s < kTcTile; ++s) gb += sm.a1[s][tid];
    __syncthreads();  // the next tile overwrites the shared arrays
  }
  // ---- one atomic add per parameter per CTA
  #pragma unroll
  for (int i = 0; i < 2; ++i)
    #pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int m = g + (q >> 1) * 8, j = 8 * (2 * warp + i) + 2 * t + (q & 1);
      atomicAdd(&grad[kOffW1 + m * kMlpH + j], g1[i][q]);
    }
  #pragma unroll
  for (int nt = 0; nt < 8; ++nt)
    #pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int m = 16 * warp + g + (q >> 1) * 8, j = 8 * nt + 2 * t + (q & 1);
      atomicAdd(&grad[kOffW2 + m * kMlpH + j], g2[nt][q]);
    }
  #pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int m = 16 * warp + g + (q >> 1) * 8, cc = 2 * t + (q & 1);
    if (cc < kMlpOut) atomicAdd(&grad[kOffW3 + m * kMlpOut + cc], g3[q]);
  }
  if (tid < kMlpH) atomicAdd(&grad[kOffB1 + tid], gb);
  else atomicAdd(&grad[kOffB2 + tid - kMlpH], gb);
  if (tid < kMlpOut) atomicAdd(&grad[kOffB3 + tid], gb3);
  for (int o = 16; o > 0; o >>= 1) my_loss += __shfl_xor_sync(~0u, my_loss, o);
  if (lane == 0 && my_loss != 0.0f) atomicAdd(loss, my_loss * inv_n);
}

__global__ void k_mlp_adam(float* __restrict__ master, uint16_t* __restrict__ wbf, float* __restrict__ m1,
                           float* __restrict__ m2, float* __restrict__ grad, float lr, float bc1, float bc2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kMlpParams) return;
  const float g = grad[p];
  const float a = 0.9f * m1[p] + 0.1f * g;
  const float b = 0.999f * m2[p] + 0.001f * g * g;
  m1[p] = a;
  m2[p] = b;
  const float mh = a / bc1, vh = b / bc2;
  const float wn = master[p] - lr * mh / (sqrtf(vh) + 1e-8f);
  master[p] = wn;
  wbf[p] = float_to_bf16(wn);
  grad[p] = 0.0f;
}

__global__ void k_mlp_predict(const uint16_t* __restrict__ w, const float* __restrict__ x, uint32_t n,
                              float* __restrict__ logits) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float xi[kMlpIn];
  for (int k = 0; k < kMlpIn; ++k) xi[k] = bf16_round(x[(size_t)i * kMlpIn + k]);
  float z[kMlpOut];
  mlp_infer(w, xi, z);
  for (int c = 0; c < kMlpOut; ++c) logits[(size_t)i * kMlpOut + c] = z[c];
}

__global__ void k_round_bf16(const float* __restrict__ src, uint16_t* __restrict__ dst) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kMlpParams) dst[p] = float_to_bf16(src[p]);
}

}  // namespace
}  // namespace mrh

using namespace mrh;

struct mrh_mlp {
  int device = 0;
  float* master = nullptr;  // FP32 master weights
  uint16_t* wbf = nullptr;  // BF16 copy used by forward / backward / inference
  float* m1 = nullptr;
  float* m2 = nullptr;
  float* grad = nullptr;
  long long step = 0;
};

namespace {

#define MRH_MCUDA(call)                                  \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
  } while (0)

struct MlpDevice {
  int prev = -1;
  explicit MlpDevice(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess) cudaSetDevice(dev);
  }
  ~MlpDevice() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// persistent grid: up to three CTAs per SM (shared memory), never more CTAs than tiles
cudaError_t launch_mlp_grad(const mrh_mlp* m, const float* x, const int32_t* y, uint32_t n, float* grad, float* loss,
                            cudaStream_t s) {
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device);
  const int smem = (int)sizeof(TcSmem);
  cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const uint32_t tiles = (n + kTcTile - 1) / kTcTile;
  const uint32_t grid = std::min<uint32_t>(tiles, (uint32_t)sms * 3u);
  k_mlp_grad<<<grid, kTcThreads, smem, s>>>(m->wbf, x, y, n, 1.0f / (float)n, grad, loss);
  return cudaGetLastError();
}

void mlp_free(mrh_mlp* m) {
  for (float* p : {m->master, m->m1, m->m2, m->grad})
    if (p) cudaFree(p);
  if (m->wbf) cudaFree(m->wbf);
}

}  // namespace

extern "C" {

mrh_status mrh_mlp_create(const float* init_host, int device, mrh_mlp** out) {
  if (!out || !init_host) return MRH_ERR_INVALID_ARG;
  *out = nullptr;
  for (int p = 0; p < kMlpParams; ++p)
    if (!std::isfinite(init_host[p])) return MRH_ERR_INVALID_ARG;
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return MRH_ERR_INVALID_ARG;
  mrh_mlp* m = new (std::nothrow) mrh_mlp();
  if (!m) return MRH_ERR_OUT_OF_MEMORY;
  m->device = device;
  const size_t bytes = sizeof(float) * kMlpParams;
  cudaError_t e = cudaSuccess;
  for (float** p : {&m->master, &m->m1, &m->m2, &m->grad})
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&m->wbf, sizeof(uint16_t) * kMlpParams);
  if (e == cudaSuccess) e = cudaMemcpy(m->master, init_host, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m->m1, 0, bytes);
  if (e == cudaSuccess) e = cudaMemset(m->m2, 0, bytes);
  if (e == cudaSuccess) e = cudaMemset(m->grad, 0, bytes);
  if (e == cudaSuccess) {
    k_round_bf16<<<(kMlpParams + 255) / 256, 256>>>(m->master, m->wbf);
    e = cudaDeviceSynchronize();
  }
  if (prev >= 0) cudaSetDevice(prev);
  if (e != cudaSuccess) {
    mlp_free(m);
    delete m;
    return e == cudaErrorMemoryAllocation ? MRH_ERR_OUT_OF_MEMORY : cuda_fail(e, "mrh_mlp_create");
  }
  *out = m;
  return MRH_OK;
}

mrh_status mrh_mlp_destroy(mrh_mlp* m) {
  if (!m) return MRH_OK;
  MlpDevice guard(m->device);
  cudaDeviceSynchronize();
  mlp_free(m);
  delete m;
  return MRH_OK;
}

mrh_status mrh_mlp_get_weights(const mrh_mlp* m, float* master_host, uint16_t* bf16_host, void* stream) {
  if (!m || (!master_host && !bf16_host)) return MRH_ERR_INVALID_ARG;
  MlpDevice guard(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (master_host)
    MRH_MCUDA(cudaMemcpyAsync(master_host, m->master, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, s));
  if (bf16_host)
    MRH_MCUDA(cudaMemcpyAsync(bf16_host, m->wbf, sizeof(uint16_t) * kMlpParams, cudaMemcpyDeviceToHost, s));
  MRH_MCUDA(cudaStreamSynchronize(s));
  return MRH_OK;
}

mrh_status mrh_mlp_loss_grad(const mrh_mlp* m, const float* x, const int32_t* y, uint32_t n, float* loss,
                             float* grad, void* stream) {
  if (!m || !x || !y || !loss || !grad || n == 0) return MRH_ERR_INVALID_ARG;
  MlpDevice guard(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  MRH_MCUDA(cudaMemsetAsync(loss, 0, sizeof(float), s));
  MRH_MCUDA(cudaMemsetAsync(grad, 0, sizeof(float) * kMlpParams, s));
  MRH_MCUDA(launch_mlp_grad(m, x, y, n, grad, loss, s));
  return MRH_OK;
}

mrh_status mrh_mlp_train_step(mrh_mlp* m, const float* x, const int32_t* y, uint32_t n, float lr, float* loss,
                              void* stream) {
  if (!m || !x || !y || !loss || n == 0 || !(lr > 0.0f)) return MRH_ERR_INVALID_ARG;
  MlpDevice guard(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  MRH_MCUDA(cudaMemsetAsync(loss, 0, sizeof(float), s));
  MRH_MCUDA(launch_mlp_grad(m, x, y, n, m->grad, loss, s));
  m->step += 1;
  const float bc1 = (float)(1.0 - std::pow(0.9, (double)m->step));
  const float bc2 = (float)(1.0 - std::pow(0.999, (double)m->step));
  k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, s>>>(m->master, m->wbf, m->m1, m->m2, m->grad, lr, bc1, bc2);
  MRH_MCUDA(cudaGetLastError());
  return MRH_OK;
}

mrh_status mrh_mlp_predict(const mrh_mlp* m, const float* x, uint32_t n, float* logits, void* stream) {
  if (!m || !x || !logits) return MRH_ERR_INVALID_ARG;
  MlpDevice guard(m->device);
  if (n == 0) return MRH_OK;
  k_mlp_predict<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(m->wbf, x, n, logits);
  MRH_MCUDA(cudaGetLastError());
  return MRH_OK;
}

}  // extern "C"
