// Training and batch inference of the learned level predictor (see mrh_mlp.cuh for the network and its arithmetic).
//
// k_mlp_grad: a CTA takes 32 samples; inputs, pre-activations and BF16 activations of both hidden layers stay in
// shared memory; the forward pass, softmax cross-entropy, and the backward pass through each layer run as small
// matrix products over the CTA's samples; the CTA adds its partial gradient of the mean loss to the FP32 gradient
// with one atomic add per parameter. The network sees BF16 weights; gradients update FP32 master weights.
// k_mlp_adam: Adam on the master weights (beta1 0.9, beta2 0.999, eps 1e-8), then the BF16 copy, then zero gradients.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "mrh_mlp.cuh"

namespace mrh {
namespace {

constexpr int kTile = 32;  // samples per CTA
constexpr int kGradThreads = 256;

__device__ __forceinline__ float wv(const uint16_t* __restrict__ w, int i) { return bf16_to_float(__ldg(w + i)); }

__global__ void __launch_bounds__(kGradThreads) k_mlp_grad(const uint16_t* __restrict__ w, const float* __restrict__ x,
                                                           const int32_t* __restrict__ y, uint32_t n, float inv_n,
                                                           float* __restrict__ grad, float* __restrict__ loss) {
  __shared__ float sX[kTile][kMlpIn];
  __shared__ float sA1[kTile][kMlpH];  // pre-activation, then its gradient
  __shared__ float sH1[kTile][kMlpH];
  __shared__ float sA2[kTile][kMlpH];
  __shared__ float sH2[kTile][kMlpH];
  __shared__ float sD3[kTile][kMlpOut];
  __shared__ float sLoss[kTile];
  const int tid = threadIdx.x;
  const uint32_t base = blockIdx.x * kTile;
  const int rows = (int)min((uint32_t)kTile, n - base);
  for (int e = tid; e < kTile * kMlpIn; e += kGradThreads) {
    const int i = e / kMlpIn, k = e % kMlpIn;
    sX[i][k] = i < rows ? bf16_round(x[(size_t)(base + i) * kMlpIn + k]) : 0.0f;
  }
  __syncthreads();
  // layer 1
  for (int e = tid; e < kTile * kMlpH; e += kGradThreads) {
    const int i = e / kMlpH, j = e % kMlpH;
    float a = wv(w, kOffB1 + j);
    for (int k = 0; k < kMlpIn; ++k) a = a + sX[i][k] * wv(w, kOffW1 + k * kMlpH + j);
    sA1[i][j] = a;
    sH1[i][j] = bf16_round(mlp_gelu(a));
  }
  __syncthreads();
  // layer 2
  for (int e = tid; e < kTile * kMlpH; e += kGradThreads) {
    const int i = e / kMlpH, j = e % kMlpH;
    float a = wv(w, kOffB2 + j);
    for (int k = 0; k < kMlpH; ++k) a = a + sH1[i][k] * wv(w, kOffW2 + k * kMlpH + j);
    sA2[i][j] = a;
    sH2[i][j] = bf16_round(mlp_gelu(a));
  }
  __syncthreads();
  // logits, softmax cross-entropy, d loss / d logits
  if (tid < kTile) {
    const int i = tid;
    float z[kMlpOut];
    for (int c = 0; c < kMlpOut; ++c) {
      float a = wv(w, kOffB3 + c);
      for (int k = 0; k < kMlpH; ++k) a = a + sH2[i][k] * wv(w, kOffW3 + k * kMlpOut + c);
      z[c] = a;
    }
    float zmax = z[0];
    for (int c = 1; c < kMlpOut; ++c) zmax = z[c] > zmax ? z[c] : zmax;
    float se = 0.0f, p[kMlpOut];
    for (int c = 0; c < kMlpOut; ++c) {
      p[c] = expf(z[c] - zmax);
      se = se + p[c];
    }
    float l = 0.0f;
    const int yi = i < rows ? y[base + i] : -1;
    if (yi >= 0 && yi < kMlpOut) {  // a label outside [0, 3) contributes nothing
      l = -(z[yi] - zmax - logf(se));
      for (int c = 0; c < kMlpOut; ++c) sD3[i][c] = (p[c] / se - (c == yi ? 1.0f : 0.0f)) * inv_n;
    } else {
      for (int c = 0; c < kMlpOut; ++c) sD3[i][c] = 0.0f;
    }
    sLoss[i] = l;
  }
  __syncthreads();
  if (tid == 0) {
    float l = 0.0f;
    for (int i = 0; i < kTile; ++i) l = l + sLoss[i];
    atomicAdd(loss, l * inv_n);
  }
  // W3, b3
  for (int e = tid; e < kMlpH * kMlpOut + kMlpOut; e += kGradThreads) {
    float g = 0.0f;
    if (e < kMlpH * kMlpOut) {
      const int k = e / kMlpOut, c = e % kMlpOut;
      for (int i = 0; i < kTile; ++i) g = g + sH2[i][k] * sD3[i][c];
      atomicAdd(&grad[kOffW3 + e], g);
    } else {
      const int c = e - kMlpH * kMlpOut;
      for (int i = 0; i < kTile; ++i) g = g + sD3[i][c];
      atomicAdd(&grad[kOffB3 + c], g);
    }
  }
  // d A2 = (d logits W3^T) * GELU'(A2), in place of A2
  for (int e = tid; e < kTile * kMlpH; e += kGradThreads) {
    const int i = e / kMlpH, k = e % kMlpH;
    float g = 0.0f;
    for (int c = 0; c < kMlpOut; ++c) g = g + sD3[i][c] * wv(w, kOffW3 + k * kMlpOut + c);
    sA2[i][k] = g * mlp_gelu_grad(sA2[i][k]);
  }
  __syncthreads();
  // W2, b2
  for (int e = tid; e < kMlpH * kMlpH + kMlpH; e += kGradThreads) {
    float g = 0.0f;
    if (e < kMlpH * kMlpH) {
      const int k = e / kMlpH, j = e % kMlpH;
      for (int i = 0; i < kTile; ++i) g = g + sH1[i][k] * sA2[i][j];
      atomicAdd(&grad[kOffW2 + e], g);
    } else {
      const int j = e - kMlpH * kMlpH;
      for (int i = 0; i < kTile; ++i) g = g + sA2[i][j];
      atomicAdd(&grad[kOffB2 + j], g);
    }
  }
  // d A1 = (d A2 W2^T) * GELU'(A1), in place of A1
  for (int e = tid; e < kTile * kMlpH; e += kGradThreads) {
    const int i = e / kMlpH, k = e % kMlpH;
    float g = 0.0f;
    for (int j = 0; j < kMlpH; ++j) g = g + sA2[i][j] * wv(w, kOffW2 + k * kMlpH + j);
    sA1[i][k] = g * mlp_gelu_grad(sA1[i][k]);
  }
  __syncthreads();
  // W1, b1
  for (int e = tid; e < kMlpIn * kMlpH + kMlpH; e += kGradThreads) {
    float g = 0.0f;
    if (e < kMlpIn * kMlpH) {
      const int k = e / kMlpH, j = e % kMlpH;
      for (int i = 0; i < kTile; ++i) g = g + sX[i][k] * sA1[i][j];
      atomicAdd(&grad[kOffW1 + e], g);
    } else {
      const int j = e - kMlpIn * kMlpH;
      for (int i = 0; i < kTile; ++i) g = g + sA1[i][j];
      atomicAdd(&grad[kOffB1 + j], g);
    }
  }
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
  k_mlp_grad<<<(n + kTile - 1) / kTile, kGradThreads, 0, s>>>(m->wbf, x, y, n, 1.0f / (float)n, grad, loss);
  MRH_MCUDA(cudaGetLastError());
  return MRH_OK;
}

mrh_status mrh_mlp_train_step(mrh_mlp* m, const float* x, const int32_t* y, uint32_t n, float lr, float* loss,
                              void* stream) {
  if (!m || !x || !y || !loss || n == 0 || !(lr > 0.0f)) return MRH_ERR_INVALID_ARG;
  MlpDevice guard(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  MRH_MCUDA(cudaMemsetAsync(loss, 0, sizeof(float), s));
  k_mlp_grad<<<(n + kTile - 1) / kTile, kGradThreads, 0, s>>>(m->wbf, x, y, n, 1.0f / (float)n, m->grad, loss);
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
