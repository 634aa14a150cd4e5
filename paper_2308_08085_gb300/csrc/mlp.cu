// Learned refinement proposal: a per-block MLP 27 -> 64 -> 64 -> 1 (ReLU,
// sigmoid) with hand-written training and inference kernels.  FP32 master
// weights are trained with Adam on a class-weighted binary cross-entropy; an
// FP16 copy of the weights is what inference reads.  The MLP is small enough
// that every layer runs on CUDA cores (one sample per thread for inference,
// one hidden unit per thread for the gradient).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <string>

#include "../../include/amr.h"

namespace amr {
void set_error(const std::string& msg);

namespace mlp {

constexpr int IN = AMR_MLP_INPUTS;   // 27
constexpr int H = AMR_MLP_HIDDEN;    // 64
// parameter layout: W1[H][IN], b1[H], W2[H][H], b2[H], w3[H], b3
constexpr int OW1 = 0, OB1 = OW1 + H * IN, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H,
              OB3 = OW3 + H, NP = OB3 + 1;

// SplitMix64 (Steele, Lea, Flood 2014) as a counter-based generator
__host__ __device__ inline uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ inline float uniform_pm1(uint64_t seed, uint64_t i) {
  return (float)((splitmix64(seed ^ splitmix64(i)) >> 40) * (1.0 / 16777216.0)) * 2.f - 1.f;
}

// Glorot-uniform weights, zero biases
__global__ void k_init(float* __restrict__ P, uint64_t seed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NP) return;
  float v = 0.f;
  if (i < OB1) v = uniform_pm1(seed, i) * sqrtf(6.f / (IN + H));
  else if (i >= OW2 && i < OB2) v = uniform_pm1(seed, i) * sqrtf(6.f / (H + H));
  else if (i >= OW3 && i < OB3) v = uniform_pm1(seed, i) * sqrtf(6.f / (H + 1));
  P[i] = v;
}

__device__ inline float softplus(float t) { return t > 0.f ? t + log1pf(expf(-t)) : log1pf(expf(t)); }

// Summed gradient and loss over the samples of one minibatch.  One CTA of H
// threads walks `per_cta` samples; thread k owns hidden unit k of both layers
// and accumulates its gradient rows in registers.  Sample position pos maps to
// index (pos * mul + off) mod n, a bijection when gcd(mul, n) = 1.
__global__ void __launch_bounds__(H)
    k_grad(const float* __restrict__ P, const float* __restrict__ x, const float* __restrict__ y,
           int64_t n, int64_t b0, int64_t bn, int64_t mul, int64_t off, int per_cta,
           float pos_weight, float* __restrict__ grad, float* __restrict__ loss) {
  __shared__ float sW1[H][IN + 1];
  __shared__ float sW2[H][H + 1];
  __shared__ float sb1[H], sb2[H], sw3[H];
  __shared__ float sx[IN], sh1[H], sdh2[H], sred[2];
  const int k = threadIdx.x;
  for (int t = k; t < H * IN; t += H) sW1[t / IN][t % IN] = P[OW1 + t];
  for (int t = k; t < H * H; t += H) sW2[t / H][t % H] = P[OW2 + t];
  sb1[k] = P[OB1 + k];
  sb2[k] = P[OB2 + k];
  sw3[k] = P[OW3 + k];
  const float b3 = P[OB3];
  float gW1[IN], gW2[H];
#pragma unroll
  for (int i = 0; i < IN; ++i) gW1[i] = 0.f;
#pragma unroll
  for (int j = 0; j < H; ++j) gW2[j] = 0.f;
  float gb1 = 0.f, gb2 = 0.f, gw3 = 0.f, gb3 = 0.f, lsum = 0.f;
  __syncthreads();
  const int64_t first = (int64_t)blockIdx.x * per_cta;
  for (int s = 0; s < per_cta; ++s) {
    const int64_t pos = first + s;
    if (pos >= bn) break;
    const int64_t idx = ((b0 + pos) * mul + off) % n;
    if (k < IN) sx[k] = x[idx * IN + k];
    __syncthreads();
    float a1 = sb1[k];
#pragma unroll
    for (int i = 0; i < IN; ++i) a1 += sW1[k][i] * sx[i];
    const float h1 = fmaxf(a1, 0.f);
    sh1[k] = h1;
    __syncthreads();
    float a2 = sb2[k];
#pragma unroll 16
    for (int j = 0; j < H; ++j) a2 += sW2[k][j] * sh1[j];
    const float h2 = fmaxf(a2, 0.f);
    float zp = sw3[k] * h2;
    for (int o = 16; o > 0; o >>= 1) zp += __shfl_xor_sync(0xffffffffu, zp, o);
    if ((k & 31) == 0) sred[k >> 5] = zp;
    __syncthreads();
    const float z = b3 + sred[0] + sred[1];
    const float p = 1.f / (1.f + expf(-z));
    const float yy = y[idx];
    const float dz = pos_weight * yy * (p - 1.f) + (1.f - yy) * p;
    if (k == 0) {
      lsum += pos_weight * yy * softplus(-z) + (1.f - yy) * softplus(z);
      gb3 += dz;
    }
    gw3 += dz * h2;
    const float dh2 = h2 > 0.f ? dz * sw3[k] : 0.f;
    sdh2[k] = dh2;
    __syncthreads();
    gb2 += dh2;
#pragma unroll 16
    for (int j = 0; j < H; ++j) gW2[j] += dh2 * sh1[j];
    float back = 0.f;
#pragma unroll 16
    for (int m = 0; m < H; ++m) back += sW2[m][k] * sdh2[m];
    const float dh1 = h1 > 0.f ? back : 0.f;
    gb1 += dh1;
#pragma unroll
    for (int i = 0; i < IN; ++i) gW1[i] += dh1 * sx[i];
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < IN; ++i) atomicAdd(grad + OW1 + k * IN + i, gW1[i]);
#pragma unroll
  for (int j = 0; j < H; ++j) atomicAdd(grad + OW2 + k * H + j, gW2[j]);
  atomicAdd(grad + OB1 + k, gb1);
  atomicAdd(grad + OB2 + k, gb2);
  atomicAdd(grad + OW3 + k, gw3);
  if (k == 0) {
    atomicAdd(grad + OB3, gb3);
    atomicAdd(loss, lsum);
  }
}

__global__ void k_adam(float* __restrict__ P, float* __restrict__ m, float* __restrict__ v,
                       __half* __restrict__ Ph, const float* __restrict__ grad, float inv_batch,
                       float lr, float b1, float b2, float eps, float bc1, float bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NP) return;
  const float g = grad[i] * inv_batch;
  const float mi = b1 * m[i] + (1.f - b1) * g;
  const float vi = b2 * v[i] + (1.f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  const float w = P[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  P[i] = w;
  Ph[i] = __float2half_rn(w);
}

__global__ void k_to_half(const float* __restrict__ P, __half* __restrict__ Ph) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < NP) Ph[i] = __float2half_rn(P[i]);
}

// One sample per thread; FP16 weights staged as FP32 in shared memory.
// `list` (optional) maps thread i to sample list[i]; output prob[sample].
__global__ void __launch_bounds__(256)
    k_infer(const __half* __restrict__ Ph, const float* __restrict__ x,
            const int32_t* __restrict__ list, int64_t n, float* __restrict__ prob) {
  __shared__ float sP[NP];
  for (int t = threadIdx.x; t < NP; t += blockDim.x) sP[t] = __half2float(Ph[t]);
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t idx = list ? list[i] : i;
  float xi[IN];
#pragma unroll
  for (int q = 0; q < IN; ++q) xi[q] = x[idx * IN + q];
  float h1[H];
#pragma unroll
  for (int j = 0; j < H; ++j) {
    float a = sP[OB1 + j];
#pragma unroll
    for (int q = 0; q < IN; ++q) a += sP[OW1 + j * IN + q] * xi[q];
    h1[j] = fmaxf(a, 0.f);
  }
  float z = sP[OB3];
  for (int kk = 0; kk < H; ++kk) {
    float a = sP[OB2 + kk];
#pragma unroll
    for (int j = 0; j < H; ++j) a += sP[OW2 + kk * H + j] * h1[j];
    z += sP[OW3 + kk] * fmaxf(a, 0.f);
  }
  prob[idx] = 1.f / (1.f + expf(-z));
}

}  // namespace mlp

// used by api.cu (propose marks)
void mlp_infer_list(cudaStream_t s, const void* params_half, const float* x, const int32_t* list,
                    int64_t n, float* prob) {
  if (n <= 0) return;
  mlp::k_infer<<<(int)((n + 255) / 256), 256, 0, s>>>((const __half*)params_half, x, list, n, prob);
}

}  // namespace amr

using namespace amr;

extern "C" {

int amr_mlp_param_count(void) { return mlp::NP; }

int amr_mlp_init(float* params, void* params_half, uint64_t seed, void* stream) {
  if (!params) return AMR_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  mlp::k_init<<<(mlp::NP + 255) / 256, 256, 0, s>>>(params, seed);
  if (params_half) mlp::k_to_half<<<(mlp::NP + 255) / 256, 256, 0, s>>>(params, (__half*)params_half);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("amr_mlp_init: ") + cudaGetErrorString(e));
    return AMR_E_CUDA;
  }
  return AMR_OK;
}

static int launch_grad(const float* params, const float* x, const float* y, int64_t n, int64_t b0,
                       int64_t bn, int64_t mul, int64_t off, float pos_weight, float* grad,
                       float* loss, cudaStream_t s) {
  const int per_cta = 32;
  const int grid = (int)((bn + per_cta - 1) / per_cta);
  if (grid > 0)
    mlp::k_grad<<<grid, mlp::H, 0, s>>>(params, x, y, n, b0, bn, mul, off, per_cta, pos_weight,
                                        grad, loss);
  return cudaGetLastError() == cudaSuccess ? AMR_OK : AMR_E_CUDA;
}

int amr_mlp_grad(const float* params, const float* x, const float* y, int64_t n, float pos_weight,
                 float* grad, float* loss, void* stream) {
  if (!params || !x || !y || !grad || !loss || n <= 0) return AMR_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(grad, 0, sizeof(float) * mlp::NP, s) != cudaSuccess ||
      cudaMemsetAsync(loss, 0, sizeof(float), s) != cudaSuccess)
    return AMR_E_CUDA;
  return launch_grad(params, x, y, n, 0, n, 1, 0, pos_weight, grad, loss, s);
}

static int64_t gcd64(int64_t a, int64_t b) {
  while (b) {
    const int64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

int amr_mlp_train_epoch(const amr_mlp_state* st, const float* x, const float* y, int64_t n,
                        int batch, float lr, float pos_weight, uint64_t epoch_seed,
                        double* mean_loss, void* stream) {
  if (!st || !st->params || !st->adam_m || !st->adam_v || !st->params_half || !st->grad ||
      !st->loss || !x || !y || n <= 0 || batch <= 0)
    return AMR_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  // an arithmetic progression mod n visits every sample once per epoch
  int64_t mul = (int64_t)(mlp::splitmix64(epoch_seed) % (uint64_t)n) | 1;
  while (gcd64(mul, n) != 1) mul += 2;
  const int64_t off = (int64_t)(mlp::splitmix64(epoch_seed + 1) % (uint64_t)n);
  if (cudaMemsetAsync(st->loss, 0, sizeof(float), s) != cudaSuccess) return AMR_E_CUDA;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  amr_mlp_state* mst = const_cast<amr_mlp_state*>(st);
  for (int64_t b0 = 0; b0 < n; b0 += batch) {
    const int64_t bn = std::min<int64_t>(batch, n - b0);
    if (cudaMemsetAsync(st->grad, 0, sizeof(float) * mlp::NP, s) != cudaSuccess) return AMR_E_CUDA;
    int rc = launch_grad(st->params, x, y, n, b0, bn, mul, off, pos_weight, st->grad, st->loss, s);
    if (rc != AMR_OK) return rc;
    mst->step += 1;
    const float bc1 = 1.f - powf(b1, (float)mst->step);
    const float bc2 = 1.f - powf(b2, (float)mst->step);
    mlp::k_adam<<<(mlp::NP + 255) / 256, 256, 0, s>>>(st->params, st->adam_m, st->adam_v,
                                                      (__half*)st->params_half, st->grad,
                                                      1.f / (float)bn, lr, b1, b2, eps, bc1, bc2);
  }
  if (cudaGetLastError() != cudaSuccess) return AMR_E_CUDA;
  if (mean_loss) {
    float l = 0.f;
    if (cudaMemcpyAsync(&l, st->loss, sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return AMR_E_CUDA;
    *mean_loss = (double)l / (double)n;
  }
  return AMR_OK;
}

int amr_mlp_infer(const void* params_half, const float* x, int64_t n, float* prob, void* stream) {
  if (!params_half || !x || !prob || n <= 0) return AMR_E_INVAL;
  mlp_infer_list((cudaStream_t)stream, params_half, x, nullptr, n, prob);
  return cudaGetLastError() == cudaSuccess ? AMR_OK : AMR_E_CUDA;
}

}  // extern "C"
