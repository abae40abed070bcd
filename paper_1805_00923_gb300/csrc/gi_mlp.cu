// Training and batched inference of the learned direction selector (not part
// of the paper): a 16-64-64-3 perceptron with ReLU hidden layers whose outputs
// predict the log-time of SparsePush, DensePush and DensePull for one level.
//
// Layout of the 5443 parameters: W1[64][16], b1[64], W2[64][64], b2[64],
// W3[3][64], b3[3] (row-major, out x in).
#include <cuda_runtime.h>

#include "gi_internal.cuh"

namespace gi {

constexpr int kIn = 16, kHid = 64, kOut = 3;
constexpr int kP = kHid * kIn + kHid + kHid * kHid + kHid + kOut * kHid + kOut;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kHid * kIn, kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + kHid * kHid,
              kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kOut * kHid;
constexpr int kSamplesPerBlock = 64;

// sum of the mask (the loss normaliser)
__global__ void k_mask_sum(const float *__restrict__ M, int64_t count, float *out) {
  __shared__ float sw[32];
  float s = 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    s += M[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sw[w];
    atomicAdd(out, t);
  }
}

// Forward (and, with grad != null, backward) of kSamplesPerBlock samples per
// block: thread j owns hidden unit j of both layers.  Gradients accumulate in
// registers (thread j holds row j of W1 and W2 and column j of W3) and are
// added to grad once per block.  loss gets sum M (y-t)^2 / msum.
__global__ void __launch_bounds__(kHid) k_mlp(const float *__restrict__ params, const float *__restrict__ X,
                                              const float *__restrict__ T, const float *__restrict__ M, int64_t B,
                                              const float *__restrict__ msum_p, float *grad, float *loss, float *Y) {
  __shared__ float w[kP];
  __shared__ float x[kIn], h1[kHid], h2[kHid], y[kOut], dy[kOut], dh2[kHid];
  __shared__ float red[2][kOut];
  const int j = threadIdx.x, lane = j & 31, warp = j >> 5;
  for (int i = j; i < kP; i += kHid) w[i] = params[i];
  const bool train = grad != nullptr;
  const float inv_msum = train ? (*msum_p > 0.0f ? 1.0f / *msum_p : 0.0f) : 0.0f;
  float gW1[kIn], gW2[kHid], gW3[kOut], gb1 = 0.0f, gb2 = 0.0f, gb3 = 0.0f, lsum = 0.0f;
#pragma unroll
  for (int i = 0; i < kIn; ++i) gW1[i] = 0.0f;
#pragma unroll
  for (int i = 0; i < kHid; ++i) gW2[i] = 0.0f;
#pragma unroll
  for (int k = 0; k < kOut; ++k) gW3[k] = 0.0f;
  __syncthreads();
  const int64_t s0 = (int64_t)blockIdx.x * kSamplesPerBlock;
  const int64_t s1 = s0 + kSamplesPerBlock < B ? s0 + kSamplesPerBlock : B;
  for (int64_t b = s0; b < s1; ++b) {
    if (j < kIn) x[j] = X[b * kIn + j];
    __syncthreads();
    float a1 = w[kOffB1 + j];
#pragma unroll
    for (int i = 0; i < kIn; ++i) a1 = fmaf(w[kOffW1 + j * kIn + i], x[i], a1);
    h1[j] = fmaxf(a1, 0.0f);
    __syncthreads();
    float a2 = w[kOffB2 + j];
#pragma unroll 16
    for (int i = 0; i < kHid; ++i) a2 = fmaf(w[kOffW2 + j * kHid + i], h1[i], a2);
    h2[j] = fmaxf(a2, 0.0f);
    // output layer: reduce W3[k][j]*h2[j] over the 64 threads
#pragma unroll
    for (int k = 0; k < kOut; ++k) {
      float p = w[kOffW3 + k * kHid + j] * h2[j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
      if (lane == 0) red[warp][k] = p;
    }
    __syncthreads();
    if (j < kOut) {
      const float yk = w[kOffB3 + j] + red[0][j] + red[1][j];
      y[j] = yk;
      if (Y) Y[b * kOut + j] = yk;
      if (train) {
        const float r = yk - T[b * kOut + j], mk = M[b * kOut + j];
        lsum += mk * r * r;
        dy[j] = 2.0f * mk * r * inv_msum;
      }
    }
    __syncthreads();
    if (train) {
      // layer 3
      float d2 = 0.0f;
#pragma unroll
      for (int k = 0; k < kOut; ++k) {
        gW3[k] = fmaf(dy[k], h2[j], gW3[k]);
        d2 = fmaf(w[kOffW3 + k * kHid + j], dy[k], d2);
      }
      if (j < kOut) gb3 += dy[j];
      d2 = h2[j] > 0.0f ? d2 : 0.0f;
      dh2[j] = d2;
      // layer 2: row j of W2
#pragma unroll
      for (int i = 0; i < kHid; ++i) gW2[i] = fmaf(d2, h1[i], gW2[i]);
      gb2 += d2;
      __syncthreads();
      // layer 1: unit j's delta is column j of W2 against dh2
      float d1 = 0.0f;
#pragma unroll 16
      for (int i = 0; i < kHid; ++i) d1 = fmaf(w[kOffW2 + i * kHid + j], dh2[i], d1);
      d1 = h1[j] > 0.0f ? d1 : 0.0f;
#pragma unroll
      for (int i = 0; i < kIn; ++i) gW1[i] = fmaf(d1, x[i], gW1[i]);
      gb1 += d1;
    }
    __syncthreads();
  }
  if (!train) return;
#pragma unroll
  for (int i = 0; i < kIn; ++i) atomicAdd(grad + kOffW1 + j * kIn + i, gW1[i]);
  atomicAdd(grad + kOffB1 + j, gb1);
#pragma unroll
  for (int i = 0; i < kHid; ++i) atomicAdd(grad + kOffW2 + j * kHid + i, gW2[i]);
  atomicAdd(grad + kOffB2 + j, gb2);
#pragma unroll
  for (int k = 0; k < kOut; ++k) atomicAdd(grad + kOffW3 + k * kHid + j, gW3[k]);
  if (j < kOut) {
    atomicAdd(grad + kOffB3 + j, gb3);
    atomicAdd(loss, lsum * inv_msum);
  }
}

// Adam (Kingma & Ba 2015): bias-corrected first/second moments.
__global__ void k_adam(float *p, const float *__restrict__ g, float *m, float *v, int n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi_ = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi_;
    const float vi = b2 * v[i] + (1.0f - b2) * gi_ * gi_;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

}  // namespace gi

using namespace gi;

extern "C" int gi_mlp_loss_grad(const float *params, const float *X, const float *T, const float *M, int64_t B,
                                float *grad, float *loss, void *stream) {
  GI_ARG(params && X && T && M && grad && loss, "NULL device pointer");
  GI_ARG(B >= 0 && B < ((int64_t)1 << 40), "bad batch size");
  cudaStream_t s = (cudaStream_t)stream;
  GI_CUDA(cudaMemsetAsync(grad, 0, sizeof(float) * kP, s));
  GI_CUDA(cudaMemsetAsync(loss, 0, sizeof(float) * 2, s));  // loss[0] = loss, loss[1] = mask sum
  if (B == 0) return GI_OK;
  k_mask_sum<<<64, 256, 0, s>>>(M, B * kOut, loss + 1);
  GI_LAUNCH_CHECK();
  const int64_t blocks = (B + kSamplesPerBlock - 1) / kSamplesPerBlock;
  k_mlp<<<(unsigned)blocks, kHid, 0, s>>>(params, X, T, M, B, loss + 1, grad, loss, nullptr);
  GI_LAUNCH_CHECK();
  return GI_OK;
}

extern "C" int gi_mlp_forward(const float *params, const float *X, int64_t B, float *Y, void *stream) {
  GI_ARG(params && X && Y, "NULL device pointer");
  GI_ARG(B >= 0 && B < ((int64_t)1 << 40), "bad batch size");
  if (B == 0) return GI_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t blocks = (B + kSamplesPerBlock - 1) / kSamplesPerBlock;
  k_mlp<<<(unsigned)blocks, kHid, 0, s>>>(params, X, nullptr, nullptr, B, nullptr, nullptr, nullptr, Y);
  GI_LAUNCH_CHECK();
  return GI_OK;
}

extern "C" int gi_mlp_adam(float *params, const float *grad, float *m, float *v, int32_t t, float lr, float b1,
                           float b2, float eps, void *stream) {
  GI_ARG(params && grad && m && v, "NULL device pointer");
  GI_ARG(t >= 1, "Adam step number starts at 1");
  const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
  k_adam<<<div_up(kP, 256), 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, kP, lr, b1, b2, eps, c1, c2);
  GI_LAUNCH_CHECK();
  return GI_OK;
}
