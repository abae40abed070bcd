// PageRank for callers that cannot allocate device memory while they run.
//
// gi_pagerank_static computes the same PageRank as gi_pagerank, but on CSR
// arrays the caller already holds on the device and with all working memory in
// a fixed, file-scope device array.  It calls no cudaMalloc/cudaFree and no
// allocating library routine; see include/graphit_gb.h for the contract.
#include <cuda_runtime.h>

#include <mutex>

#include "gi_internal.cuh"

namespace gi {

constexpr int64_t kStaticPrMaxN = GI_STATIC_PR_MAX_N;
constexpr int kStaticPrParts = 1024;  // FP64 partial sums of the normalisation

// Scratch: two contribution vectors (double buffer) and the partial sums.
// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) float d_static_pr_contrib[2 * kStaticPrMaxN];
static __device__ __align__(256) double d_static_pr_partial[kStaticPrParts];

// Device addresses of the arrays, looked up once per device (with that device
// current): in host code the symbol names are host-side stand-ins only.
struct StaticScratch {
  float *contrib = nullptr;
  double *partial = nullptr;
  bool ready = false;
};
static std::mutex g_static_mu;
static StaticScratch g_static[64];

static int static_scratch(StaticScratch **out) {
  int dev = 0;
  GI_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("device ordinal %d out of range", dev);
    return GI_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_static_mu);
  StaticScratch &s = g_static[dev];
  if (!s.ready) {
    GI_CUDA(cudaGetSymbolAddress(reinterpret_cast<void **>(&s.contrib), d_static_pr_contrib));
    GI_CUDA(cudaGetSymbolAddress(reinterpret_cast<void **>(&s.partial), d_static_pr_partial));
    s.ready = true;
  }
  *out = &s;
  return GI_OK;
}

__device__ __forceinline__ int32_t static_deg(const int32_t *__restrict__ off, int64_t v) {
  return __ldg(off + v + 1) - __ldg(off + v);
}

__global__ void k_spr_init(float *contrib, const int32_t *__restrict__ out_off, int64_t n, float init) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t d = static_deg(out_off, v);
    contrib[v] = d > 0 ? init / (float)d : 0.0f;
  }
}

// one warp per destination row: lanes stride over its in-edges, 4 loads in flight
__global__ void k_spr_iter(const int32_t *__restrict__ in_off, const int32_t *__restrict__ in_idx,
                           const int32_t *__restrict__ out_off, int64_t n, const float *__restrict__ cin, float *cout,
                           float *rank_out, float base, float damping) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
    const int32_t a = __ldg(in_off + v), b = __ldg(in_off + v + 1);
    float s = 0.0f;
    for (int32_t e0 = a + lane; e0 < b; e0 += 128) {
      int32_t u[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) u[j] = e0 + 32 * j < b ? __ldg(in_idx + e0 + 32 * j) : -1;
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (u[j] >= 0) s += __ldg(cin + u[j]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      const float r = fmaf(damping, s, base);
      if (rank_out) {
        rank_out[v] = r;
      } else {
        const int32_t d = static_deg(out_off, v);
        cout[v] = d > 0 ? r / (float)d : 0.0f;
      }
    }
  }
}

__global__ void k_spr_sum(const float *__restrict__ x, int64_t n, double *partial) {
  __shared__ double sw[32];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += (double)x[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sw[w];
    partial[blockIdx.x] = t;
  }
}

__global__ void k_spr_scale(float *x, int64_t n, const double *__restrict__ partial, int32_t np) {
  __shared__ double total;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < np; ++i) t += partial[i];
    total = t;
  }
  __syncthreads();
  const double inv = total != 0.0 ? 1.0 / total : 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = (float)((double)x[i] * inv);
}

}  // namespace gi

using namespace gi;

extern "C" int gi_pagerank_static(const int32_t *in_offsets, const int32_t *in_indices, const int32_t *out_offsets,
                                  int64_t n, int64_t m, float damping, int32_t iters, float *rank, void *stream) {
  GI_ARG(n >= 0 && m >= 0, "n and m must be >= 0");
  if (n > kStaticPrMaxN) {
    set_error("gi_pagerank_static handles at most %lld vertices (GI_STATIC_PR_MAX_N); got %lld",
              (long long)kStaticPrMaxN, (long long)n);
    return GI_ERR_INVALID_ARG;
  }
  if (m >= INT32_MAX) {
    set_error("graphs need m < 2^31; got m=%lld", (long long)m);
    return GI_ERR_UNSUPPORTED;
  }
  GI_ARG(iters >= 0, "iters must be >= 0");
  GI_ARG(damping >= 0.0f && damping <= 1.0f, "damping must be in [0,1]");
  if (n == 0) return GI_OK;
  GI_ARG(in_offsets != nullptr && rank != nullptr && (m == 0 || in_indices != nullptr), "NULL device pointer");
  StaticScratch *sc = nullptr;
  GI_TRY(static_scratch(&sc));
  cudaStream_t s = (cudaStream_t)stream;
  const int32_t *oo = out_offsets ? out_offsets : in_offsets;
  float *buf[2] = {sc->contrib, sc->contrib + kStaticPrMaxN};
  const float base = (1.0f - damping) / (float)n, init = 1.0f / (float)n;
  int sms = 0, dev = 0;
  GI_CUDA(cudaGetDevice(&dev));
  GI_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int vgrid = (int)((n + 255) / 256 < (int64_t)sms * 8 ? (n + 255) / 256 : (int64_t)sms * 8);
  const int wgrid = (int)((n * 32 + 255) / 256 < (int64_t)sms * 16 ? (n * 32 + 255) / 256 : (int64_t)sms * 16);
  k_spr_init<<<vgrid, 256, 0, s>>>(buf[0], oo, n, init);
  GI_LAUNCH_CHECK();
  if (iters == 0) {
    // PR_0 = 1/n before normalisation: reuse the iteration kernel with d = 0
    k_spr_iter<<<wgrid, 256, 0, s>>>(in_offsets, in_indices, oo, n, buf[0], buf[1], rank, init, 0.0f);
    GI_LAUNCH_CHECK();
  }
  for (int32_t k = 0; k < iters; ++k) {
    const bool last = (k == iters - 1);
    k_spr_iter<<<wgrid, 256, 0, s>>>(in_offsets, in_indices, oo, n, buf[k & 1], buf[(k + 1) & 1],
                                     last ? rank : nullptr, base, damping);
    GI_LAUNCH_CHECK();
  }
  const int np = sms * 2 < kStaticPrParts ? sms * 2 : kStaticPrParts;
  k_spr_sum<<<np, 256, 0, s>>>(rank, n, sc->partial);
  GI_LAUNCH_CHECK();
  k_spr_scale<<<vgrid, 256, 0, s>>>(rank, n, sc->partial, np);
  GI_LAUNCH_CHECK();
  return GI_OK;
}
