// Graph storage, vertexsets, scans, pull tiles, frontier statistics and the
// direction decision (Beamer / Ligra threshold or the learned selector).
#include <cuda_runtime.h>

#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "gi_features.cuh"
#include "gi_internal.cuh"

namespace gi {

// ================================================================ errors ==
static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
  set_error("CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e), what, file, line);
  return e == cudaErrorMemoryAllocation ? GI_ERR_OOM : GI_ERR_CUDA;
}

// ======================================================= launch accounting ==
static std::atomic<long long> g_launches{0};
static std::atomic<bool> g_timing{false};
struct TimedRec {
  int kclass;
  cudaEvent_t a, b;
};
static std::mutex g_timing_mu;
static std::vector<TimedRec> g_recs;
static std::vector<cudaEvent_t> g_event_pool;

void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int launch_status(int n) {
  note_launch(n);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch", __FILE__, __LINE__);
  return GI_OK;
}

static cudaEvent_t pool_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

bool timing_on() { return g_timing.load(std::memory_order_relaxed); }

int timing_begin(int kclass, cudaStream_t s) {
  if (!g_timing.load(std::memory_order_relaxed)) return -1;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return -1;  // graph capture
  std::lock_guard<std::mutex> lk(g_timing_mu);
  TimedRec r{kclass, pool_event(), pool_event()};
  if (!r.a || !r.b) return -1;
  cudaEventRecord(r.a, s);
  g_recs.push_back(r);
  return (int)g_recs.size() - 1;
}

void timing_end(int token, cudaStream_t s) {
  if (token < 0) return;
  std::lock_guard<std::mutex> lk(g_timing_mu);
  if (token < (int)g_recs.size()) cudaEventRecord(g_recs[token].b, s);
}

// ============================================================ allocation ==
// Stream-ordered allocations from the device's default pool; the pool keeps
// freed memory (release threshold = max) so repeated graph loads reuse it.
static std::once_flag g_pool_once[64];

// test hook: after g_alloc_budget more successes every allocation fails (< 0: off)
static std::atomic<long long> g_alloc_budget{-1};

int dev_alloc(void **p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  if (g_alloc_budget.load() >= 0 && g_alloc_budget.fetch_sub(1) <= 0) {
    g_alloc_budget.store(0);
    set_error("device allocation of %zu bytes refused by the fault-injection hook", bytes);
    return GI_ERR_OOM;
  }
  int dev = 0;
  GI_CUDA(cudaGetDevice(&dev));
  if (dev >= 0 && dev < 64) {
    std::call_once(g_pool_once[dev], [dev]() {
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
      }
    });
  }
  cudaError_t e = cudaMallocAsync(p, bytes, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    set_error("device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    return GI_ERR_OOM;
  }
  return GI_OK;
}

void dev_free(void *p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

// Pinned host control blocks (kCtrlWords int64 each, one per graph), carved
// from 64 KB slabs that live as long as the process: pinning and unpinning
// host memory per graph costs more than the rest of a small graph's load,
// and cudaFreeHost synchronises the device.
static std::mutex g_pinned_mu;
static std::vector<int64_t *> g_pinned_free;

static int pinned_ctrl_get(int64_t **out) {
  std::lock_guard<std::mutex> lock(g_pinned_mu);
  if (g_pinned_free.empty()) {
    constexpr size_t kSlab = 64 * 1024, kBlock = sizeof(int64_t) * kCtrlWords;
    void *slab = nullptr;
    if (cudaHostAlloc(&slab, kSlab, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      set_error("pinned host allocation failed");
      return GI_ERR_OOM;
    }
    for (size_t off = 0; off + kBlock <= kSlab; off += kBlock)
      g_pinned_free.push_back(reinterpret_cast<int64_t *>(static_cast<char *>(slab) + off));
  }
  *out = g_pinned_free.back();
  g_pinned_free.pop_back();
  memset(*out, 0, sizeof(int64_t) * kCtrlWords);
  return GI_OK;
}

static void pinned_ctrl_put(int64_t *p) {
  if (!p) return;
  std::lock_guard<std::mutex> lock(g_pinned_mu);
  g_pinned_free.push_back(p);
}

// One non-blocking stream per device for the side copies of graph loads,
// created on first use and kept: the loads order their work on it with events.
static std::once_flag g_side_once[64];
static cudaStream_t g_side_stream[64];

static int side_stream(int dev, cudaStream_t *out) {
  if (dev < 0 || dev >= 64) {
    set_error("device %d out of range", dev);
    return GI_ERR_UNSUPPORTED;
  }
  std::call_once(g_side_once[dev], [dev]() {
    if (cudaStreamCreateWithFlags(&g_side_stream[dev], cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      g_side_stream[dev] = nullptr;
    }
  });
  if (!g_side_stream[dev]) {
    set_error("side copy stream could not be created");
    return GI_ERR_CUDA;
  }
  *out = g_side_stream[dev];
  return GI_OK;
}

int bfs_defer_get(gi_graph *g, cudaStream_t s) {
  if (g->bfs_defer) return GI_OK;
  // the deferred-scan kernel returns counter and ticket to zero after each use
  GI_TRY(dev_alloc(&g->bfs_defer, 16 + 16 * (size_t)bfs_defer_cap(g->m), s));
  GI_CUDA(cudaMemsetAsync(g->bfs_defer, 0, 16, s));
  return GI_OK;
}

__global__ void k_has_in_arcs(const int32_t *__restrict__ ptr, int64_t n, int32_t *flag) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    flag[v] = __ldg(ptr + v + 1) > __ldg(ptr + v) ? 1 : 0;
}

__global__ void k_live_scatter(const int32_t *__restrict__ flag, const int32_t *__restrict__ pos, int64_t n,
                               int32_t *live) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    if (flag[v]) live[pos[v]] = (int32_t)v;
}

int bfs_unv_get(gi_graph *g, cudaStream_t s, BfsUnv *out) {
  if (!g->bfs_unv) {
    // vertices with in-arcs, ascending: flags, exclusive scan, scatter
    int32_t *flag = nullptr, *pos = nullptr;
    GI_TRY(ws_scratch(g, &flag, &pos, s));
    k_has_in_arcs<<<grid_for(g, g->n, 256), 256, 0, s>>>(g->in.ptr, g->n, flag);
    GI_LAUNCH_CHECK();
    GI_TRY(scan_exclusive(g, flag, pos, g->n, s));
    int32_t total = 0;
    GI_CUDA(cudaMemcpyAsync(&total, pos + g->n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    GI_CUDA(cudaStreamSynchronize(s));
    // st (4 words, padded to 16 bytes), live, list0, list1
    const size_t len = (size_t)(total > 0 ? total : 1);
    void *mem = nullptr;
    GI_TRY(dev_alloc(&mem, 16 + 3 * sizeof(int32_t) * len, s));
    int32_t *live = reinterpret_cast<int32_t *>(static_cast<unsigned char *>(mem) + 16);
    k_live_scatter<<<grid_for(g, g->n, 256), 256, 0, s>>>(flag, pos, g->n, live);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      dev_free(mem, s);
      return cuda_fail(e, "live list", __FILE__, __LINE__);
    }
    g->bfs_unv = mem;
    g->bfs_unv_n = total;
  }
  const size_t len = (size_t)(g->bfs_unv_n > 0 ? g->bfs_unv_n : 1);
  unsigned char *b = static_cast<unsigned char *>(g->bfs_unv);
  out->st = reinterpret_cast<int32_t *>(b);
  out->live = reinterpret_cast<const int32_t *>(b + 16);
  out->list0 = reinterpret_cast<int32_t *>(b + 16) + len;
  out->list1 = out->list0 + len;
  out->nlive = g->bfs_unv_n;
  return GI_OK;
}

void bfs_unv_free(gi_graph *g, cudaStream_t s) {
  dev_free(g->bfs_unv, s);
  g->bfs_unv = nullptr;
  g->bfs_unv_n = 0;
  g->bfs_unv_query = BfsUnv{};
}

int heavy_get(gi_graph *g, cudaStream_t s) {
  if (g->heavy_mem) return GI_OK;
  // the expansion kernel returns counter and ticket to zero after each use
  GI_TRY(dev_alloc(&g->heavy_mem, 16 + 8 * (size_t)(g->n > 0 ? g->n : 1), s));
  GI_CUDA(cudaMemsetAsync(g->heavy_mem, 0, 16, s));
  return GI_OK;
}

int grid_for(const gi_graph *g, int64_t work, int block, int per_sm) {
  int64_t want = (work + block - 1) / block;
  int64_t cap = (int64_t)g->num_sms * per_sm;
  if (want < 1) want = 1;
  return (int)(want < cap ? want : cap);
}

// ============================================================= workspace ==
struct Workspace {
  int32_t *scan_blocks = nullptr;  // block sums for scans
  int64_t scan_cap = 0;
  int32_t *tmp_i32 = nullptr;      // n+1 scratch
  int32_t *tmp2_i32 = nullptr;     // n+1 scratch
};

static void ws_free(gi_graph *g, cudaStream_t s);

static int ws_get(gi_graph *g, cudaStream_t s) {
  if (g->ws) return GI_OK;
  g->ws = new Workspace();
  int64_t nb = (g->n + 2047) / 2048 + 2;
  nb = nb < ((g->m + 255) / 256 + 2) ? ((g->m + 255) / 256 + 2) : nb;  // tile counts can exceed n/2048
  int st = dev_alloc_n(&g->ws->scan_blocks, nb + 2048, s);
  g->ws->scan_cap = nb + 2048;
  if (st == GI_OK) st = dev_alloc_n(&g->ws->tmp_i32, g->n + 2, s);
  if (st == GI_OK) st = dev_alloc_n(&g->ws->tmp2_i32, g->n + 2, s);
  if (st != GI_OK) ws_free(g, s);  // all or nothing
  return st;
}

static void ws_free(gi_graph *g, cudaStream_t s) {
  if (!g->ws) return;
  dev_free(g->ws->scan_blocks, s);
  dev_free(g->ws->tmp_i32, s);
  dev_free(g->ws->tmp2_i32, s);
  delete g->ws;
  g->ws = nullptr;
}

int ws_scratch(gi_graph *g, int32_t **a, int32_t **b, cudaStream_t s) {
  GI_TRY(ws_get(g, s));
  *a = g->ws->tmp_i32;
  *b = g->ws->tmp2_i32;
  return GI_OK;
}

// ================================================================== scan ==
// Three-phase exclusive scan of int32 counts: per-block scan of 2048 items,
// scan of the block totals by one block, then add the block offsets.
constexpr int kScanThreads = 256, kScanItems = 8, kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t *total, int32_t *smem_warp) {
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) smem_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int32_t w = lane < nw ? smem_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) smem_warp[lane] = w;
  }
  __syncthreads();
  int32_t warp_off = warp > 0 ? smem_warp[warp - 1] : 0;
  *total = smem_warp[nw - 1];
  __syncthreads();
  return warp_off + x - v;
}

__global__ void k_scan_blocks(const int32_t *__restrict__ in, int32_t *__restrict__ out, int64_t n,
                              int32_t *__restrict__ block_sums) {
  __shared__ int32_t s[kScanTile];
  __shared__ int32_t sw[32];
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + threadIdx.x + k * kScanThreads;
    s[threadIdx.x + k * kScanThreads] = i < n ? in[i] : 0;
  }
  __syncthreads();
  int32_t loc[kScanItems], sum = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    loc[k] = sum;
    sum += s[threadIdx.x * kScanItems + k];
  }
  int32_t total;
  int32_t off = block_exclusive_scan(sum, &total, sw);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) s[threadIdx.x * kScanItems + k] = loc[k] + off;
  __syncthreads();
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + threadIdx.x + k * kScanThreads;
    if (i < n) out[i] = s[threadIdx.x + k * kScanThreads];
  }
  if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

// single block: exclusive scan of nb block sums in place; writes grand total to *total_out
__global__ void k_scan_top(int32_t *sums, int64_t nb, int32_t *total_out) {
  __shared__ int32_t sw[32];
  int32_t carry = 0;
  for (int64_t base = 0; base < nb; base += kScanThreads) {
    int64_t i = base + threadIdx.x;
    int32_t v = i < nb ? sums[i] : 0;
    int32_t total;
    int32_t ex = block_exclusive_scan(v, &total, sw);
    if (i < nb) sums[i] = ex + carry;
    carry += total;
  }
  if (threadIdx.x == 0) *total_out = carry;
}

__global__ void k_scan_add(int32_t *out, int64_t n, const int32_t *__restrict__ block_off) {
  int64_t i = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
  int32_t off = block_off[blockIdx.x];
  for (int k = 0; k < kScanItems; ++k, i += kScanThreads)
    if (i < n) out[i] += off;
}

int scan_exclusive(gi_graph *g, const int32_t *in, int32_t *out, int64_t n, cudaStream_t s) {
  GI_TRY(ws_get(g, s));
  int64_t nb = (n + kScanTile - 1) / kScanTile;
  if (nb + 1 > g->ws->scan_cap) {
    set_error("scan of %lld items exceeds workspace", (long long)n);
    return GI_ERR_UNSUPPORTED;
  }
  if (nb > 0) {
    k_scan_blocks<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, g->ws->scan_blocks);
    GI_LAUNCH_CHECK();
  }
  k_scan_top<<<1, kScanThreads, 0, s>>>(g->ws->scan_blocks, nb, out + n);
  GI_LAUNCH_CHECK();
  if (nb > 0) {
    k_scan_add<<<(unsigned)nb, kScanThreads, 0, s>>>(out, n, g->ws->scan_blocks);
    GI_LAUNCH_CHECK();
  }
  return GI_OK;
}

// ============================================================ graph load ==
__global__ void k_validate(const int32_t *__restrict__ ptr, const int32_t *__restrict__ idx, int64_t n, int64_t m,
                           int64_t *err) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    int32_t a = ptr[v], b = ptr[v + 1];
    if (a > b || a < 0 || b > m) {
      atomicCAS(reinterpret_cast<unsigned long long *>(err), 0ull, (unsigned long long)(1 + v));
      continue;
    }
    for (int32_t e = a; e < b; ++e) {
      int32_t u = idx[e];
      if (u < 0 || u >= n || (e > a && idx[e - 1] >= u))
        atomicCAS(reinterpret_cast<unsigned long long *>(err), 0ull, (unsigned long long)(1 + v));
    }
  }
}

__global__ void k_degrees(const int32_t *__restrict__ ptr, int64_t n, int32_t *__restrict__ deg,
                          float *__restrict__ inv, int32_t *__restrict__ max_deg) {
  int32_t local_max = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    int32_t d = ptr[v + 1] - ptr[v];
    deg[v] = d;
    inv[v] = d > 0 ? 1.0f / (float)d : 0.0f;
    local_max = d > local_max ? d : local_max;
  }
  for (int o = 16; o > 0; o >>= 1) local_max = max(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
  if ((threadIdx.x & 31) == 0) atomicMax(max_deg, local_max);
}

__global__ void k_sum_weights(const int32_t *__restrict__ wt, int64_t m, unsigned long long *out) {
  unsigned long long s = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
    s += (unsigned long long)(long long)wt[e];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

static int copy_in(int32_t **dst, const int32_t *src, int64_t count, uint32_t flags, cudaStream_t s) {
  GI_TRY(dev_alloc_n(dst, count, s));
  if (count > 0)
    GI_CUDA(cudaMemcpyAsync(*dst, src, sizeof(int32_t) * (size_t)count,
                            (flags & GI_HOST_PTRS) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
  return GI_OK;
}

// The index and weight arrays of a load are copied on a side stream in up to
// kChunks pieces, one event per piece, so that the degree, tile and hot-set
// work on the caller's stream runs under the copy (host-to-device copies are
// bound by the host link, ~210 GB/s on a GB300 node, not by the SMs), and
// the hot-set remap of each piece starts as soon as the piece has landed.
struct SideCopy {
  static constexpr int kChunks = 8;
  cudaStream_t cs = nullptr;
  cudaEvent_t done[kChunks] = {}, wt_done = nullptr;
  int64_t cut[kChunks + 1] = {};
  int chunks = 0, waited = 0;
  bool recorded = true;  // every copy enqueued so far is covered by an event

  int start(gi_graph *g, Csr *c, const int32_t *idx, const int32_t *wt, uint32_t flags, cudaStream_t s) {
    const int64_t m = g->m;
    GI_TRY(dev_alloc_n(&c->idx, m, s));
    if (wt) GI_TRY(dev_alloc_n(&c->wt, m, s));
    if (m == 0) return GI_OK;
    const cudaMemcpyKind kind = (flags & GI_HOST_PTRS) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    GI_TRY(side_stream(g->device, &cs));
    recorded = false;
    cudaEvent_t ready = nullptr;
    GI_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    cudaError_t e = cudaEventRecord(ready, s);  // the allocations above, and any producer of device inputs
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ready, 0);
    cudaEventDestroy(ready);
    if (e != cudaSuccess) return cuda_fail(e, "side copy stream", __FILE__, __LINE__);
    const int64_t want = m >> 22;  // pieces of at least 4M arcs
    chunks = want < 1 ? 1 : (want > kChunks ? kChunks : (int)want);
    for (int i = 0; i <= chunks; ++i) cut[i] = m * i / chunks;
    for (int i = 0; i < chunks; ++i) {
      GI_CUDA(cudaMemcpyAsync(c->idx + cut[i], idx + cut[i], sizeof(int32_t) * (size_t)(cut[i + 1] - cut[i]), kind,
                              cs));
      GI_CUDA(cudaEventCreateWithFlags(&done[i], cudaEventDisableTiming));
      GI_CUDA(cudaEventRecord(done[i], cs));
    }
    if (wt) {
      GI_CUDA(cudaMemcpyAsync(c->wt, wt, sizeof(int32_t) * (size_t)m, kind, cs));
      GI_CUDA(cudaEventCreateWithFlags(&wt_done, cudaEventDisableTiming));
      GI_CUDA(cudaEventRecord(wt_done, cs));
    }
    recorded = true;
    return GI_OK;
  }
  // s waits for pieces [0, upto)
  int wait(int upto, cudaStream_t s) {
    for (; waited < upto && waited < chunks; ++waited) GI_CUDA(cudaStreamWaitEvent(s, done[waited], 0));
    return GI_OK;
  }
  int wait_weights(cudaStream_t s) {
    if (wt_done) GI_CUDA(cudaStreamWaitEvent(s, wt_done, 0));
    return GI_OK;
  }
  int wait_all(cudaStream_t s) {
    if (wt_done) GI_CUDA(cudaStreamWaitEvent(s, wt_done, 0));
    return wait(chunks, s);
  }
  // this load's copies have finished (or never started) when this returns
  void release() {
    if (cs && !recorded) cudaStreamSynchronize(cs);  // a start() that failed half way
    for (auto &ev : done)
      if (ev) cudaEventSynchronize(ev);
    if (wt_done) cudaEventSynchronize(wt_done);
    for (auto &ev : done)
      if (ev) cudaEventDestroy(ev);
    if (wt_done) cudaEventDestroy(wt_done);
    cs = nullptr;
    wt_done = nullptr;
    for (auto &ev : done) ev = nullptr;
  }
};

static int hot_build_overlapped(gi_graph *g, SideCopy &sc, cudaStream_t s);

static int validate_csr_dev(gi_graph *g, const Csr &c, cudaStream_t s) {
  GI_CUDA(cudaMemsetAsync(g->ctrl + kErr, 0, sizeof(int64_t), s));
  k_validate<<<grid_for(g, g->n, 256), 256, 0, s>>>(c.ptr, c.idx, g->n, g->m, g->ctrl + kErr);
  GI_LAUNCH_CHECK();
  int32_t first_last[2];
  GI_CUDA(cudaMemcpyAsync(&first_last[0], c.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  GI_CUDA(cudaMemcpyAsync(&first_last[1], c.ptr + g->n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  int64_t err = 0;
  GI_CUDA(cudaMemcpyAsync(&err, g->ctrl + kErr, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GI_CUDA(cudaStreamSynchronize(s));
  if (first_last[0] != 0 || first_last[1] != g->m) {
    set_error("bad graph: offsets[0]=%d offsets[n]=%d, expected 0 and %lld", first_last[0], first_last[1],
              (long long)g->m);
    return GI_ERR_BAD_GRAPH;
  }
  if (err) {
    set_error("bad graph: row %lld has non-monotone offsets, an index out of range or an unsorted/duplicate entry",
              (long long)(err - 1));
    return GI_ERR_BAD_GRAPH;
  }
  return GI_OK;
}

}  // namespace gi

using namespace gi;

extern "C" const char *gi_last_error(void) { return g_err; }

extern "C" int gi_debug_fail_allocs_after(int64_t n) {
  g_alloc_budget.store(n < 0 ? -1 : n);
  return GI_OK;
}

extern "C" int gi_debug_pool_used(int64_t *bytes) {
  GI_ARG(bytes != nullptr, "NULL output");
  int dev = 0;
  GI_CUDA(cudaGetDevice(&dev));
  cudaMemPool_t pool;
  GI_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
  uint64_t used = 0;
  GI_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used));
  *bytes = (int64_t)used;
  return GI_OK;
}

extern "C" int gi_stats_enable(int timing_on) {
  g_timing.store(timing_on != 0);
  return GI_OK;
}

extern "C" int gi_stats_reset(void) {
  std::lock_guard<std::mutex> lk(g_timing_mu);
  for (auto &r : g_recs) {
    g_event_pool.push_back(r.a);
    g_event_pool.push_back(r.b);
  }
  g_recs.clear();
  g_launches.store(0);
  return GI_OK;
}

extern "C" int gi_stats_read(int32_t kclass, int64_t *launches, int64_t *timed_launches, double *timed_ms) {
  GI_ARG(kclass >= -1 && kclass < kNumClasses, "unknown kernel class");
  std::lock_guard<std::mutex> lk(g_timing_mu);
  if (launches) *launches = g_launches.load();
  int64_t cnt = 0;
  double ms = 0.0;
  for (auto &r : g_recs) {
    if (kclass >= 0 && r.kclass != kclass) continue;
    GI_CUDA(cudaEventSynchronize(r.b));
    float t = 0.0f;
    GI_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
    ms += t;
    ++cnt;
  }
  if (timed_launches) *timed_launches = cnt;
  if (timed_ms) *timed_ms = ms;
  return GI_OK;
}
extern "C" int gi_stats_pull_arcs(gi_graph *g, int32_t reset, int64_t *arcs) {
  GI_ARG(g != nullptr && arcs != nullptr, "NULL argument");
  GI_CUDA(cudaDeviceSynchronize());
  GI_CUDA(cudaMemcpy(arcs, g->ctrl + kPullArcs, sizeof(int64_t), cudaMemcpyDeviceToHost));
  if (reset) GI_CUDA(cudaMemset(g->ctrl + kPullArcs, 0, sizeof(int64_t)));
  return GI_OK;
}

extern "C" int gi_version(void) { return 100; }

namespace gi {
// Ceiling of the pull's gathers: stream m source ids with 16-byte loads and
// gather one 4-byte value per id (each a separate 32-byte sector unless a
// neighbouring id shares it), nothing else; the sum keeps the loads alive.
__global__ void __launch_bounds__(256) k_gather_rate(const int32_t *__restrict__ idx, int64_t m,
                                                     const float *__restrict__ table, float *out) {
  const int64_t m4 = m >> 2;
  const int4 *idx4 = reinterpret_cast<const int4 *>(idx);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  float acc = 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m4; i += 2 * stride) {
    const int4 a = __ldg(idx4 + i);
    int4 b = make_int4(-1, -1, -1, -1);
    if (i + stride < m4) b = __ldg(idx4 + i + stride);
    acc += __ldg(table + a.x) + __ldg(table + a.y) + __ldg(table + a.z) + __ldg(table + a.w);
    if (b.x >= 0) acc += __ldg(table + b.x) + __ldg(table + b.y) + __ldg(table + b.z) + __ldg(table + b.w);
  }
  for (int64_t i = (m4 << 2) + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride)
    acc += __ldg(table + __ldg(idx + i));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc == -1.0f) out[0] = acc;  // practically never: keeps the sum live
}
}  // namespace gi

extern "C" int gi_gather_rate(const int32_t *idx, int64_t m, const float *table, int64_t n, float *out,
                              void *stream) {
  GI_ARG(m >= 0 && n > 0, "m must be >= 0 and n > 0");
  GI_ARG((idx != nullptr || m == 0) && table != nullptr && out != nullptr, "NULL device pointer");
  GI_ARG((reinterpret_cast<uintptr_t>(idx) & 15) == 0, "idx must be 16-byte aligned");
  if (m == 0) return GI_OK;
  int dev = 0, sms = 0;
  GI_CUDA(cudaGetDevice(&dev));
  GI_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  gi::k_gather_rate<<<sms * 8, 256, 0, (cudaStream_t)stream>>>(idx, m, table, out);
  GI_LAUNCH_CHECK();
  return GI_OK;
}

namespace gi {
static void segs_free(gi_graph *g, cudaStream_t s);
}

static void graph_release(gi_graph *g, cudaStream_t s) {
  if (!g) return;
  graph_loop_free(g);
  dstep_free(g, s);
  free_tile_cache(g, s);
  segs_free(g, s);
  if (!g->symmetric) {
    dev_free(g->in.ptr, s);
    dev_free(g->in.idx, s);
    dev_free(g->in.wt, s);
  }
  dev_free(g->out.ptr, s);
  dev_free(g->out.idx, s);
  dev_free(g->out.wt, s);
  dev_free(g->out_deg, s);
  dev_free(g->inv_out_deg, s);
  dev_free(g->ctrl, s);
  dev_free(g->heavy_mem, s);
  dev_free(g->bfs_defer, s);
  bfs_unv_free(g, s);
  ws_free(g, s);
  pinned_ctrl_put(g->ctrl_host);
  delete g;
}

extern "C" int gi_load_csr(const int32_t *offsets, const int32_t *indices, const int32_t *weights, int64_t n,
                           int64_t m, uint32_t flags, void *stream, gi_graph **out) {
  GI_ARG(out != nullptr, "out is NULL");
  *out = nullptr;
  GI_ARG(n >= 0 && m >= 0, "n and m must be >= 0");
  GI_ARG(((flags & GI_HOST_PTRS) != 0) != ((flags & GI_DEV_PTRS) != 0), "exactly one of GI_HOST_PTRS/GI_DEV_PTRS");
  GI_ARG(offsets != nullptr, "offsets is NULL");
  GI_ARG(m == 0 || indices != nullptr, "indices is NULL");
  if (n >= INT32_MAX || m >= INT32_MAX) {
    set_error("graphs need n, m < 2^31 (int32 ids and offsets); got n=%lld m=%lld", (long long)n, (long long)m);
    return GI_ERR_UNSUPPORTED;
  }
  cudaStream_t s = (cudaStream_t)stream;
  gi_graph *g = new gi_graph();
  g->n = n;
  g->m = m;
  g->symmetric = (flags & GI_SYMMETRIC) != 0;
  int st = GI_OK;
  SideCopy side;
  do {
    if (cudaGetDevice(&g->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess) {
      st = cuda_fail(cudaGetLastError(), "device query", __FILE__, __LINE__);
      break;
    }
    if ((st = dev_alloc_n(&g->ctrl, kCtrlWords, s)) != GI_OK) break;
    if (cudaMemsetAsync(g->ctrl, 0, sizeof(int64_t) * kCtrlWords, s) != cudaSuccess) { st = GI_ERR_CUDA; break; }
    if ((st = pinned_ctrl_get(&g->ctrl_host)) != GI_OK) break;
    if ((st = copy_in(&g->out.ptr, offsets, n + 1, flags, s)) != GI_OK) break;
    if ((st = side.start(g, &g->out, indices, weights, flags, s)) != GI_OK) break;
    if ((flags & GI_VALIDATE) && ((st = side.wait_all(s)) != GI_OK || (st = validate_csr_dev(g, g->out, s)) != GI_OK))
      break;
    if ((st = dev_alloc_n(&g->out_deg, n, s)) != GI_OK) break;
    if ((st = dev_alloc_n(&g->inv_out_deg, n, s)) != GI_OK) break;
    if (cudaMemsetAsync(g->ctrl + kErr, 0, sizeof(int64_t), s) != cudaSuccess) { st = GI_ERR_CUDA; break; }
    k_degrees<<<grid_for(g, n, 256), 256, 0, s>>>(g->out.ptr, n, g->out_deg, g->inv_out_deg,
                                                  reinterpret_cast<int32_t *>(g->ctrl + kErr));
    if ((st = launch_status(1)) != GI_OK) break;
    int64_t md = 0;
    if (cudaMemcpyAsync(&md, g->ctrl + kErr, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      st = cuda_fail(cudaGetLastError(), "max degree", __FILE__, __LINE__);
      break;
    }
    g->max_deg = (int32_t)(md & 0xffffffff);
    if (g->symmetric) {
      g->in = g->out;
      g->has_csc = true;
      if ((st = use_tiles(g, 2048, s)) != GI_OK) break;
      if ((flags & GI_HOT_SOURCES) && (st = hot_build_overlapped(g, side, s)) != GI_OK) break;
    }
    if (weights && m > 0) {
      unsigned long long wsum = 0;
      if ((st = side.wait_weights(s)) != GI_OK) break;
      if (cudaMemsetAsync(g->ctrl + kErr, 0, sizeof(int64_t), s) != cudaSuccess) { st = GI_ERR_CUDA; break; }
      k_sum_weights<<<grid_for(g, m, 256), 256, 0, s>>>(g->out.wt, m,
                                                        reinterpret_cast<unsigned long long *>(g->ctrl + kErr));
      if ((st = launch_status(1)) != GI_OK) break;
      if (cudaMemcpyAsync(&wsum, g->ctrl + kErr, sizeof(wsum), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) {
        st = cuda_fail(cudaGetLastError(), "weight sum", __FILE__, __LINE__);
        break;
      }
      g->wt_mean = (double)(long long)wsum / (double)m;
    }
    if ((st = side.wait_all(s)) != GI_OK) break;
    if (cudaStreamSynchronize(s) != cudaSuccess) {
      st = cuda_fail(cudaGetLastError(), "load sync", __FILE__, __LINE__);
      break;
    }
  } while (0);
  side.release();  // no copy may still write into memory that graph_release frees
  if (st != GI_OK) {
    cudaStreamSynchronize(s);
    graph_release(g, s);
    return st;
  }
  *out = g;
  return GI_OK;
}

extern "C" int gi_load_csc(gi_graph *g, const int32_t *in_offsets, const int32_t *in_indices,
                           const int32_t *in_weights, uint32_t flags, void *stream) {
  GI_ARG(g != nullptr, "graph is NULL");
  GI_ARG(in_offsets != nullptr && (g->m == 0 || in_indices != nullptr), "in-edge arrays are NULL");
  GI_ARG(((flags & GI_HOST_PTRS) != 0) != ((flags & GI_DEV_PTRS) != 0), "exactly one of GI_HOST_PTRS/GI_DEV_PTRS");
  cudaStream_t s = (cudaStream_t)stream;
  if (g->symmetric) return GI_OK;  // the CSR already is the in-edge view
  graph_loop_free(g);              // its kernels hold the in-edge arrays
  bfs_unv_free(g, s);              // built from the in-edges
  if (g->has_csc) {
    free_tile_cache(g, s);
    dev_free(g->in.ptr, s);
    dev_free(g->in.idx, s);
    dev_free(g->in.wt, s);
    g->in = Csr();
    g->has_csc = false;
  }
  GI_TRY(copy_in(&g->in.ptr, in_offsets, g->n + 1, flags, s));
  SideCopy side;
  int st = side.start(g, &g->in, in_indices, in_weights, flags, s);
  if (st == GI_OK && (flags & GI_VALIDATE) && (st = side.wait_all(s)) == GI_OK) st = validate_csr_dev(g, g->in, s);
  if (st == GI_OK) {
    g->has_csc = true;
    st = use_tiles(g, 2048, s);
  }
  if (st == GI_OK && (flags & GI_HOT_SOURCES)) st = hot_build_overlapped(g, side, s);
  if (st == GI_OK) st = side.wait_all(s);
  if (st == GI_OK && cudaStreamSynchronize(s) != cudaSuccess)
    st = cuda_fail(cudaGetLastError(), "load sync", __FILE__, __LINE__);
  side.release();
  return st;
}

extern "C" int gi_graph_free(gi_graph *g) {
  if (!g) return GI_OK;
  cudaStream_t s = 0;
  cudaDeviceSynchronize();
  graph_release(g, s);
  GI_CUDA(cudaStreamSynchronize(s));
  return GI_OK;
}

extern "C" int gi_graph_info(const gi_graph *g, int64_t *n, int64_t *m, int32_t *max_deg) {
  GI_ARG(g != nullptr, "graph is NULL");
  if (n) *n = g->n;
  if (m) *m = g->m;
  if (max_deg) *max_deg = g->max_deg;
  return GI_OK;
}

extern "C" int gi_graph_device_csr(const gi_graph *g, const int32_t **offsets, const int32_t **indices,
                                   const int32_t **weights) {
  GI_ARG(g != nullptr, "graph is NULL");
  if (offsets) *offsets = g->out.ptr;
  if (indices) *indices = g->out.idx;
  if (weights) *weights = g->out.wt;
  return GI_OK;
}

namespace gi {

// ================================================================= tiles ==
// Row r starts a short tile when it is short and (r is the first row, the
// previous row is long, r is a multiple of kTileRows, or ptr[r] lies in a
// different tile_edges bucket than ptr[r-1]).  Rows with degree above
// tile_edges/kLongRowDiv get ceil(deg/tile_edges) tiles of their own.  So a
// short tile holds at most kTileRows rows and fewer than
// tile_edges*(1+1/kLongRowDiv) arcs.
__global__ void k_tile_count(const int32_t *__restrict__ ptr, int64_t n, int32_t te, int32_t rows_max, int32_t *cnt,
                             int32_t *split_cnt) {
  const int32_t t_long = te / kLongRowDiv;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    int32_t a = ptr[r], d = ptr[r + 1] - a;
    int32_t c, sc = 0;
    if (d > t_long) {
      c = (d + te - 1) / te;
      sc = c > 1 ? 1 : 0;
    } else if (r == 0 || (r % rows_max) == 0) {
      c = 1;
    } else {
      int32_t pa = ptr[r - 1];
      bool prev_long = (a - pa) > t_long;
      c = (prev_long || (a / te) != (pa / te)) ? 1 : 0;
    }
    cnt[r] = c;
    split_cnt[r] = sc;
  }
}

__global__ void k_tile_write(const int32_t *__restrict__ ptr, int64_t n, int32_t te, const int32_t *__restrict__ off,
                             const int32_t *__restrict__ soff, int4 *tiles, int4 *splits, int32_t *tile_row) {
  const int32_t t_long = te / kLongRowDiv;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    int32_t c = off[r + 1] - off[r];
    if (c == 0) continue;
    int32_t t = off[r];
    int32_t a = ptr[r], d = ptr[r + 1] - a;
    if (d > t_long) {
      for (int32_t k = 0; k < c; ++k) {
        int32_t e0 = a + k * te, e1 = min(a + (k + 1) * te, a + d);
        tiles[t + k] = make_int4((int32_t)r, c > 1 ? -1 : (int32_t)r, e0, e1);
        tile_row[t + k] = (int32_t)r;
      }
      if (c > 1) splits[soff[r]] = make_int4((int32_t)r, t, c, 0);
    } else {
      tiles[t] = make_int4((int32_t)r, 0, 0, 0);  // r1 filled by k_tile_close
      tile_row[t] = (int32_t)r;
    }
  }
}

// short tile t ends where tile t+1 begins (or at n); its arc range is
// [ptr[r0], ptr[r1])
__global__ void k_tile_close(int4 *tiles, const int32_t *__restrict__ tile_row, const int32_t *__restrict__ ptr,
                             int32_t nt, int64_t n) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += (int64_t)gridDim.x * blockDim.x) {
    int4 x = tiles[t];
    if (x.y == 0 && x.z == 0 && x.w == 0) {
      x.y = (t + 1 < nt) ? tile_row[t + 1] : (int32_t)n;
      x.z = ptr[x.x];
      x.w = ptr[x.y];
      tiles[t] = x;
    }
  }
}

int build_tiles(gi_graph *g, const Csr &c, int32_t tile_edges, TileSet *ts, cudaStream_t s, int64_t nrows) {
  free_tiles(ts, s);
  GI_TRY(ws_get(g, s));
  ts->tile_edges = tile_edges;
  int64_t n = nrows >= 0 ? nrows : g->n;
  if (n == 0) return GI_OK;
  int32_t *cnt = g->ws->tmp_i32, *scnt = g->ws->tmp2_i32;
  int32_t *off = nullptr, *soff = nullptr, *tile_row = nullptr;
  int st = dev_alloc_n(&off, n + 1, s);
  if (st == GI_OK) st = dev_alloc_n(&soff, n + 1, s);
  if (st == GI_OK) {
    k_tile_count<<<grid_for(g, n, 256), 256, 0, s>>>(c.ptr, n, tile_edges, tile_rows_for(tile_edges), cnt, scnt);
    st = launch_status(1);
  }
  if (st == GI_OK) st = scan_exclusive(g, cnt, off, n, s);
  if (st == GI_OK) st = scan_exclusive(g, scnt, soff, n, s);
  int32_t totals[2] = {0, 0};
  if (st == GI_OK &&
      (cudaMemcpyAsync(&totals[0], off + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
       cudaMemcpyAsync(&totals[1], soff + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
       cudaStreamSynchronize(s) != cudaSuccess))
    st = cuda_fail(cudaGetLastError(), "tile counts", __FILE__, __LINE__);
  ts->num_tiles = totals[0];
  ts->num_splits = totals[1];
  if (st == GI_OK) st = dev_alloc_n(&ts->tiles, ts->num_tiles, s);
  if (st == GI_OK) st = dev_alloc_n(&ts->splits, ts->num_splits, s);
  if (st == GI_OK) st = dev_alloc(&ts->partial, 16 * (size_t)(ts->num_tiles > 0 ? ts->num_tiles : 1), s);
  if (st == GI_OK) st = dev_alloc_n(&tile_row, ts->num_tiles, s);
  if (st == GI_OK) {
    k_tile_write<<<grid_for(g, n, 256), 256, 0, s>>>(c.ptr, n, tile_edges, off, soff, ts->tiles, ts->splits,
                                                     tile_row);
    st = launch_status(1);
  }
  if (st == GI_OK && ts->num_tiles > 0) {
    k_tile_close<<<grid_for(g, ts->num_tiles, 256), 256, 0, s>>>(ts->tiles, tile_row, c.ptr, ts->num_tiles, n);
    st = launch_status(1);
  }
  dev_free(off, s);
  dev_free(soff, s);
  dev_free(tile_row, s);
  if (st != GI_OK) free_tiles(ts, s);  // leaves ts empty (tile_edges 0: rebuilt on next use)
  return st;
}

int use_tiles(gi_graph *g, int32_t tile_edges, cudaStream_t s) {
  int k = 0;
  while (k < 6 && (256 << k) != tile_edges) ++k;
  if (k == 6) {
    set_error("unsupported tile size %d", tile_edges);
    return GI_ERR_UNSUPPORTED;
  }
  if (g->tile_cache[k].tile_edges != tile_edges) GI_TRY(build_tiles(g, g->in, tile_edges, &g->tile_cache[k], s));
  g->in_tiles = g->tile_cache[k];
  return GI_OK;
}

void free_tile_cache(gi_graph *g, cudaStream_t s) {
  for (auto &t : g->tile_cache) free_tiles(&t, s);
  g->in_tiles = TileSet();
  hot_free(g, s);  // derived from the in-edges as well
}

void free_tiles(TileSet *ts, cudaStream_t s) {
  dev_free(ts->tiles, s);
  dev_free(ts->splits, s);
  dev_free(ts->partial, s);
  *ts = TileSet();
}

// =========================================================== hot sources ==
// Selection of the hot sources for the on-chip cache of the dense pull: a
// histogram of out-degrees (65,536 bins, the last one open-ended) gives the
// smallest degree threshold whose count of sources does not exceed kHotMax.
// Since m < 2^31, fewer than 32,768 vertices have degree >= 65,535, so the
// threshold always exists.  Slots follow descending degree (bin by bin from
// the top; the order inside a bin is immaterial), so the most-gathered values
// share the first cache lines.
constexpr int kHotBins = 65536, kHotSmemBins = 4096;

__global__ void k_hot_hist(const int32_t *__restrict__ deg, int64_t n, int32_t *hist) {
  __shared__ int32_t sh[kHotSmemBins];
  for (int i = threadIdx.x; i < kHotSmemBins; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t d = min(deg[v], kHotBins - 1);
    if (d < kHotSmemBins) atomicAdd(sh + d, 1);
    else atomicAdd(hist + d, 1);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kHotSmemBins; i += blockDim.x)
    if (sh[i]) atomicAdd(hist + i, sh[i]);
}

// One block of 1024 threads; thread t owns bins [64t, 64t+64).  start[d] =
// number of vertices in bins above d; out = {threshold, count}.
__global__ void __launch_bounds__(1024) k_hot_pick(const int32_t *__restrict__ hist, int32_t cap, int32_t *start,
                                                   int32_t *out) {
  constexpr int kPer = kHotBins / 1024;
  __shared__ int64_t s_warp[32];
  __shared__ int32_t s_best;
  const int t = threadIdx.x;
  int64_t own = 0;
  for (int i = 0; i < kPer; ++i) own += hist[t * kPer + i];
  // suffix sum over threads t' >= t: an inclusive scan in reversed thread order
  const int r = 1023 - t, rl = r & 31, rw = r >> 5;
  int64_t x = own;
  // lanes of one warp hold consecutive r (reversed), so shuffle down in t
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_down_sync(0xffffffffu, x, o);
    if (rl >= o) x += y;
  }
  if (rl == 31) s_warp[rw] = x;  // warp total (its lowest t, lane 0)
  if (t == 0) s_best = kHotBins;
  __syncthreads();
  int64_t before = 0;  // totals of the warps with larger t
  for (int w = 0; w < rw; ++w) before += s_warp[w];
  const int64_t after = before + x - own;  // vertices in bins above this thread's range
  int64_t run = after;
  for (int d = t * kPer + kPer - 1; d >= t * kPer; --d) {
    start[d] = (int32_t)(run < INT32_MAX ? run : INT32_MAX);
    run += hist[d];
  }
  run = after;
  int32_t cand = kHotBins;
  for (int d = t * kPer + kPer - 1; d >= t * kPer && d >= 1; --d) {
    run += hist[d];
    if (run <= cap) cand = d;
    else break;
  }
  if (cand < kHotBins) atomicMin(&s_best, cand);
  __syncthreads();
  if (cand == s_best && cand < kHotBins) {
    int64_t cnt = after;
    for (int d = t * kPer + kPer - 1; d >= cand; --d) cnt += hist[d];
    out[0] = cand;
    out[1] = (int32_t)cnt;
  }
  if (t == 0 && s_best == kHotBins) {
    out[0] = kHotBins;
    out[1] = 0;
  }
}

// code[v] = ~slot for hot vertices (slot = bin start + arrival order in the
// bin; src[slot] = v), v for the others
__global__ void k_hot_slots(const int32_t *__restrict__ deg, int64_t n, int32_t min_deg,
                            const int32_t *__restrict__ start, int32_t *fill, int32_t *code, int32_t *src) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t d = deg[v];
    int32_t c = (int32_t)v;
    if (d >= min_deg) {
      const int32_t b = min(d, kHotBins - 1);
      const int32_t s = start[b] + atomicAdd(fill + b, 1);
      src[s] = (int32_t)v;
      c = ~s;
    }
    code[v] = c;
  }
}

// the in-edge sources with hot ones replaced by ~slot: one gather per arc
__global__ void k_hot_remap(const int32_t *__restrict__ idx, int64_t m, const int32_t *__restrict__ code,
                            int32_t *hidx) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
    hidx[e] = __ldg(code + idx[e]);
}

// Threshold, slots and code[] (in the workspace) of the hot set; h.src,
// h.vals and h.idx are allocated, h.idx not yet written (hot_remap).
static int hot_select(gi_graph *g, HotSet &h, cudaStream_t s) {
  const int64_t n = g->n, m = g->m;
  if (n == 0 || m == 0 || !g->has_csc) return GI_OK;
  // hist[kHotBins] | start[kHotBins] | fill[kHotBins] | {threshold, count}
  int32_t *hist = nullptr;
  int st = dev_alloc_n(&hist, 3 * kHotBins + 2, s);
  int32_t *start = hist + kHotBins, *fill = hist + 2 * kHotBins, *pick_out = hist + 3 * kHotBins;
  if (st == GI_OK && cudaMemsetAsync(hist, 0, sizeof(int32_t) * (3 * kHotBins + 2), s) != cudaSuccess)
    st = cuda_fail(cudaGetLastError(), "hot histogram", __FILE__, __LINE__);
  if (st == GI_OK) {
    k_hot_hist<<<grid_for(g, n, 256, 2), 256, 0, s>>>(g->out_deg, n, hist);
    k_hot_pick<<<1, 1024, 0, s>>>(hist, kHotMax, start, pick_out);
    st = launch_status(2);
  }
  int32_t pick[2] = {kHotBins, 0};
  if (st == GI_OK && (cudaMemcpyAsync(pick, pick_out, sizeof(pick), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                      cudaStreamSynchronize(s) != cudaSuccess))
    st = cuda_fail(cudaGetLastError(), "hot threshold", __FILE__, __LINE__);
  h.min_deg = pick[0];
  h.k = pick[1];
  if (st == GI_OK && h.k > 0) {
    const int k4 = (h.k + 3) & ~3;
    st = dev_alloc_n(&h.src, h.k, s);
    if (st == GI_OK) st = dev_alloc_n(&h.vals, k4, s);
    if (st == GI_OK) st = dev_alloc_n(&h.idx, m, s);
    if (st == GI_OK && cudaMemsetAsync(h.vals, 0, sizeof(float) * k4, s) != cudaSuccess)
      st = cuda_fail(cudaGetLastError(), "hot values", __FILE__, __LINE__);
    if (st == GI_OK) {
      k_hot_slots<<<grid_for(g, n, 256), 256, 0, s>>>(g->out_deg, n, h.min_deg, start, fill, g->ws->tmp_i32, h.src);
      st = launch_status(1);
    }
  }
  dev_free(hist, s);
  return st;
}

// h.idx[e0, e1) from the in-edge sources (needs hot_select's code[] intact)
static int hot_remap(gi_graph *g, const HotSet &h, int64_t e0, int64_t e1, cudaStream_t s) {
  if (h.k == 0 || e1 <= e0) return GI_OK;
  k_hot_remap<<<grid_for(g, e1 - e0, 256), 256, 0, s>>>(g->in.idx + e0, e1 - e0, g->ws->tmp_i32, h.idx + e0);
  return launch_status(1);
}

static void hot_discard(HotSet &h, cudaStream_t s) {
  dev_free(h.src, s);
  dev_free(h.vals, s);
  dev_free(h.idx, s);
  h = HotSet();
}

static void hot_commit(gi_graph *g, HotSet &h) {
  h.built = true;
  if (h.k == 0) h.min_deg = 0;
  g->hot = h;
}

int hot_get(gi_graph *g, cudaStream_t s) {
  if (g->hot.built) return GI_OK;
  GI_TRY(ws_get(g, s));
  HotSet h;
  int st = hot_select(g, h, s);
  if (st == GI_OK) st = hot_remap(g, h, 0, g->m, s);
  if (st != GI_OK) {
    hot_discard(h, s);
    return st;
  }
  hot_commit(g, h);
  return GI_OK;
}

// Hot set built during a load: select on the caller's stream while the
// indices are still arriving, then remap each piece once it has landed.
static int hot_build_overlapped(gi_graph *g, SideCopy &sc, cudaStream_t s) {
  GI_TRY(ws_get(g, s));
  HotSet h;
  int st = hot_select(g, h, s);
  for (int i = 0; st == GI_OK && i < sc.chunks; ++i) {
    st = sc.wait(i + 1, s);
    if (st == GI_OK) st = hot_remap(g, h, sc.cut[i], sc.cut[i + 1], s);
  }
  if (st != GI_OK) {
    hot_discard(h, s);
    return st;
  }
  hot_commit(g, h);
  return GI_OK;
}

}  // namespace gi

extern "C" int gi_graph_hot_info(gi_graph *g, int32_t *k, int32_t *min_deg, void *stream) {
  GI_ARG(g != nullptr, "graph is NULL");
  if (!g->has_csc) {
    gi::set_error("the hot-source set needs the in-edges: load a symmetric graph or call gi_load_csc");
    return GI_ERR_UNSUPPORTED;
  }
  cudaStream_t s = (cudaStream_t)stream;
  GI_TRY(gi::hot_get(g, s));
  GI_CUDA(cudaStreamSynchronize(s));
  if (k) *k = g->hot.k;
  if (min_deg) *min_deg = g->hot.min_deg;
  return GI_OK;
}

namespace gi {

void hot_free(gi_graph *g, cudaStream_t s) {
  dev_free(g->hot.src, s);
  dev_free(g->hot.idx, s);
  dev_free(g->hot.vals, s);
  g->hot = HotSet();
}

// ============================================================== segments ==
// Segment s keeps in-arcs whose source lies in [lo, hi) = [bounds[s],
// bounds[s+1]), rows kept in destination order and sources ascending (a stable
// filter of the CSC).  Fixed vertex count (FVC): equal source ranges;
// edge-aware vertex count (EVC): ranges holding about m/S arcs each, found in
// the prefix sum of the sources' out-degrees (the CSR offsets).
__global__ void k_seg_count(const int32_t *__restrict__ ptr, const int32_t *__restrict__ idx, int64_t n,
                            int32_t lo, int32_t hi, int32_t *cnt) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    int32_t c = 0;
    for (int32_t e = ptr[r]; e < ptr[r + 1]; ++e) {
      int32_t u = idx[e];
      c += (u >= lo && u < hi);
    }
    cnt[r] = c;
  }
}

__global__ void k_seg_fill(const int32_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                           const int32_t *__restrict__ wt, int64_t n, int32_t lo, int32_t hi,
                           const int32_t *__restrict__ sptr, int32_t *sidx, int32_t *swt) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    int32_t o = sptr[r];
    for (int32_t e = ptr[r]; e < ptr[r + 1]; ++e) {
      int32_t u = idx[e];
      if (u >= lo && u < hi) {
        sidx[o] = u;
        if (swt) swt[o] = wt[e];
        ++o;
      }
    }
  }
}

// EVC bounds: bounds[s] = smallest v with optr[v] >= s*m/S (bounds[0] = 0, bounds[S] = n)
__global__ void k_seg_bounds_evc(const int32_t *__restrict__ optr, int64_t n, int64_t m, int32_t S,
                                 int32_t *bounds) {
  const int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s > S) return;
  if (s == 0 || s == S) {
    bounds[s] = s == 0 ? 0 : (int32_t)n;
    return;
  }
  const int64_t target = m * (int64_t)s / S;
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((int64_t)optr[mid] >= target) hi = mid;
    else lo = mid + 1;
  }
  bounds[s] = (int32_t)lo;
}

static void segs_free(gi_graph *g, cudaStream_t s) {
  if (g->segs.seg) {
    for (int i = 0; i < g->segs.num; ++i) {
      dev_free(g->segs.seg[i].ptr, s);
      dev_free(g->segs.seg[i].idx, s);
      dev_free(g->segs.seg[i].wt, s);
      free_tiles(&g->segs.tiles[i], s);
    }
  }
  delete[] g->segs.seg;
  delete[] g->segs.tiles;
  delete[] g->segs.bounds;
  delete[] g->segs.arcs;
  g->segs = Segments();
}

}  // namespace gi

extern "C" int gi_graph_build_segments(gi_graph *g, int32_t num_segments, int32_t strategy, void *stream) {
  GI_ARG(g != nullptr, "graph is NULL");
  GI_ARG(num_segments >= 1 && num_segments <= 1024, "num_segments must be in [1, 1024]");
  GI_ARG(strategy == GI_SEG_FVC || strategy == GI_SEG_EVC, "strategy must be GI_SEG_FVC or GI_SEG_EVC");
  if (!g->has_csc) {
    set_error("segmented pull needs the in-edges: load a symmetric graph or call gi_load_csc");
    return GI_ERR_UNSUPPORTED;
  }
  cudaStream_t s = (cudaStream_t)stream;
  segs_free(g, s);
  if (num_segments == 1) return GI_OK;
  GI_TRY(ws_get(g, s));
  const int64_t n = g->n;
  const int S = num_segments;
  Segments sg;
  sg.num = S;
  sg.strategy = strategy;
  sg.bounds = new int32_t[S + 1];
  sg.arcs = new int64_t[S];
  sg.seg = new Csr[S];
  sg.tiles = new TileSet[S];
  int st = GI_OK;
  if (strategy == GI_SEG_FVC) {
    const int64_t seg_size = (n + S - 1) / S;
    for (int k = 0; k <= S; ++k) sg.bounds[k] = (int32_t)(k * seg_size < n ? k * seg_size : n);
  } else {
    int32_t *db = nullptr;
    st = dev_alloc_n(&db, S + 1, s);
    if (st == GI_OK) {
      k_seg_bounds_evc<<<div_up(S + 1, 256), 256, 0, s>>>(g->out.ptr, n, g->m, S, db);
      st = launch_status(1);
    }
    if (st == GI_OK && (cudaMemcpyAsync(sg.bounds, db, sizeof(int32_t) * (S + 1), cudaMemcpyDeviceToHost, s) !=
                            cudaSuccess ||
                        cudaStreamSynchronize(s) != cudaSuccess))
      st = cuda_fail(cudaGetLastError(), "segment bounds", __FILE__, __LINE__);
    dev_free(db, s);
  }
  for (int sid = 0; sid < S && st == GI_OK; ++sid) {
    Csr &c = sg.seg[sid];
    const int32_t lo = sg.bounds[sid], hi = sg.bounds[sid + 1];
    st = dev_alloc_n(&c.ptr, n + 1, s);
    if (st == GI_OK) {
      k_seg_count<<<grid_for(g, n, 256), 256, 0, s>>>(g->in.ptr, g->in.idx, n, lo, hi, g->ws->tmp_i32);
      st = launch_status(1);
    }
    if (st == GI_OK) st = scan_exclusive(g, g->ws->tmp_i32, c.ptr, n, s);
    int32_t cnt = 0;
    if (st == GI_OK && (cudaMemcpyAsync(&cnt, c.ptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                        cudaStreamSynchronize(s) != cudaSuccess))
      st = cuda_fail(cudaGetLastError(), "segment size", __FILE__, __LINE__);
    sg.arcs[sid] = cnt;
    if (st == GI_OK) st = dev_alloc_n(&c.idx, cnt, s);
    if (st == GI_OK && g->in.wt) st = dev_alloc_n(&c.wt, cnt, s);
    if (st == GI_OK) {
      k_seg_fill<<<grid_for(g, n, 256), 256, 0, s>>>(g->in.ptr, g->in.idx, g->in.wt, n, lo, hi, c.ptr, c.idx, c.wt);
      st = launch_status(1);
    }
    if (st == GI_OK)
      st = build_tiles(g, c, g->in_tiles.tile_edges > 0 ? g->in_tiles.tile_edges : 2048, &sg.tiles[sid], s);
  }
  g->segs = sg;  // owned by the graph from here; freed whole on failure
  if (st != GI_OK) {
    segs_free(g, s);
    return st;
  }
  GI_CUDA(cudaStreamSynchronize(s));
  return GI_OK;
}

extern "C" int gi_graph_segment_info(const gi_graph *g, int32_t *num, int32_t *strategy, int32_t *bounds,
                                     int64_t *arcs, int32_t cap) {
  GI_ARG(g != nullptr, "graph is NULL");
  const int S = g->segs.seg ? g->segs.num : 1;
  if (num) *num = S;
  if (strategy) *strategy = g->segs.strategy;
  if (g->segs.seg) {
    for (int k = 0; k <= S && bounds && k < cap + 1; ++k) bounds[k] = g->segs.bounds[k];
    for (int k = 0; k < S && arcs && k < cap; ++k) arcs[k] = g->segs.arcs[k];
  } else {
    if (bounds && cap >= 1) {
      bounds[0] = 0;
      bounds[1] = (int32_t)g->n;
    }
    if (arcs && cap >= 1) arcs[0] = g->m;
  }
  return GI_OK;
}

namespace gi {

// ============================================================ vertexsets ==
__global__ void k_bitmap_from_queue(const int32_t *__restrict__ q, const int32_t *__restrict__ count, uint32_t *bm) {
  int32_t c = *count;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < c; i += gridDim.x * blockDim.x) {
    int32_t v = q[i];
    atomicOr(bm + (v >> 5), 1u << (v & 31));
  }
}

__global__ void k_bitmap_from_bool(const uint8_t *__restrict__ b, int64_t n, uint32_t *bm) {
  // one warp writes one word: lane i tests vertex 32*w + i
  int64_t nw = (n + 31) / 32;
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nw;
       w += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    int64_t v = w * 32 + lane_id();
    unsigned word = __ballot_sync(0xffffffffu, v < n && b[v]);
    if (lane_id() == 0) bm[w] = word;
  }
}

__global__ void k_bool_from_bitmap(const uint32_t *__restrict__ bm, int64_t n, uint8_t *b) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    b[v] = (bm[v >> 5] >> (v & 31)) & 1u;
}

__global__ void k_word_popc(const uint32_t *__restrict__ bm, int64_t nw, int32_t *cnt) {
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += (int64_t)gridDim.x * blockDim.x)
    cnt[w] = __popc(bm[w]);
}

// ordered compaction: word w writes its set bits at off[w]...
__global__ void k_compact_bitmap(const uint32_t *__restrict__ bm, int64_t nw, const int32_t *__restrict__ off,
                                 int32_t *q, int32_t *count) {
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += (int64_t)gridDim.x * blockDim.x) {
    uint32_t x = bm[w];
    int32_t o = off[w];
    while (x) {
      int b = __ffs(x) - 1;
      q[o++] = (int32_t)(w * 32 + b);
      x &= x - 1;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *count = off[nw];
}

__global__ void k_vset_init(int32_t *q, int32_t *count, uint32_t *bm, int64_t words, int64_t n, int32_t init,
                            int32_t v) {
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += (int64_t)gridDim.x * blockDim.x) {
    uint32_t word = 0;
    if (init == GI_VSET_ALL) {
      int64_t lo = w * 32, rem = n - lo;
      word = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
    } else if (init == GI_VSET_SINGLE && (v >> 5) == w) {
      word = 1u << (v & 31);
    }
    bm[w] = word;
  }
  if (init == GI_VSET_ALL) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
      q[i] = (int32_t)i;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (init == GI_VSET_SINGLE) q[0] = v;
    *count = init == GI_VSET_ALL ? (int32_t)n : (init == GI_VSET_SINGLE ? 1 : 0);
  }
}

int vset_alloc(gi_graph *g, gi_vset *v, cudaStream_t s) {
  v->g = g;
  v->n = g->n;
  v->words = (g->n + 31) / 32;
  GI_TRY(dev_alloc_n(&v->queue, g->n, s));
  GI_TRY(dev_alloc_n(&v->count, 1, s));
  GI_TRY(dev_alloc_n(&v->bitmap, v->words, s));
  return GI_OK;
}

int vset_clear(gi_vset *v, cudaStream_t s) {
  GI_CUDA(cudaMemsetAsync(v->bitmap, 0, sizeof(uint32_t) * (size_t)(v->words > 0 ? v->words : 1), s));
  GI_CUDA(cudaMemsetAsync(v->count, 0, sizeof(int32_t), s));
  if (v->boolmap) GI_CUDA(cudaMemsetAsync(v->boolmap, 0, (size_t)(v->n > 0 ? v->n : 1), s));
  v->reps = GI_REP_SPARSE | GI_REP_BITMAP | (v->boolmap ? GI_REP_BOOL : 0);
  return GI_OK;
}

int vset_ensure_bitmap(gi_vset *v, cudaStream_t s) {
  if (v->reps & GI_REP_BITMAP) return GI_OK;
  gi_graph *g = v->g;
  if (v->reps & GI_REP_BOOL) {
    k_bitmap_from_bool<<<grid_for(g, v->words * 32, 256), 256, 0, s>>>(v->boolmap, v->n, v->bitmap);
  } else {
    GI_CUDA(cudaMemsetAsync(v->bitmap, 0, sizeof(uint32_t) * (size_t)(v->words > 0 ? v->words : 1), s));
    k_bitmap_from_queue<<<grid_for(g, v->n, 256), 256, 0, s>>>(v->queue, v->count, v->bitmap);
  }
  GI_LAUNCH_CHECK();
  v->reps |= GI_REP_BITMAP;
  return GI_OK;
}

int vset_ensure_bool(gi_vset *v, cudaStream_t s) {
  if (v->reps & GI_REP_BOOL) return GI_OK;
  if (!v->boolmap) GI_TRY(dev_alloc_n(&v->boolmap, v->n, s));
  GI_TRY(vset_ensure_bitmap(v, s));
  k_bool_from_bitmap<<<grid_for(v->g, v->n, 256), 256, 0, s>>>(v->bitmap, v->n, v->boolmap);
  GI_LAUNCH_CHECK();
  v->reps |= GI_REP_BOOL;
  return GI_OK;
}

// sparse from bitmap: ascending ids (ordered compaction by word popcount scan)
int vset_ensure_queue(gi_vset *v, cudaStream_t s) {
  if (v->reps & GI_REP_SPARSE) return GI_OK;
  GI_TRY(vset_ensure_bitmap(v, s));
  gi_graph *g = v->g;
  GI_TRY(ws_get(g, s));
  k_word_popc<<<grid_for(g, v->words, 256), 256, 0, s>>>(v->bitmap, v->words, g->ws->tmp_i32);
  GI_LAUNCH_CHECK();
  GI_TRY(scan_exclusive(g, g->ws->tmp_i32, g->ws->tmp2_i32, v->words, s));
  k_compact_bitmap<<<grid_for(g, v->words, 256), 256, 0, s>>>(v->bitmap, v->words, g->ws->tmp2_i32, v->queue,
                                                              v->count);
  GI_LAUNCH_CHECK();
  v->reps |= GI_REP_SPARSE;
  return GI_OK;
}

}  // namespace gi

extern "C" int gi_vset_create(gi_graph *g, int32_t init, int32_t v, void *stream, gi_vset **out) {
  GI_ARG(g != nullptr && out != nullptr, "NULL graph or output");
  GI_ARG(init == GI_VSET_EMPTY || init == GI_VSET_ALL || init == GI_VSET_SINGLE, "unknown init");
  GI_ARG(init != GI_VSET_SINGLE || (v >= 0 && v < g->n), "vertex out of range");
  cudaStream_t s = (cudaStream_t)stream;
  gi_vset *x = new gi_vset();
  int st = vset_alloc(g, x, s);
  if (st == GI_OK) {
    k_vset_init<<<grid_for(g, g->n > x->words ? g->n : x->words, 256), 256, 0, s>>>(x->queue, x->count, x->bitmap,
                                                                                   x->words, g->n, init, v);
    st = launch_status(1);
  }
  if (st != GI_OK) {
    gi_vset_free(x);
    return st;
  }
  x->reps = GI_REP_SPARSE | GI_REP_BITMAP;
  *out = x;
  return GI_OK;
}

extern "C" int gi_vset_free(gi_vset *x) {
  if (!x) return GI_OK;
  cudaStream_t s = 0;
  cudaDeviceSynchronize();
  dev_free(x->queue, s);
  dev_free(x->count, s);
  dev_free(x->bitmap, s);
  dev_free(x->boolmap, s);
  delete x;
  GI_CUDA(cudaStreamSynchronize(s));
  return GI_OK;
}

extern "C" int gi_vset_reps(const gi_vset *x, uint32_t *reps) {
  GI_ARG(x != nullptr && reps != nullptr, "NULL argument");
  *reps = x->reps;
  return GI_OK;
}

extern "C" int gi_vset_size(gi_vset *x, int64_t *out, void *stream) {
  GI_ARG(x != nullptr && out != nullptr, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  GI_TRY(vset_ensure_queue(x, s));
  int32_t c = 0;
  GI_CUDA(cudaMemcpyAsync(&c, x->count, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  GI_CUDA(cudaStreamSynchronize(s));
  *out = c;
  return GI_OK;
}

extern "C" int gi_vset_to_sparse(gi_vset *x, void *stream) {
  GI_ARG(x != nullptr, "NULL vertexset");
  return vset_ensure_queue(x, (cudaStream_t)stream);
}

extern "C" int gi_vset_to_dense(gi_vset *x, uint32_t rep, void *stream) {
  GI_ARG(x != nullptr, "NULL vertexset");
  GI_ARG(rep == GI_REP_BOOL || rep == GI_REP_BITMAP, "rep must be GI_REP_BOOL or GI_REP_BITMAP");
  cudaStream_t s = (cudaStream_t)stream;
  return rep == GI_REP_BOOL ? vset_ensure_bool(x, s) : vset_ensure_bitmap(x, s);
}

extern "C" int gi_vset_export(gi_vset *x, int32_t *dev_out, int64_t cap, int64_t *count, void *stream) {
  GI_ARG(x != nullptr && count != nullptr, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  // ascending order: go through the bitmap
  GI_TRY(vset_ensure_bitmap(x, s));
  x->reps = GI_REP_BITMAP | (x->reps & GI_REP_BOOL);
  GI_TRY(vset_ensure_queue(x, s));
  int32_t c = 0;
  GI_CUDA(cudaMemcpyAsync(&c, x->count, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  GI_CUDA(cudaStreamSynchronize(s));
  *count = c;
  if (c > cap) {
    set_error("vertexset has %d members, output holds %lld", c, (long long)cap);
    return GI_ERR_INVALID_ARG;
  }
  GI_ARG(c == 0 || dev_out != nullptr, "dev_out is NULL");
  if (c > 0) GI_CUDA(cudaMemcpyAsync(dev_out, x->queue, sizeof(int32_t) * (size_t)c, cudaMemcpyDeviceToDevice, s));
  GI_CUDA(cudaStreamSynchronize(s));
  return GI_OK;
}

namespace gi {
__global__ void k_import(const int32_t *__restrict__ ids, int64_t k, int64_t n, uint32_t *bm, int64_t *err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t v = ids[i];
    if (v < 0 || v >= n) {
      atomicCAS(reinterpret_cast<unsigned long long *>(err), 0ull, (unsigned long long)(i + 1));
      continue;
    }
    atomicOr(bm + (v >> 5), 1u << (v & 31));
  }
}
}  // namespace gi

extern "C" int gi_vset_import(gi_vset *x, const int32_t *dev_ids, int64_t k, void *stream) {
  GI_ARG(x != nullptr, "NULL vertexset");
  GI_ARG(k >= 0 && (k == 0 || dev_ids != nullptr), "bad id array");
  cudaStream_t s = (cudaStream_t)stream;
  gi_graph *g = x->g;
  GI_CUDA(cudaMemsetAsync(x->bitmap, 0, sizeof(uint32_t) * (size_t)(x->words > 0 ? x->words : 1), s));
  GI_CUDA(cudaMemsetAsync(g->ctrl + kErr, 0, sizeof(int64_t), s));
  if (k > 0) {
    k_import<<<grid_for(g, k, 256), 256, 0, s>>>(dev_ids, k, x->n, x->bitmap, g->ctrl + kErr);
    GI_LAUNCH_CHECK();
  }
  int64_t err = 0;
  GI_CUDA(cudaMemcpyAsync(&err, g->ctrl + kErr, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GI_CUDA(cudaStreamSynchronize(s));
  if (err) {
    set_error("vertex id at position %lld is out of range", (long long)(err - 1));
    return GI_ERR_INVALID_ARG;
  }
  x->reps = GI_REP_BITMAP;
  return vset_ensure_queue(x, s);
}

// ========================================================= selector MLP ==
namespace gi {

constexpr int kDIn = 16, kH = 64, kDOut = 3;
constexpr int kNParam = kH * kDIn + kH + kH * kH + kH + kDOut * kH + kDOut;

__device__ __align__(16) float d_sel_params[kNParam];  // 16-byte aligned rows: W2 and W3 start at multiples of 4
__device__ float d_sel_mean[kDIn];
__device__ float d_sel_istd[kDIn];
static bool g_sel_loaded = false;

bool selector_loaded() { return g_sel_loaded; }

// The learned selector is consulted only where the two directions can cost
// alike: a frontier with |F| + m_f below m / kSelGate is pushed without an
// evaluation (a pull walks every row or tile, a push of so few arcs costs a
// small fraction of that), which also keeps the network's latency off the
// many small levels and rounds.
constexpr int64_t kSelGate = 200;
__device__ __forceinline__ bool selector_gated(int64_t nf, int64_t mf, int64_t m) { return (nf + mf) * kSelGate < m; }

// MLP forward by one block (>= 64 threads); returns argmin of predicted log-time
__device__ int32_t selector_forward(const float *x_raw, float *sh /* >= 16+64+64+3 floats */) {
  // Called by all 256 threads of one block.  Layers 1 and 2: four threads
  // per hidden unit, each a quarter of the dot product with 16-byte weight
  // loads, summed by shuffles; layer 3: one warp per output.  Every load is
  // independent, so a decision costs a few memory round trips rather than a
  // chain of 64 dependent ones per thread.
  float *x = sh, *h1 = sh + kDIn, *h2 = h1 + kH, *y = h2 + kH;
  const float *W1 = d_sel_params, *b1 = W1 + kH * kDIn, *W2 = b1 + kH, *b2 = W2 + kH * kH, *W3 = b2 + kH,
              *b3 = W3 + kDOut * kH;
  const int t = threadIdx.x, lane = t & 31;
  if (t < kDIn) x[t] = (x_raw[t] - d_sel_mean[t]) * d_sel_istd[t];
  __syncthreads();
  const int unit = t >> 2, part = t & 3;  // 64 units x 4 parts = 256 threads
  if (unit < kH) {
    const float4 w = *reinterpret_cast<const float4 *>(W1 + unit * kDIn + part * 4);
    float s = w.x * x[part * 4] + w.y * x[part * 4 + 1] + w.z * x[part * 4 + 2] + w.w * x[part * 4 + 3];
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    if (part == 0) h1[unit] = fmaxf(s + b1[unit], 0.0f);
  }
  __syncthreads();
  if (unit < kH) {
    const float4 *w4 = reinterpret_cast<const float4 *>(W2 + unit * kH + part * 16);
    const float *hp = h1 + part * 16;
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float4 w = w4[j];
      s += w.x * hp[4 * j] + w.y * hp[4 * j + 1] + w.z * hp[4 * j + 2] + w.w * hp[4 * j + 3];
    }
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    if (part == 0) h2[unit] = fmaxf(s + b2[unit], 0.0f);
  }
  __syncthreads();
  const int out = t >> 5;
  if (out < kDOut) {
    const float2 w = *reinterpret_cast<const float2 *>(W3 + out * kH + lane * 2);
    float s = w.x * h2[lane * 2] + w.y * h2[lane * 2 + 1];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[out] = s + b3[out];
  }
  __syncthreads();
  int32_t best = 0;
  for (int j = 1; j < kDOut; ++j)
    if (y[j] < y[best]) best = j;
  return best;  // 0 SparsePush, 1 DensePush, 2 DensePull
}

// ================================================ frontier statistics ==
// One pass over F's queue sums out-degrees; the last block to finish
// (ticket) computes the features and the direction for this iteration.
__global__ void k_frontier_decide(const int32_t *__restrict__ q, const int32_t *__restrict__ count,
                                  const int32_t *__restrict__ deg, int64_t *ctrl, DecideParams p, int64_t n,
                                  int64_t m, int32_t maxdeg, int use_selector) {
  __shared__ unsigned long long s_sum[32];
  __shared__ float sh[kDIn + kH + kH + 4];
  __shared__ float feat[kDIn];
  __shared__ bool last;
  int32_t c = *count;
  unsigned long long local = 0;
  // 8 independent queue loads, then 8 independent degree gathers, per round trip
  const int32_t stride = gridDim.x * blockDim.x;
  if (p.clear_bm) {  // graph-driven: empty the set this level fills
    const int32_t cc = *p.clear_qc;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cc; i += stride) p.clear_bm[p.clear_q[i] >> 5] = 0u;
  }
  for (int32_t i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < c; i0 += 8 * stride) {
    int32_t v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = i0 + j * stride < c ? q[i0 + j * stride] : -1;
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (v[j] >= 0) local += deg[v[j]];
  }
  for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
  if (lane_id() == 0) s_sum[threadIdx.x >> 5] = local;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += s_sum[w];
    atomicAdd(reinterpret_cast<unsigned long long *>(ctrl + kMfAcc), b);
    __threadfence();
    unsigned long long t = atomicAdd(reinterpret_cast<unsigned long long *>(ctrl + kTicket), 1ull);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  int64_t nf = c;
  int64_t mf = *(volatile int64_t *)(ctrl + kMfAcc);
  int64_t nu = ctrl[kNu], mu = ctrl[kMu];
  if (p.track_unvisited) {
    nu -= nf;
    mu -= mf;
  }
  int32_t was_pull = (int32_t)ctrl[kWasPull];
  int64_t nf_prev = ctrl[kNfPrev];
  const int32_t level = p.gm ? *(volatile int32_t *)(p.gm + kGmNext) : p.level;
  if (threadIdx.x == 0) level_features(feat, n, m, maxdeg, nf, mf, nu, mu, level, was_pull, nf_prev);
  __syncthreads();
  int32_t dir;
  if (p.mode == 0) {
    dir = p.forced;
  } else if (p.mode == 2 && use_selector) {
    if (selector_gated(nf, mf, m)) {
      dir = GI_DIR_SPARSE_PUSH;
    } else {
      int32_t k = selector_forward(feat, sh);
      dir = k == 0 ? GI_DIR_SPARSE_PUSH : (k == 1 ? GI_DIR_DENSE_PUSH : GI_DIR_DENSE_PULL);
    }
  } else {
    bool dense;
    if (p.rule == GI_RULE_LIGRA || !p.track_unvisited) {
      dense = (nf + mf) > m / 20;
    } else if (!was_pull) {
      dense = (double)mf > (double)mu / (double)p.alpha;
    } else {
      dense = !((double)nf < (double)n / (double)p.beta);
    }
    int32_t dense_dir = (p.hybrid_kind == GI_DIR_HYBRID_DPUSH) ? GI_DIR_DENSE_PUSH : GI_DIR_DENSE_PULL;
    dir = dense ? dense_dir : GI_DIR_SPARSE_PUSH;
  }
  if (threadIdx.x < kDIn) reinterpret_cast<float *>(ctrl + kFeat)[threadIdx.x] = feat[threadIdx.x];
  if (threadIdx.x == 0) {
    ctrl[kNf] = nf;
    ctrl[kMf] = mf;
    ctrl[kNu] = nu;
    ctrl[kMu] = mu;
    ctrl[kDecision] = dir;
    // the previous-level features describe the last non-empty frontier: a
    // statistics pass over an empty set (delta-stepping's R before a heavy
    // round; the last check of the other loops) leaves them as they were
    if (nf > 0) {
      ctrl[kWasPull] = (dir == GI_DIR_DENSE_PULL) ? 1 : 0;
      ctrl[kNfPrev] = nf;
    }
    ctrl[kLevel] = level;
    ctrl[kTicket] = 0;
    ctrl[kMfAcc] = 0;
    if (p.clear_qc) *p.clear_qc = 0;  // every block has passed its clearing loop
    if (p.gm) {  // graph-driven: both traversals of the level read their part
      const bool go = nf > 0 && level < p.gm[kGmCap];
      if (nf > 0 && !go) p.gm[kGmErr] = 1;
      p.gm[kGmPush] = (go && dir != GI_DIR_DENSE_PULL) ? (int32_t)nf : 0;
      p.gm[kGmPull] = (go && dir == GI_DIR_DENSE_PULL) ? 1 : 0;
      p.gm[kGmLevel] = level;
      if (go) p.gm[kGmNext] = level + 1;
      cudaGraphSetConditional((cudaGraphConditionalHandle)p.cond_handle, go ? 1u : 0u);
    }
  }
}

// One round of graph-driven delta-stepping, set-up and decision (see
// dsg_step_launch): the split of P into R / S / far pile with R's light and
// S's heavy arc counts, then in the last block the features, the direction
// (rule, or the MLP as in k_frontier_decide) and the round's mode.
__global__ void k_dsg_step(DsgBuffers B, int64_t *ctrl, DecideParams p, int64_t n, int64_t m, int32_t maxdeg,
                           int use_selector, int32_t delta, int pull_ok, unsigned long long switch_handle,
                           unsigned long long while_handle) {
  __shared__ unsigned long long s_sum[2][32];
  __shared__ float sh[kDIn + kH + kH + 4];
  __shared__ float feat[kDIn];
  __shared__ bool last;
  int32_t *dw = B.dw;
  const int lane = lane_id();
  // P holds each vertex once, so the membership flags need no atomics
  const int32_t c = *B.Pc, hi = dw[kDgHi], cur = dw[kDgCur], epoch = dw[kDgEpoch];
  int32_t *pile = cur ? B.pile1 : B.pile0;
  int32_t *pile_count = dw + kDgPile0 + cur;
  const int32_t stride = gridDim.x * blockDim.x;
  int32_t fmin = INT32_MAX;
  unsigned long long ml = 0, mh = 0;
  for (int32_t i0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < c; i0 += stride) {
    const int32_t i = i0 + lane;
    int32_t v = -1, d = INT32_MAX, sm = epoch, dl = 0, dh = 0;
    uint8_t pin = 0;
    if (i < c) {
      v = B.P[i];
      // every per-vertex word the split may need, loaded together (one
      // round trip after v instead of a chain of them behind the branches)
      d = B.x[v];
      sm = B.s_mark[v];
      pin = B.pile_in[v];
      dl = B.deg_l[v];
      dh = B.deg_h[v];
      B.Pbm[v >> 5] = 0u;  // the whole word: every bit set in it belongs to P
    }
    const bool near = v >= 0 && d < hi, far = v >= 0 && !near;
    bool snew = false, pnew = false;
    if (near) {
      B.snap[v] = d;
      B.snap_h[v] = d;
      if (pin) B.pile_in[v] = 0;  // its pile entry is now stale
      ml += dl;
      if (sm != epoch) {
        B.s_mark[v] = epoch;
        snew = true;
        mh += dh;
      }
    }
    if (far) {
      fmin = min(fmin, d);
      if (!pin) {
        B.pile_in[v] = 1;
        pnew = true;
      }
    }
    warp_append3(B.Rq, dw + kDgRc, near, B.Sq, dw + kDgSc, snew, pile, pile_count, pnew, v);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    fmin = min(fmin, __shfl_xor_sync(0xffffffffu, fmin, o));
    ml += __shfl_xor_sync(0xffffffffu, ml, o);
    mh += __shfl_xor_sync(0xffffffffu, mh, o);
  }
  if (lane == 0) {
    if (fmin < INT32_MAX) atomicMin(dw + kDgPmin, fmin);
    s_sum[0][threadIdx.x >> 5] = ml;
    s_sum[1][threadIdx.x >> 5] = mh;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long bl = 0, bh = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      bl += s_sum[0][w];
      bh += s_sum[1][w];
    }
    if (bl) atomicAdd(reinterpret_cast<unsigned long long *>(ctrl + kMfAcc), bl);
    if (bh) atomicAdd(reinterpret_cast<unsigned long long *>(ctrl + kSHeavyMf), bh);
    __threadfence();
    const unsigned long long t = atomicAdd(reinterpret_cast<unsigned long long *>(ctrl + kTicket), 1ull);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int32_t rc = *(volatile int32_t *)(dw + kDgRc), sc = *(volatile int32_t *)(dw + kDgSc);
  const bool light = rc > 0, heavy = !light && sc > 0;
  const int64_t nf = light ? rc : (heavy ? sc : 0);
  const int64_t mf = light ? *(volatile int64_t *)(ctrl + kMfAcc)
                           : (heavy ? *(volatile int64_t *)(ctrl + kSHeavyMf) : 0);
  const int32_t was_pull = (int32_t)ctrl[kWasPull];
  const int64_t nf_prev = ctrl[kNfPrev];
  const int32_t round = dw[kDgRound];
  const bool relax = light || heavy;
  if (relax && threadIdx.x == 0) level_features(feat, n, m, maxdeg, nf, mf, 0, 0, round, was_pull, nf_prev);
  __syncthreads();
  int32_t dir = GI_DIR_SPARSE_PUSH;
  if (relax) {
    if (p.mode == 0) {
      dir = p.forced;
    } else if (p.mode == 2 && use_selector) {
      if (!selector_gated(nf, mf, m)) {
        const int32_t k = selector_forward(feat, sh);
        dir = k == 2 ? GI_DIR_DENSE_PULL : GI_DIR_SPARSE_PUSH;
      }
    } else {
      dir = (nf + mf) > m / 20 ? GI_DIR_DENSE_PULL : GI_DIR_SPARSE_PUSH;
    }
    if (dir != GI_DIR_DENSE_PULL || !pull_ok) dir = GI_DIR_SPARSE_PUSH;
  }
  if (threadIdx.x == 0) {
    int32_t mode;
    // every block has read P's count and appended to R: both are spent (the
    // light push reads R's length from kDgPushL)
    *B.Pc = 0;
    dw[kDgRc] = 0;
    if (relax) {
      const bool pull = dir == GI_DIR_DENSE_PULL;
      // sources without arcs of the class relax nothing: the push branch with
      // an empty queue, whatever the direction (no pull over the class's arcs)
      const bool run_pull = pull && mf > 0;
      mode = light ? (run_pull ? kDgLightPull : kDgLightPush) : (run_pull ? kDgHeavyPull : kDgHeavyPush);
      ctrl[kWasPull] = pull ? 1 : 0;
      ctrl[kNfPrev] = nf;
      // a heavy round without heavy arcs only empties S: not a relaxation round
      if (light || mf > 0) dw[kDgRound] = round + 1;
      if (!light) {
        // the heavy round closes the bucket: S starts again (the heavy push
        // reads S's length from kDgPushH, and S's members are settled, so
        // none of them is in a later P)
        dw[kDgSc] = 0;
        dw[kDgEpoch] = epoch + 1;
        ctrl[kSHeavyMf] = 0;
      }
    } else if (dw[kDgPile0 + cur] > 0) {
      // the bucket and its heavy round are done: next bucket from the pile,
      // which the pile split reads from buffer cur and thins into cur ^ 1
      mode = kDgAdvance;
      const int64_t hi2 = ((int64_t)dw[kDgPmin] / delta + 1) * (int64_t)delta;
      dw[kDgHi] = (int32_t)(hi2 < INT32_MAX ? hi2 : INT32_MAX);
      dw[kDgPile0 + (cur ^ 1)] = 0;
      dw[kDgPmin] = INT32_MAX;
      dw[kDgCur] = cur ^ 1;
    } else {
      mode = kDgDone;
    }
    if (mode != kDgDone && round >= dw[kDgCap]) {
      dw[kDgErr] = 1;
      mode = kDgDone;
    }
    dw[kDgMode] = mode;
    dw[kDgPushL] = (mode == kDgLightPush && mf > 0) ? rc : 0;
    dw[kDgPushH] = (mode == kDgHeavyPush && mf > 0) ? sc : 0;
    ctrl[kNf] = nf;
    ctrl[kMf] = mf;
    ctrl[kDecision] = dir;
    ctrl[kTicket] = 0;
    ctrl[kMfAcc] = 0;
    cudaGraphSetConditional((cudaGraphConditionalHandle)switch_handle, (unsigned)mode);
    cudaGraphSetConditional((cudaGraphConditionalHandle)while_handle, mode != kDgDone ? 1u : 0u);
  }
}

int dsg_step_launch(gi_graph *g, const DsgBuffers &b, const DecideParams &p, int32_t delta, bool pull_ok,
                    unsigned long long switch_handle, unsigned long long while_handle, cudaStream_t s) {
  // six blocks per SM: the kernel's registers allow six 256-thread blocks,
  // and its per-vertex chain of dependent loads wants every warp it can get
  k_dsg_step<<<g->num_sms * 6, 256, 0, s>>>(b, g->ctrl, p, g->n, g->m, g->max_deg, g_sel_loaded ? 1 : 0, delta,
                                            pull_ok ? 1 : 0, switch_handle, while_handle);
  GI_LAUNCH_CHECK();
  return GI_OK;
}

__global__ void k_ctrl_init(int64_t *ctrl, int64_t nu, int64_t mu) {
  for (int i = threadIdx.x; i < kCtrlWords; i += blockDim.x)
    if (i != kPullArcs) ctrl[i] = 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    ctrl[kNu] = nu;
    ctrl[kMu] = mu;
  }
}

int ctrl_init(gi_graph *g, int64_t nu, int64_t mu, cudaStream_t s) {
  k_ctrl_init<<<1, 64, 0, s>>>(g->ctrl, nu, mu);
  GI_LAUNCH_CHECK();
  return GI_OK;
}

int frontier_decide(gi_graph *g, gi_vset *F, const DecideParams &p, cudaStream_t s, const int32_t *deg) {
  GI_TRY(vset_ensure_queue(F, s));
  int blocks = g->num_sms * 6;  // as many resident 256-thread blocks as its registers allow
  k_frontier_decide<<<blocks, 256, 0, s>>>(F->queue, F->count, deg ? deg : g->out_deg, g->ctrl, p, g->n, g->m,
                                           g->max_deg, g_sel_loaded ? 1 : 0);
  GI_LAUNCH_CHECK();
  return GI_OK;
}

int ctrl_fetch(gi_graph *g, cudaStream_t s) {
  GI_CUDA(cudaMemcpyAsync(g->ctrl_host, g->ctrl, sizeof(int64_t) * kCtrlWords, cudaMemcpyDeviceToHost, s));
  GI_CUDA(cudaStreamSynchronize(s));
  return GI_OK;
}

}  // namespace gi

extern "C" int gi_selector_num_params(void) { return gi::kNParam; }

extern "C" int gi_selector_load(const float *params, int32_t count, const float *mean, const float *inv_std) {
  GI_ARG(params != nullptr && mean != nullptr && inv_std != nullptr, "NULL argument");
  GI_ARG(count == gi::kNParam, "selector expects 5443 parameters");
  GI_CUDA(cudaMemcpyToSymbol(gi::d_sel_params, params, sizeof(float) * gi::kNParam));
  GI_CUDA(cudaMemcpyToSymbol(gi::d_sel_mean, mean, sizeof(float) * gi::kDIn));
  GI_CUDA(cudaMemcpyToSymbol(gi::d_sel_istd, inv_std, sizeof(float) * gi::kDIn));
  GI_TRY(gi::batch_selector_upload(params, mean, inv_std));
  gi::g_sel_loaded = true;
  return GI_OK;
}

extern "C" void gi_schedule_default(gi_schedule *s) {
  if (!s) return;
  s->direction = GI_DIR_HYBRID_PULL;
  s->dense_rep = GI_REP_BITMAP;
  s->balance = GI_BAL_EDGE_AWARE;
  s->num_segments = 1;
  s->block = 256;
  s->t_warp = 32;
  s->t_cta = 256;
  s->rule = GI_RULE_BEAMER;
  s->alpha = 14.0f;
  s->beta = 24.0f;
  s->tile_edges = 2048;
  s->t_heavy = 256;
  s->persistent = 0;
  s->hot_cache = 0;
  s->seg_strategy = GI_SEG_FVC;
  s->delta = 0;
  s->dst_list = 1;
}
