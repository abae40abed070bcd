// Batched multi-query traversal in one persistent launch (not part of the
// paper; the paper runs one query at a time on a multicore CPU).
//
// The launch is a grid of thread-block clusters.  Each cluster repeatedly
// claims the next query from a global counter and runs it to completion:
// level-synchronous BFS (SparsePush or early-exit DensePull per level, chosen
// by Beamer's rule or the learned selector) or Bellman-Ford SSSP with
// asynchronous min relaxation (push).  The only waits are cluster barriers (barrier.cluster, hardware
// co-scheduled CTAs) taken the same number of times by every CTA of a
// cluster: all loop bounds come from values read after a barrier.  Clusters
// never wait on each other, so a cluster that starts late simply finds the
// work counter exhausted.  A level cap bounds every loop; exceeding it sets
// an error flag that the host reports as GI_ERR_TIMEOUT.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cmath>
#include <algorithm>
#include <vector>

#include "gi_features.cuh"
#include "gi_internal.cuh"
#include "gi_traverse.cuh"

namespace cg = cooperative_groups;

namespace gi {

// this translation unit's copy of the selector weights (see gi_selector_load);
// internal linkage, so it never collides with gi_core.cu's copy
static __device__ float d_bsel_params[64 * 16 + 64 + 64 * 64 + 64 + 3 * 64 + 3];
static __device__ float d_bsel_mean[16];
static __device__ float d_bsel_istd[16];

int batch_selector_upload(const float *params, const float *mean, const float *inv_std) {
  GI_CUDA(cudaMemcpyToSymbol(d_bsel_params, params, sizeof(d_bsel_params)));
  GI_CUDA(cudaMemcpyToSymbol(d_bsel_mean, mean, sizeof(d_bsel_mean)));
  GI_CUDA(cudaMemcpyToSymbol(d_bsel_istd, inv_std, sizeof(d_bsel_istd)));
  return GI_OK;
}

struct BatchGraph {
  const int32_t *ptr, *idx, *wt, *iptr, *iidx;
  int64_t n, m;
  int32_t maxdeg;
  int32_t delta;  // SSSP distance-threshold step (0: relax every frontier source each round)
  int32_t t_warp, t_cta;  // expansion bins: sources with >= t_cta arcs go to the CTA, >= t_warp to a warp
};

struct BatchQuery {
  int32_t graph, src, algo;
  int32_t *out;
  int32_t index;    // position in the caller's query arrays (times and levels are reported there)
  int32_t *parent;  // BFS: canonical parents (NULL: depths only)
};

struct ClusterWs {  // per-cluster working memory (device pointers)
  int32_t *q[2];    // frontier queues
  int32_t *qd[2];   // SSSP: start-of-round distance of each queue entry
  uint32_t *inq;    // SSSP: dedup bitmap of the next frontier
  int64_t *cnt;     // [0..2] rotating counts, [3..5] rotating out-degree sums, [6] claimed query,
                    // [8..11] rotating relaxed-source counts, [12..15] rotating minimum deferred distance
};

constexpr int kBT = 256;  // threads per CTA

__device__ __forceinline__ void csync(cg::cluster_group &cl) {
  __threadfence();
  cl.sync();
}

// Software barrier over the whole (cooperatively launched, hence co-resident)
// grid: arrival counter + generation word.  The wait gives up after
// kBarrierLimitNs of %globaltimer time, sets *err = 2 and reports failure, so
// a broken barrier ends the kernel instead of hanging it.  The outcome is
// taken by thread 0 and shared through shared memory, so a block decides
// uniformly.  `nblocks` is the arrival count that releases the barrier.
constexpr unsigned long long kBarrierLimitNs = 2000000000ull;

__device__ __forceinline__ unsigned long long barrier_clock() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool grid_sync(unsigned *count, unsigned *gen, unsigned nblocks, int32_t *err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    bool ok = true;
    __threadfence();
    const unsigned g0 = *(volatile unsigned *)gen;
    if (atomicAdd(count, 1u) == nblocks - 1) {
      *(volatile unsigned *)count = 0u;
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      const unsigned long long t0 = barrier_clock();
      while (*(volatile unsigned *)gen == g0) {
        if (barrier_clock() - t0 > kBarrierLimitNs) {
          atomicExch(err, 2);
          ok = false;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    s_ok = ok && *(volatile int32_t *)err == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

// One barrier interface for both launch shapes: a hardware cluster barrier
// (cluster mode) or the bounded software grid barrier (whole-GPU mode).
template <bool kGrid>
struct Barrier {
  unsigned *count, *gen;
  int32_t *err;
  int32_t phantoms;  // extra arrivals expected (a test hook; 0 in normal use)
  __device__ bool operator()() const {
    if constexpr (kGrid) {
      return grid_sync(count, gen, gridDim.x + (unsigned)phantoms, err);
    } else {
      cg::cluster_group cl = cg::this_cluster();
      csync(cl);
      return true;
    }
  }
};

// learned / rule decision for BFS level, computed identically by every CTA
__device__ bool batch_decide_pull(const BatchGraph &G, int64_t nf, int64_t mf, int64_t nu, int64_t mu, int32_t level,
                                  int32_t was_pull, int64_t nf_prev, int mode, float alpha, float beta, float *sh) {
  if (mode == 2) {
    // as the single-query selector: frontiers with |F| + m_f below m / 200
    // push without an evaluation (uniform across the CTAs: same inputs)
    if ((nf + mf) * 200 < G.m) return false;
    float *x = sh, *h1 = sh + 16, *h2 = h1 + 64, *y = h2 + 64;
    const float *W1 = d_bsel_params, *b1 = W1 + 64 * 16, *W2 = b1 + 64, *b2 = W2 + 64 * 64, *W3 = b2 + 64,
                *b3 = W3 + 3 * 64;
    const int t = threadIdx.x;
    if (t == 0) {
      float raw[16];
      level_features(raw, G.n, G.m, G.maxdeg, nf, mf, nu, mu, level, was_pull, nf_prev);
      for (int i = 0; i < 16; ++i) x[i] = (raw[i] - d_bsel_mean[i]) * d_bsel_istd[i];
    }
    __syncthreads();
    if (t < 64) {
      float s = b1[t];
      for (int i = 0; i < 16; ++i) s = fmaf(W1[t * 16 + i], x[i], s);
      h1[t] = fmaxf(s, 0.0f);
    }
    __syncthreads();
    if (t < 64) {
      float s = b2[t];
      for (int i = 0; i < 64; ++i) s = fmaf(W2[t * 64 + i], h1[i], s);
      h2[t] = fmaxf(s, 0.0f);
    }
    __syncthreads();
    if (t < 3) {
      float s = b3[t];
      for (int i = 0; i < 64; ++i) s = fmaf(W3[t * 64 + i], h2[i], s);
      y[t] = s;
    }
    __syncthreads();
    // the engine has push and pull; DensePush predictions fold into push
    const float push = fminf(y[0], y[1]);
    const bool pull = y[2] < push;
    __syncthreads();
    return pull;
  }
  if (!was_pull) return (double)mf > (double)mu / (double)alpha;
  return !((double)nf < (double)G.n / (double)beta);
}

// Frontier expansion shared by BFS and SSSP push: every thread takes one
// queue entry; arcs of sources with >= 1024 arcs are spread over the block,
// >= 32 over the warp; the arcs of the remaining sources of the block are laid
// out back to back (block scan of the degrees, an owner byte per arc) and
// expanded one arc per thread, kBatchArcs loads in flight.  fn(du, e, v)
// handles arc e (destination v) of a source whose snapshot value is du.
constexpr int kBatchArcs = 4;

template <class Fn>
__device__ __forceinline__ void strided_arcs(int32_t du, int32_t a, int32_t d, int32_t k0, int32_t step,
                                             const int32_t *__restrict__ idx, Fn &fn) {
  for (int32_t k = k0; k < d; k += kBatchArcs * step) {
    int32_t dd[kBatchArcs], e[kBatchArcs], v[kBatchArcs];
#pragma unroll
    for (int j = 0; j < kBatchArcs; ++j) {
      dd[j] = du;
      e[j] = a + k + j * step;
      v[j] = k + j * step < d ? __ldg(idx + e[j]) : -1;
    }
    fn(dd, e, v);
  }
}

// du of a source: curd[i] (a snapshot), else the current value in live[u], else 0
struct KeepAll {
  __device__ bool operator()(int32_t, int32_t) const { return true; }
};

// kSrcValue: fn receives the source id itself as its value (BFS parents).
template <class Fn, class Keep = KeepAll, bool kSrcValue = false>
__device__ void cta_expand(const BatchGraph &G, const int32_t *cur, const int32_t *curd, const int32_t *live,
                           int64_t nf, int rank, int csize, Fn &fn, Keep keep = Keep()) {
  __shared__ int32_t s_owner, s_a, s_d, s_du;
  __shared__ int32_t s_beg[kBT], s_off[kBT], s_dus[kBT], s_sw[32];
  __shared__ uint8_t s_own[kBT * 31];
  const int tid = threadIdx.x, lane = tid & 31;
  const int64_t T = (int64_t)csize * kBT;
  for (int64_t base = (int64_t)rank * kBT; base < nf; base += T) {
    const int64_t i = base + tid;
    int32_t a = 0, d = 0, du = 0;
    if (i < nf) {
      const int32_t u = cur[i];
      du = kSrcValue ? u : (curd ? curd[i] : (live ? *(volatile const int32_t *)(live + u) : 0));
      if (keep(u, du)) {
        a = __ldg(G.ptr + u);
        d = __ldg(G.ptr + u + 1) - a;
      }
    }
    while (true) {
      if (tid == 0) s_owner = -1;
      __syncthreads();
      if (d >= G.t_cta) s_owner = tid;
      __syncthreads();
      const int owner = s_owner;
      if (owner < 0) break;
      if (tid == owner) {
        s_a = a;
        s_d = d;
        s_du = du;
        d = 0;
      }
      __syncthreads();
      strided_arcs(s_du, s_a, s_d, tid, kBT, G.idx, fn);
      __syncthreads();
    }
    while (true) {
      const unsigned bal = __ballot_sync(0xffffffffu, d >= G.t_warp);
      if (!bal) break;
      const int l = __ffs(bal) - 1;
      const int32_t wa = __shfl_sync(0xffffffffu, a, l), wd = __shfl_sync(0xffffffffu, d, l),
                    wdu = __shfl_sync(0xffffffffu, du, l);
      if (lane == l) d = 0;
      strided_arcs(wdu, wa, wd, lane, 32, G.idx, fn);
    }
    int32_t total;
    const int32_t off = block_excl_scan(d, &total, s_sw);
    s_beg[tid] = a;
    s_off[tid] = off;
    s_dus[tid] = du;
    for (int32_t k = 0; k < d; ++k) s_own[off + k] = (uint8_t)tid;
    __syncthreads();
    for (int32_t j0 = tid; j0 < total; j0 += kBatchArcs * kBT) {
      int32_t e[kBatchArcs], dd[kBatchArcs], v[kBatchArcs];
#pragma unroll
      for (int b2 = 0; b2 < kBatchArcs; ++b2) {
        const int32_t j = j0 + b2 * kBT;
        if (j < total) {
          const int o = s_own[j];
          e[b2] = s_beg[o] + (j - s_off[o]);
          dd[b2] = s_dus[o];
          v[b2] = __ldg(G.idx + e[b2]);
        } else {
          e[b2] = 0;
          dd[b2] = 0;
          v[b2] = -1;
        }
      }
      fn(dd, e, v);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ void append_warp(bool want, int32_t v, int32_t *next, int64_t *ncnt) {
  const int lane = threadIdx.x & 31;
  const unsigned active = __activemask();
  const unsigned ball = __ballot_sync(active, want);
  if (!ball) return;
  const int leader = __ffs(ball) - 1;
  long long base = 0;
  if (lane == leader) base = atomicAdd(reinterpret_cast<unsigned long long *>(ncnt), (unsigned long long)__popc(ball));
  base = __shfl_sync(active, base, leader);
  if (want) next[base + __popc(ball & ((1u << lane) - 1u))] = v;
}

// One warp-aggregated append of a batch (v[j] where want[j]): one atomic for
// the batch instead of one per arc.
__device__ __forceinline__ void append_batch(const bool (&want)[kBatchArcs], const int32_t (&v)[kBatchArcs],
                                             int32_t *next, int64_t *ncnt) {
  const int lane = threadIdx.x & 31;
  const unsigned active = __activemask();
  unsigned ball[kBatchArcs];
  int32_t tot = 0;
#pragma unroll
  for (int j = 0; j < kBatchArcs; ++j) {
    ball[j] = __ballot_sync(active, want[j]);
    tot += __popc(ball[j]);
  }
  if (tot == 0) return;
  const int leader = __ffs(active) - 1;
  long long base = 0;
  if (lane == leader) base = atomicAdd(reinterpret_cast<unsigned long long *>(ncnt), (unsigned long long)tot);
  base = __shfl_sync(active, base, leader);
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int j = 0; j < kBatchArcs; ++j) {
    if (want[j]) next[base + __popc(ball[j] & lt)] = v[j];
    base += __popc(ball[j]);
  }
}

// BFS SparsePush of this level's queue: newly reached vertices get depth L+1
// and join the next queue (their out-degrees summed into the edge count).
// With parents, every source u reaching a vertex of depth L+1 lowers its
// parent to u by atomicMin (after a plain read shows u is smaller), so the
// parent ends as the smallest-id in-neighbour one level closer.
__device__ void batch_bfs_push(const BatchGraph &G, int32_t *depth, int32_t *parent, const int32_t *cur, int64_t nf,
                               int32_t *next, int64_t *ncnt, int64_t *necnt, int32_t L, int rank, int csize) {
  // a batch's claims first, then one append and one edge-count add per warp
  auto fn = [&](const int32_t (&u)[kBatchArcs], const int32_t (&)[kBatchArcs], const int32_t (&v)[kBatchArcs]) {
    bool won[kBatchArcs];
#pragma unroll
    for (int j = 0; j < kBatchArcs; ++j) {
      won[j] = false;
      if (v[j] < 0) continue;
      int32_t d = *(volatile int32_t *)(depth + v[j]);
      if (d == -1) {
        d = atomicCAS(depth + v[j], -1, L + 1);
        won[j] = d == -1;
        if (won[j]) d = L + 1;
      }
      if (parent && d == L + 1 && u[j] < *(volatile int32_t *)(parent + v[j])) atomicMin(parent + v[j], u[j]);
    }
    append_batch(won, v, next, ncnt);
    // the won vertices are distinct, so a warp's degree sum is below m < 2^31
    uint32_t deg = 0;
#pragma unroll
    for (int j = 0; j < kBatchArcs; ++j)
      if (won[j]) deg += (uint32_t)(__ldg(G.ptr + v[j] + 1) - __ldg(G.ptr + v[j]));
    const unsigned active = __activemask();
    const uint32_t wdeg = __reduce_add_sync(active, deg);
    if (wdeg && (threadIdx.x & 31) == __ffs(active) - 1)
      atomicAdd(reinterpret_cast<unsigned long long *>(necnt), (unsigned long long)wdeg);
  };
  cta_expand<decltype(fn), KeepAll, true>(G, cur, nullptr, nullptr, nf, rank, csize, fn);
}

// BFS DensePull with early exit: the frontier is {u : depth[u] == L}; the
// first frontier in-neighbour in ascending order is the canonical parent.
__device__ void batch_bfs_pull(const BatchGraph &G, int32_t *depth, int32_t *parent, int32_t *next, int64_t *ncnt,
                               int64_t *necnt, int32_t L, int rank, int csize) {
  // as the single-query early-exit pull: each lane probes its row's first 4
  // arcs before any warp-wide scan, the next rows' depth and bounds are
  // fetched under the current probe, found vertices are staged per warp and
  // appended kQBuf - 32 or more at a time, and the edge count is summed per
  // lane and added once per warp
  constexpr int kQBuf = 128;
  __shared__ int32_t s_q[kBT / 32][kQBuf];
  const int lane = threadIdx.x & 31;
  int32_t *wq = s_q[threadIdx.x >> 5];
  int32_t qn = 0;
  unsigned long long edges = 0;
  const auto flush = [&]() {
    __syncwarp();
    long long base = 0;
    if (lane == 0) base = atomicAdd(reinterpret_cast<unsigned long long *>(ncnt), (unsigned long long)qn);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (int32_t j = lane; j < qn; j += 32) next[base + j] = wq[j];
    __syncwarp();
    qn = 0;
  };
  const int64_t nw = (G.n + 31) >> 5;
  const int64_t wstride = (int64_t)csize * (kBT / 32);
  int32_t ndv = 0, na = 0, nb = 0;
  const auto fetch = [&](int64_t ww) {
    const int64_t vv = ww * 32 + lane;
    if (ww < nw && vv < G.n) {
      ndv = depth[vv];
      na = G.iptr[vv];
      nb = G.iptr[vv + 1];
    }
  };
  int64_t w = (int64_t)rank * (kBT / 32) + (threadIdx.x >> 5);
  fetch(w);
  for (; w < nw; w += wstride) {
    const int64_t v = w * 32 + lane;
    const int32_t dv = ndv;
    int32_t a = na, b = nb;
    fetch(w + wstride);
    const bool active = v < G.n && dv == -1;
    if (!active) b = a;
    bool found = false;
    int32_t par = -1;
    for (int32_t e = a; e < b && !found; e += 4) {
      int32_t u[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) u[j] = e + j < b ? G.iidx[e + j] : -1;
#pragma unroll
      for (int j = 3; j >= 0; --j)
        if (u[j] >= 0 && depth[u[j]] == L) {
          found = true;
          par = u[j];
        }
      if (b - a >= 32) break;
    }
    const bool big = active && !found && (b - a) >= 32;
    unsigned bal = __ballot_sync(0xffffffffu, big);
    while (bal) {
      const int l = __ffs(bal) - 1;
      bal &= bal - 1;
      const int32_t lb = __shfl_sync(0xffffffffu, b, l), la = __shfl_sync(0xffffffffu, a, l) + 4;
      int32_t hit = -1;
      for (int32_t base = la; base < lb && hit < 0; base += 32) {
        const int32_t e = base + lane;
        const int32_t u = e < lb ? G.iidx[e] : -1;
        const unsigned h = __ballot_sync(0xffffffffu, u >= 0 && depth[u] == L);
        if (h) hit = __shfl_sync(0xffffffffu, u, __ffs(h) - 1);
      }
      if (lane == l && hit >= 0) {
        found = true;
        par = hit;
      }
    }
    if (found) {
      depth[v] = L + 1;
      if (parent) parent[v] = par;
      edges += (unsigned long long)(G.ptr[v + 1] - G.ptr[v]);
    }
    const unsigned word = __ballot_sync(0xffffffffu, found);
    if (word) {
      if (found) wq[qn + __popc(word & ((1u << lane) - 1u))] = (int32_t)v;
      qn += __popc(word);
      if (qn > kQBuf - 32) flush();
    }
  }
  if (qn > 0) flush();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) edges += __shfl_xor_sync(0xffffffffu, edges, o);
  if (lane == 0 && edges) atomicAdd(reinterpret_cast<unsigned long long *>(necnt), edges);
}

// SSSP push relax of this round's queue with asynchronous min updates (the
// asyncMin of Sec. 6): each source offers its current distance, so an
// improvement made earlier in the round propagates at once.  The final
// distances are the unique shortest distances, as with synchronous rounds;
// the rounds and frontiers are not (the engine does not report them per
// round).  Each improved destination joins the next queue once (dedup bitmap).
//
// With a threshold theta (G.delta > 0), a frontier source whose distance is
// >= theta is not relaxed this round: it stays in the frontier, and the
// smallest such distance is recorded so that theta can move past it when a
// round relaxes nothing (a near/far ordering of the same label-correcting
// relaxation; any order reaches the same distances).
__device__ void batch_sssp_push(const BatchGraph &G, int32_t *dist, const int32_t *cur, int64_t nf, int32_t *next,
                                int64_t *ncnt, uint32_t *inq, int64_t theta, int64_t *relaxed, int64_t *mindef,
                                int rank, int csize) {
  const int lane = threadIdx.x & 31;
  auto keep = [&](int32_t u, int32_t du) -> bool {
    const bool near = (int64_t)du < theta;
    bool fresh = false;
    if (!near) {
      const uint32_t mask = 1u << (u & 31);
      fresh = (atomicOr(inq + (u >> 5), mask) & mask) == 0;
      atomicMin(reinterpret_cast<long long *>(mindef), (long long)du);
    }
    append_warp(fresh, u, next, ncnt);
    const unsigned active = __activemask();
    const unsigned ball = __ballot_sync(active, near);
    if (ball && lane == __ffs(ball) - 1)
      atomicAdd(reinterpret_cast<unsigned long long *>(relaxed), (unsigned long long)__popc(ball));
    return near;
  };
  // a batch's relaxations first, then its dedup tests, then one append
  auto fn = [&](const int32_t (&du)[kBatchArcs], const int32_t (&e)[kBatchArcs], const int32_t (&v)[kBatchArcs]) {
    bool better[kBatchArcs], fresh[kBatchArcs];
#pragma unroll
    for (int j = 0; j < kBatchArcs; ++j) {
      better[j] = false;
      if (v[j] >= 0) {
        const long long nd = (long long)du[j] + __ldg(G.wt + e[j]);
        if (nd < *(volatile int32_t *)(dist + v[j])) better[j] = nd < atomicMin(dist + v[j], (int32_t)nd);
      }
    }
#pragma unroll
    for (int j = 0; j < kBatchArcs; ++j) {
      fresh[j] = false;
      if (better[j]) {
        const uint32_t mask = 1u << (v[j] & 31);
        fresh[j] = (atomicOr(inq + (v[j] >> 5), mask) & mask) == 0;
      }
    }
    append_batch(fresh, v, next, ncnt);
  };
  cta_expand(G, cur, nullptr, dist, nf, rank, csize, fn, keep);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <bool kGrid>
__global__ void __launch_bounds__(kBT) k_batch(const BatchGraph *__restrict__ graphs,
                                               const BatchQuery *__restrict__ queries, int32_t n_q,
                                               int32_t *work, ClusterWs *ws, int64_t *q_ns, int32_t *q_levels,
                                               int mode, float alpha, float beta, int64_t level_cap, int32_t *err,
                                               int32_t phantoms) {
  int rank, csize;
  if constexpr (kGrid) {
    rank = blockIdx.x;
    csize = gridDim.x;
  } else {
    cg::cluster_group cl = cg::this_cluster();
    rank = (int)cl.block_rank();
    csize = (int)cl.num_blocks();
  }
  const Barrier<kGrid> bar{reinterpret_cast<unsigned *>(work + 2), reinterpret_cast<unsigned *>(work + 3), err,
                           phantoms};
  const int cid = blockIdx.x / csize;
  const int64_t T = (int64_t)csize * kBT;
  const int64_t gtid = (int64_t)rank * kBT + threadIdx.x;
  ClusterWs W = ws[cid];
  __shared__ float sh[16 + 64 + 64 + 4];
  while (true) {
    if (rank == 0 && threadIdx.x == 0) W.cnt[6] = atomicAdd(work, 1);
    if (!bar()) return;
    const int32_t qi = (int32_t)*(volatile int64_t *)(W.cnt + 6);
    if (!bar()) return;  // everyone has read the claim before it can be overwritten
    if (qi >= n_q) break;
    const BatchQuery Q = queries[qi];
    const BatchGraph G = graphs[Q.graph];
    unsigned long long t0 = 0;
    if (gtid == 0) t0 = global_ns();
    const bool bfs = Q.algo == GI_ALGO_BFS;
    for (int64_t v = gtid; v < G.n; v += T) Q.out[v] = bfs ? -1 : INT32_MAX;
    if (bfs && Q.parent)
      for (int64_t v = gtid; v < G.n; v += T) Q.parent[v] = v == Q.src ? Q.src : INT32_MAX;
    if (!bfs)
      for (int64_t w = gtid; w < (G.n + 31) / 32; w += T) W.inq[w] = 0u;
    if (gtid == 0) {
      for (int k = 0; k < 6; ++k) W.cnt[k] = 0;
      for (int k = 8; k < 12; ++k) W.cnt[k] = 0;
      for (int k = 12; k < 16; ++k) W.cnt[k] = INT64_MAX;
      W.cnt[0] = 1;
      W.cnt[3] = G.ptr[Q.src + 1] - G.ptr[Q.src];
      W.q[0][0] = Q.src;
      W.qd[0][0] = 0;
    }
    if (!bar()) return;
    if (gtid == 0) Q.out[Q.src] = 0;
    if (!bar()) return;
    int64_t nu = G.n, mu = G.m, nf_prev = 0;
    int32_t was_pull = 0, levels = 0;
    int64_t theta = G.delta > 0 ? (int64_t)G.delta : INT64_MAX;
    for (int32_t L = 0;; ++L) {
      const int64_t nf = *(volatile int64_t *)(W.cnt + (L % 3));
      const int64_t mf = *(volatile int64_t *)(W.cnt + 3 + (L % 3));
      levels = L;
      if (nf == 0) break;
      if (L >= level_cap) {  // uniform: every CTA sees the same L
        if (gtid == 0) atomicExch(err, 1);
        break;
      }
      if (gtid == 0) {
        W.cnt[(L + 2) % 3] = 0;
        W.cnt[3 + (L + 2) % 3] = 0;
        // slots read at the end of round L-2 (barriers since), written in round L+2
        W.cnt[8 + (L + 2) % 4] = 0;
        W.cnt[12 + (L + 2) % 4] = INT64_MAX;
      }
      int32_t *cur = W.q[L & 1], *next = W.q[(L + 1) & 1];
      int64_t *ncnt = W.cnt + (L + 1) % 3, *necnt = W.cnt + 3 + (L + 1) % 3;
      if (bfs) {
        nu -= nf;
        mu -= mf;
        const bool pull = (mode == 0) ? false
                                      : batch_decide_pull(G, nf, mf, nu, mu, L, was_pull, nf_prev, mode, alpha, beta,
                                                          sh);
        if (pull) batch_bfs_pull(G, Q.out, Q.parent, next, ncnt, necnt, L, rank, csize);
        else batch_bfs_push(G, Q.out, Q.parent, cur, nf, next, ncnt, necnt, L, rank, csize);
        was_pull = pull ? 1 : 0;
        nf_prev = nf;
        if (!bar()) return;
      } else {
        batch_sssp_push(G, Q.out, cur, nf, next, ncnt, W.inq, theta, W.cnt + 8 + L % 4, W.cnt + 12 + L % 4,
                        rank, csize);
        if (!bar()) return;
        const int64_t nn = *(volatile int64_t *)ncnt;
        for (int64_t i = gtid; i < nn; i += T) {
          const int32_t v = next[i];
          atomicAnd(W.inq + (v >> 5), ~(1u << (v & 31)));
        }
        if (!bar()) return;
        if (G.delta > 0 && *(volatile int64_t *)(W.cnt + 8 + L % 4) == 0)
          theta = *(volatile int64_t *)(W.cnt + 12 + L % 4) + G.delta;  // nothing was near: move past the nearest
      }
    }
    if (bfs && Q.parent) {  // unreached vertices: -1
      if (!bar()) return;
      for (int64_t v = gtid; v < G.n; v += T)
        if (Q.parent[v] == INT32_MAX) Q.parent[v] = -1;
    }
    if (gtid == 0 && q_ns) q_ns[Q.index] = (int64_t)(global_ns() - t0);
    if (gtid == 0 && q_levels) q_levels[Q.index] = levels;
    if (!bar()) return;
  }
}

}  // namespace gi

using namespace gi;

// test hook (gi_debug_barrier_phantoms): extra arrivals the grid barrier waits for
static int32_t g_barrier_phantoms = 0;

extern "C" int gi_debug_barrier_phantoms(int32_t k) {
  GI_ARG(k >= 0 && k <= 1024, "phantom count must be in [0, 1024]");
  g_barrier_phantoms = k;
  return GI_OK;
}

struct gi_batch_plan {
  gi::BatchGraph *dg = nullptr;
  gi::BatchQuery *dq = nullptr;
  gi::ClusterWs *dws = nullptr;
  int32_t *work = nullptr;  // [0] query counter, [1] error flag
  int32_t *slab = nullptr;
  int64_t *cnts = nullptr, *dns = nullptr;
  int32_t *dlev = nullptr;
  int32_t n_q = 0, clusters = 0, cluster_size = 0, selector = 0, grid_blocks = 0;
  float alpha = 14.0f, beta = 24.0f;
  int64_t cap = 0;
  int32_t *levels_host = nullptr;
};

static void plan_release(gi_batch_plan *p, cudaStream_t s) {
  dev_free(p->dg, s);
  dev_free(p->dq, s);
  dev_free(p->dws, s);
  dev_free(p->work, s);
  dev_free(p->slab, s);
  dev_free(p->cnts, s);
  dev_free(p->dns, s);
  dev_free(p->dlev, s);
  delete p;
}

extern "C" int gi_batch_plan_create(gi_graph *const *graphs, int32_t n_graphs, const int32_t *q_graph,
                                    const int32_t *q_src, const int32_t *q_algo, int32_t n_q,
                                    int32_t *const *out_dev, const gi_batch_opts *opts, void *stream,
                                    gi_batch_plan **out) {
  GI_ARG(out != nullptr, "out is NULL");
  *out = nullptr;
  GI_ARG(graphs != nullptr && n_graphs > 0, "no graphs");
  GI_ARG(n_q > 0 && q_graph && q_src && q_algo && out_dev, "bad query arrays");
  gi_batch_opts o;
  gi_batch_opts_default(&o);
  if (opts) o = *opts;
  GI_ARG(o.cluster_size == 0 || o.cluster_size == 1 || o.cluster_size == 2 || o.cluster_size == 4 ||
             o.cluster_size == 8,
         "cluster_size must be 0 (whole GPU), 1, 2, 4 or 8");
  GI_ARG(o.selector == GI_DIR_SPARSE_PUSH || o.selector == GI_DIR_HYBRID_PULL || o.selector == GI_DIR_LEARNED,
         "selector must be GI_DIR_SPARSE_PUSH, GI_DIR_HYBRID_PULL or GI_DIR_LEARNED");
  GI_ARG(o.order == 0 || o.order == 1, "order must be 0 (as given) or 1 (largest first)");
  const int32_t tw = o.t_warp > 0 ? o.t_warp : 32, tc = o.t_cta > 0 ? o.t_cta : 1024;
  GI_ARG(tw >= 1 && tw <= 32, "t_warp must be in [1, 32] (0: 32)");
  GI_ARG(tc >= tw, "t_cta must be >= t_warp (0: 1024)");
  std::vector<BatchGraph> hg(n_graphs);
  int64_t nmax = 1;
  for (int i = 0; i < n_graphs; ++i) {
    const gi_graph *g = graphs[i];
    GI_ARG(g != nullptr, "NULL graph");
    int32_t delta = 0;
    if (g->out.wt && o.sssp_delta >= 0.0f) {
      const double scale = o.sssp_delta > 0.0f ? o.sssp_delta : 2.0;
      delta = (int32_t)fmin(scale * g->wt_mean + 0.5, 1e9);
      if (delta < 1) delta = 1;
    }
    hg[i] = BatchGraph{g->out.ptr, g->out.idx, g->out.wt, g->in.ptr, g->in.idx, g->n, g->m, g->max_deg, delta,
                       tw, tc};
    nmax = g->n > nmax ? g->n : nmax;
  }
  std::vector<BatchQuery> hq(n_q);
  for (int i = 0; i < n_q; ++i) {
    GI_ARG(q_graph[i] >= 0 && q_graph[i] < n_graphs, "query graph index out of range");
    const gi_graph *g = graphs[q_graph[i]];
    GI_ARG(q_src[i] >= 0 && q_src[i] < g->n, "query source out of range");
    GI_ARG(q_algo[i] == GI_ALGO_BFS || q_algo[i] == GI_ALGO_SSSP, "query algorithm must be BFS or SSSP");
    if (q_algo[i] == GI_ALGO_SSSP) GI_ARG(g->out.wt != nullptr, "SSSP query on a graph without weights");
    if (q_algo[i] == GI_ALGO_BFS && o.selector != GI_DIR_SPARSE_PUSH)
      GI_ARG(g->has_csc, "pull levels need the in-edges (symmetric graph or gi_load_csc)");
    GI_ARG(out_dev[i] != nullptr, "NULL output");
    int32_t *par = (o.parents && q_algo[i] == GI_ALGO_BFS) ? o.parents[i] : nullptr;
    GI_ARG(par == nullptr || (par != out_dev[i]), "a parent array aliases its depth array");
    hq[i] = BatchQuery{q_graph[i], q_src[i], q_algo[i], out_dev[i], i, par};
  }
  if (o.order == 1) {
    // largest first (longest-processing-time order): vertex count is the proxy
    // for both the work and, on road-like graphs, the number of levels; SSSP
    // before BFS on the same graph; ties keep the caller's order
    std::stable_sort(hq.begin(), hq.end(), [&](const BatchQuery &x, const BatchQuery &y) {
      const int64_t nx = graphs[x.graph]->n, ny = graphs[y.graph]->n;
      if (nx != ny) return nx > ny;
      return x.algo == GI_ALGO_SSSP && y.algo != GI_ALGO_SSSP;
    });
  }
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  GI_CUDA(cudaGetDevice(&dev));
  GI_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  gi_batch_plan *p = new gi_batch_plan();
  p->n_q = n_q;
  p->cluster_size = o.cluster_size;
  if (o.cluster_size == 0) {
    // whole-GPU mode: one group of every co-resident block (cooperative launch)
    int per_sm = 0;
    GI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<true>, kBT, 0));
    if (per_sm < 1) {
      set_error("the persistent kernel does not fit on an SM");
      return GI_ERR_UNSUPPORTED;
    }
    p->clusters = 1;
    p->grid_blocks = sms * (per_sm < 2 ? per_sm : 2);
  } else {
    p->clusters = o.clusters > 0 ? o.clusters : sms / o.cluster_size;
    if (p->clusters > n_q) p->clusters = n_q;
    if (p->clusters < 1) p->clusters = 1;
  }
  p->selector = o.selector;
  p->alpha = o.alpha;
  p->beta = o.beta;
  p->cap = o.level_cap > 0 ? o.level_cap : 4 * nmax + 16;  // threshold rounds can exceed n
  const int64_t words = (nmax + 31) / 32;
  const int64_t per = 4 * nmax + words;  // 2 queues + 2 distance queues + bitmap, in int32 words
  std::vector<ClusterWs> hws(p->clusters);
  int st = dev_alloc_n(&p->dg, n_graphs, s);
  if (st == GI_OK) st = dev_alloc_n(&p->dq, n_q, s);
  if (st == GI_OK) st = dev_alloc_n(&p->dws, p->clusters, s);
  if (st == GI_OK) st = dev_alloc_n(&p->work, 4, s);
  if (st == GI_OK) st = dev_alloc_n(&p->slab, per * p->clusters, s);
  if (st == GI_OK) st = dev_alloc_n(&p->cnts, 16 * p->clusters, s);
  if (st == GI_OK) st = dev_alloc_n(&p->dns, n_q, s);
  if (st == GI_OK) st = dev_alloc_n(&p->dlev, n_q, s);
  if (st == GI_OK) {
    for (int c = 0; c < p->clusters; ++c) {
      int32_t *b = p->slab + per * c;
      hws[c].q[0] = b;
      hws[c].q[1] = b + nmax;
      hws[c].qd[0] = b + 2 * nmax;
      hws[c].qd[1] = b + 3 * nmax;
      hws[c].inq = reinterpret_cast<uint32_t *>(b + 4 * nmax);
      hws[c].cnt = p->cnts + 16 * c;
    }
    if (cudaMemcpyAsync(p->dg, hg.data(), sizeof(BatchGraph) * n_graphs, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(p->dq, hq.data(), sizeof(BatchQuery) * n_q, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(p->dws, hws.data(), sizeof(ClusterWs) * p->clusters, cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      st = cuda_fail(cudaGetLastError(), "batch plan", __FILE__, __LINE__);
  }
  if (st != GI_OK) {
    cudaStreamSynchronize(s);
    plan_release(p, s);
    return st;
  }
  *out = p;
  return GI_OK;
}

extern "C" int gi_batch_plan_launch(gi_batch_plan *p, void *stream) {
  GI_ARG(p != nullptr, "plan is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  // work: [0] query counter, [1] error flag, [2] grid-barrier arrivals, [3] grid-barrier generation
  GI_CUDA(cudaMemsetAsync(p->work, 0, 4 * sizeof(int32_t), s));
  const bool grid_mode = p->cluster_size == 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(grid_mode ? p->grid_blocks : p->clusters * p->cluster_size));
  cfg.blockDim = dim3(kBT);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  if (grid_mode) {
    attr[0].id = cudaLaunchAttributeCooperative;  // guarantees co-residency for the grid barrier
    attr[0].val.cooperative = 1;
  } else {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)p->cluster_size;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
  }
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const int mode = p->selector == GI_DIR_SPARSE_PUSH ? 0 : (p->selector == GI_DIR_LEARNED && selector_loaded() ? 2 : 1);
  const int tok = timing_begin(kClassBatch, s);
  cudaError_t e = grid_mode
                      ? cudaLaunchKernelEx(&cfg, k_batch<true>, (const BatchGraph *)p->dg, (const BatchQuery *)p->dq,
                                           p->n_q, p->work, p->dws, p->dns, p->dlev, mode, p->alpha, p->beta, p->cap,
                                           p->work + 1, g_barrier_phantoms)
                      : cudaLaunchKernelEx(&cfg, k_batch<false>, (const BatchGraph *)p->dg,
                                           (const BatchQuery *)p->dq, p->n_q, p->work, p->dws, p->dns, p->dlev, mode,
                                           p->alpha, p->beta, p->cap, p->work + 1, 0);
  timing_end(tok, s);
  note_launch(1);
  if (e != cudaSuccess) return cuda_fail(e, "batch launch", __FILE__, __LINE__);
  return GI_OK;
}

extern "C" int gi_batch_plan_results(gi_batch_plan *p, int64_t *q_ns, int32_t *levels, void *stream) {
  GI_ARG(p != nullptr, "plan is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  int32_t err = 0;
  GI_CUDA(cudaMemcpyAsync(&err, p->work + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  if (q_ns) GI_CUDA(cudaMemcpyAsync(q_ns, p->dns, sizeof(int64_t) * p->n_q, cudaMemcpyDeviceToHost, s));
  if (levels) GI_CUDA(cudaMemcpyAsync(levels, p->dlev, sizeof(int32_t) * p->n_q, cudaMemcpyDeviceToHost, s));
  GI_CUDA(cudaStreamSynchronize(s));
  if (err) {
    set_error(err == 2 ? "a grid barrier of the persistent kernel timed out"
                       : "a query exceeded the level cap of the batched engine");
    return GI_ERR_TIMEOUT;
  }
  return GI_OK;
}

extern "C" int gi_batch_plan_free(gi_batch_plan *p) {
  if (!p) return GI_OK;
  cudaDeviceSynchronize();
  plan_release(p, 0);
  GI_CUDA(cudaStreamSynchronize(0));
  return GI_OK;
}

extern "C" int gi_batch_run(gi_graph *const *graphs, int32_t n_graphs, const int32_t *q_graph, const int32_t *q_src,
                            const int32_t *q_algo, int32_t n_q, int32_t *const *out_dev, int64_t *q_ns,
                            const gi_batch_opts *opts, void *stream) {
  GI_ARG(n_q >= 0, "n_q must be >= 0");
  if (n_q == 0) return GI_OK;
  gi_batch_plan *p = nullptr;
  GI_TRY(gi_batch_plan_create(graphs, n_graphs, q_graph, q_src, q_algo, n_q, out_dev, opts, stream, &p));
  int st = gi_batch_plan_launch(p, stream);
  if (st == GI_OK) st = gi_batch_plan_results(p, q_ns, opts ? opts->levels : nullptr, stream);
  const int st2 = gi_batch_plan_free(p);
  return st != GI_OK ? st : st2;
}

extern "C" void gi_batch_opts_default(gi_batch_opts *o) {
  if (!o) return;
  o->cluster_size = 4;
  o->clusters = 0;
  o->selector = GI_DIR_HYBRID_PULL;
  o->alpha = 14.0f;
  o->beta = 24.0f;
  o->level_cap = 0;
  o->levels = nullptr;
  o->sssp_delta = 0.0f;
  o->order = 1;
  o->t_warp = 32;
  o->t_cta = 1024;
  o->parents = nullptr;
}
