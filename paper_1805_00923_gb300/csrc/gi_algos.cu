// Algorithm drivers built on the edgeset apply kernels: BFS, Bellman-Ford
// SSSP, label-propagation CC, PageRank, PageRankDelta and single-source
// Betweenness Centrality (Sec. 7's benchmarks).  Each iteration: fused frontier statistics + direction choice,
// one traversal, and (where the algorithm needs one) a vertex epilogue.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "gi_traverse.cuh"

namespace gi {

// ------------------------------------------------------------ helper kernels --
__global__ void k_fill_i32(int32_t *x, int64_t n, int32_t val) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = val;
}

__global__ void k_iota2(int32_t *a, int32_t *b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = b[i] = (int32_t)i;
}

__global__ void k_bfs_init(int32_t *depth, int32_t *parent, int64_t n, int32_t src, int32_t *unv_st = nullptr) {
  // the compacted unvisited walk starts from the live list (BfsUnv)
  if (unv_st && blockIdx.x == 0 && threadIdx.x < 4) unv_st[threadIdx.x] = threadIdx.x == 0 ? -1 : 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    depth[i] = i == src ? 0 : -1;
    if (parent) parent[i] = i == src ? src : INT32_MAX;
  }
}

__global__ void k_parent_fix(int32_t *parent, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (parent[i] == INT32_MAX) parent[i] = -1;
}

// the graph-driven loop's parents copied out with the same fix-up (one pass)
__global__ void k_parent_copy_fix(int32_t *__restrict__ dst, const int32_t *__restrict__ src, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = src[i];
    dst[i] = p == INT32_MAX ? -1 : p;
  }
}

__global__ void k_set_one(int32_t *x, int32_t i, int32_t val) { x[i] = val; }

// snapshot maintenance for synchronous rounds: frontier members carry their
// start-of-round value in snap[], everyone else INT32_MAX
__global__ void k_snap_reset(const int32_t *__restrict__ q, const int32_t *__restrict__ qc, int32_t *snap) {
  int32_t c = *qc;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < c; i += gridDim.x * blockDim.x) snap[q[i]] = INT32_MAX;
}

__global__ void k_snap_set(const int32_t *__restrict__ q, const int32_t *__restrict__ qc, int32_t *snap,
                           const int32_t *__restrict__ x) {
  int32_t c = *qc;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < c; i += gridDim.x * blockDim.x) {
    int32_t v = q[i];
    snap[v] = x[v];
  }
}

__global__ void k_pr_init(float *contrib, const float *__restrict__ inv_deg, int64_t n, float init) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    contrib[i] = init * inv_deg[i];
}

__global__ void k_fill_f32(float *x, int64_t n, float val) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = val;
}

// PageRank vertex update after a push iteration: rank = base + d*acc
template <class A>
__global__ void k_pr_vertex(A *acc, float *contrib_out, float *rank_out, const float *__restrict__ inv_deg,
                            int64_t n, float base, float damping) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float r = fmaf(damping, (float)acc[i], base);
    acc[i] = 0;
    if (rank_out) rank_out[i] = r;
    else contrib_out[i] = r * inv_deg[i];
  }
}

// FP64 sum of ranks: per-block partial sums, then each block of the scale
// kernel adds the partials in the same fixed order and divides its range.
__global__ void k_sum_f64(const float *__restrict__ x, int64_t n, double *partial) {
  __shared__ double sw[32];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += (double)x[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += sw[w];
    partial[blockIdx.x] = b;
  }
}

__global__ void k_scale_f64(float *x, int64_t n, const double *__restrict__ partial, int32_t np) {
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

// PageRankDelta vertex filter after a push round (Fig. 1): Delta, Rank,
// DeltaSum reset, next frontier (bitmap word per warp + queue), next contrib.
template <class A>
__global__ void k_prd_vertex(A *dsum, float *rank, float *contrib_out, const float *__restrict__ inv_deg,
                             int64_t n, float damping, float first_base, float inv_n, float eps, int32_t first_round,
                             uint32_t *out_bm, int32_t *out_q, int32_t *out_qc) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (n + 31) >> 5;
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nw;
       w += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t v = w * 32 + lane;
    bool active = false;
    if (v < n) {
      float s = (float)dsum[v], r = rank[v], delta;
      if (first_round) {
        delta = fmaf(damping, s, first_base);
        r += delta;
        delta -= inv_n;
      } else {
        delta = damping * s;
        r += delta;
      }
      rank[v] = r;
      dsum[v] = 0;
      active = fabsf(delta) > eps * r;
      contrib_out[v] = active ? delta * inv_deg[v] : 0.0f;
    }
    const unsigned word = __ballot_sync(0xffffffffu, active);
    if (lane == 0) out_bm[w] = word;
    if (word) {
      int32_t base = 0;
      if (lane == 0) base = atomicAdd(out_qc, __popc(word));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (active) out_q[base + __popc(word & ((1u << lane) - 1u))] = (int32_t)v;
    }
  }
}

// Segmented min pull, vertex pass: x[v] = min(x[v], acc[v]) (acc holds the
// minimum over all segments), marks lowered vertices (bitmap word per warp +
// queue) and resets acc for the next round.
__global__ void k_min_apply(int32_t *x, int32_t *acc, int64_t n, uint32_t *out_bm, int32_t *out_q, int32_t *out_qc) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (n + 31) >> 5;
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nw;
       w += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t v = w * 32 + lane;
    bool low = false;
    if (v < n) {
      const int32_t c = acc[v];
      acc[v] = INT32_MAX;
      if (c < x[v]) {
        x[v] = c;
        low = true;
      }
    }
    const unsigned word = __ballot_sync(0xffffffffu, low);
    if (lane == 0) out_bm[w] = word;
    if (word) {
      int32_t base = 0;
      if (lane == 0) base = atomicAdd(out_qc, __popc(word));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (low) out_q[base + __popc(word & ((1u << lane) - 1u))] = (int32_t)v;
    }
  }
}

// ----------------------------------------------------------------- helpers --
struct VsetPair {
  gi_vset a, b;
  gi_vset *F = &a, *N = &b;
  void swap() {
    gi_vset *t = F;
    F = N;
    N = t;
  }
};

static int pair_alloc(gi_graph *g, VsetPair &p, cudaStream_t s) {
  GI_TRY(vset_alloc(g, &p.a, s));
  GI_TRY(vset_alloc(g, &p.b, s));
  return GI_OK;
}

static void pair_free(VsetPair &p, cudaStream_t s) {
  for (gi_vset *v : {&p.a, &p.b}) {
    dev_free(v->queue, s);
    dev_free(v->count, s);
    dev_free(v->bitmap, s);
    dev_free(v->boolmap, s);
    v->queue = v->count = nullptr;
    v->bitmap = nullptr;
    v->boolmap = nullptr;
  }
}

// F = {v} (v >= 0), all vertices (v == -1)
__global__ void k_front_init(int32_t *q, int32_t *qc, uint32_t *bm, int64_t words, int64_t n, int32_t v) {
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += (int64_t)gridDim.x * blockDim.x) {
    uint32_t word = 0;
    if (v < 0) {
      int64_t rem = n - w * 32;
      word = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
    } else if ((v >> 5) == w) {
      word = 1u << (v & 31);
    }
    bm[w] = word;
  }
  if (v < 0) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
      q[i] = (int32_t)i;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (v >= 0) q[0] = v;
    *qc = v >= 0 ? 1 : (int32_t)n;
  }
}

static int front_init(gi_graph *g, gi_vset *F, int32_t v, cudaStream_t s) {
  int64_t work = g->n > F->words ? g->n : F->words;
  k_front_init<<<grid_for(g, work, 256), 256, 0, s>>>(F->queue, F->count, F->bitmap, F->words, g->n, v);
  GI_LAUNCH_CHECK();
  F->reps = GI_REP_SPARSE | GI_REP_BITMAP;
  return GI_OK;
}

static void trace_put(gi_trace *tr, int32_t it, const int64_t *ctrl_host, int32_t phase = 0) {
  if (!tr) return;
  tr->iterations = it + 1;
  if (it >= tr->cap) return;
  if (tr->phase) tr->phase[it] = phase;
  if (tr->direction) tr->direction[it] = (int32_t)ctrl_host[kDecision];
  if (tr->frontier) tr->frontier[it] = ctrl_host[kNf];
  if (tr->edges) tr->edges[it] = ctrl_host[kMf];
  if (tr->features) {
    const float *f = reinterpret_cast<const float *>(ctrl_host + kFeat);
    for (int k = 0; k < 16; ++k) tr->features[16 * it + k] = f[k];
  }
}

static int pull_available(gi_graph *g, int32_t dir) {
  if (dir == GI_DIR_DENSE_PULL && !g->has_csc) {
    set_error("DensePull needs the in-edges: load a symmetric graph or call gi_load_csc");
    return GI_ERR_UNSUPPORTED;
  }
  return GI_OK;
}

// Frontier loop shared by BFS / SSSP / CC: decide, stop when empty, traverse.
template <class Step>
static int frontier_loop(gi_graph *g, VsetPair &P, const gi_schedule &sc, bool track_unvisited, gi_trace *tr,
                         cudaStream_t s, Step step, bool pull_ok = true) {
  for (int32_t it = 0;; ++it) {
    DecideParams p = decide_params(sc, it, track_unvisited);
    GI_TRY(frontier_decide(g, P.F, p, s));
    GI_TRY(ctrl_fetch(g, s));
    if (g->ctrl_host[kNf] == 0) {
      if (tr) tr->iterations = it;
      break;
    }
    int32_t dir = (int32_t)g->ctrl_host[kDecision];
    if (dir == GI_DIR_DENSE_PULL && (!g->has_csc || !pull_ok)) dir = GI_DIR_DENSE_PUSH;
    g->ctrl_host[kDecision] = dir;
    trace_put(tr, it, g->ctrl_host);
    g->hint_vset = P.F;
    g->hint_nf = g->ctrl_host[kNf];
    g->hint_mf = g->ctrl_host[kMf];
    const int r = step(it, dir);
    g->hint_vset = nullptr;
    g->hint_nf = -1;
    g->hint_mf = -1;
    GI_TRY(r);
    P.swap();
  }
  return GI_OK;
}

}  // namespace gi

using namespace gi;

// Single query in the batched engine's whole-GPU persistent mode (BFS parents
// from the engine too when parent is non-NULL).
static int run_persistent(gi_graph *g, int32_t algo, int32_t src, int32_t *out, const gi_schedule &sc,
                          gi_trace *trace, cudaStream_t s, int32_t *parent = nullptr) {
  gi_batch_opts o;
  gi_batch_opts_default(&o);
  o.cluster_size = 0;
  o.selector = sc.direction == GI_DIR_LEARNED
                   ? GI_DIR_LEARNED
                   : ((sc.direction == GI_DIR_SPARSE_PUSH || sc.direction == GI_DIR_DENSE_PUSH || !g->has_csc)
                          ? GI_DIR_SPARSE_PUSH
                          : GI_DIR_HYBRID_PULL);
  o.alpha = sc.alpha > 0 ? sc.alpha : 14.0f;
  o.beta = sc.beta > 0 ? sc.beta : 24.0f;
  gi_graph *gs[1] = {g};
  int32_t *outs[1] = {out};
  int32_t *pars[1] = {parent};
  if (parent) o.parents = pars;
  const int32_t qg = 0, qs = src, qa = algo;
  gi_batch_plan *p = nullptr;
  GI_TRY(gi_batch_plan_create(gs, 1, &qg, &qs, &qa, 1, outs, &o, s, &p));
  int32_t levels = 0;
  int st = gi_batch_plan_launch(p, s);
  if (st == GI_OK) st = gi_batch_plan_results(p, nullptr, &levels, s);
  const int st2 = gi_batch_plan_free(p);
  if (trace) trace->iterations = levels;
  return st != GI_OK ? st : st2;
}

// ========================================================= graph-driven BFS ==
// gi_schedule.persistent = 2: the level loop runs on the device as a CUDA
// graph.  One WHILE node repeats a body of two levels (the frontier sets
// alternate roles); each level is the statistics + direction kernel, which
// empties the next frontier, writes the level's control words and sets the
// loop condition, then the push (with the all-block expansion of deferred
// sources) and the early-exit pull, each a no-op unless the level uses it.
// No host round trip per level.
// The graph is built once per graph and schedule; depths go to an internal
// buffer that is copied out after the launch.
namespace gi {

struct OpBFSDev {  // BFS claim with the level read from the control words; canonical parent as OpBFS
  int32_t *depth;
  int32_t *parent;
  const int32_t *gm;
  __device__ bool push(int32_t u, int32_t v, int32_t) const {
    const int32_t lvl = gm[kGmLevel] + 1;
    const int32_t d = *(volatile int32_t *)(depth + v);
    if (d != -1 && d != lvl) return false;
    bool won = false;
    if (d == -1) {
      const int32_t old = atomicCAS(depth + v, -1, lvl);
      won = (old == -1);
      if (!won && old != lvl) return false;
    }
    if (u < *(volatile int32_t *)(parent + v)) atomicMin(parent + v, u);
    return won;
  }
};

struct GraphLoop {
  gi_schedule sc{};
  int use_selector = -1;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int32_t *depth = nullptr;
  int32_t *parent = nullptr;  // canonical parents, INT32_MAX until found
  int32_t *gm = nullptr;
  BfsUnv unv;  // compacted unvisited walk of the pull levels (st == nullptr: off)
  gi_vset a, b;
};

__global__ void k_gm_init(int32_t *gm, int32_t cap) {
  if (threadIdx.x < kGmWords) gm[threadIdx.x] = threadIdx.x == kGmCap ? cap : 0;
}

void graph_loop_free(gi_graph *g) {
  GraphLoop *L = static_cast<GraphLoop *>(g->graph_loop);
  if (!L) return;
  if (L->exec) cudaGraphExecDestroy(L->exec);
  if (L->graph) cudaGraphDestroy(L->graph);
  for (gi_vset *v : {&L->a, &L->b}) {
    dev_free(v->queue, nullptr);
    dev_free(v->count, nullptr);
    dev_free(v->bitmap, nullptr);
    dev_free(v->boolmap, nullptr);
  }
  dev_free(L->depth, nullptr);
  dev_free(L->parent, nullptr);
  dev_free(L->gm, nullptr);
  delete L;
  g->graph_loop = nullptr;
}

// one level, F -> N, captured into the loop body: the statistics kernel
// (which also empties N and writes the level's control words), the push
// (queue length 0 unless this level pushes) and the early-exit pull (returns
// at once unless this level pulls).  Kernels that exit at once measured
// cheaper than IF nodes around them (grid 4096^2: 82 vs 103 ms per BFS).
static int graph_level(gi_graph *g, const gi_schedule &sc, GraphLoop *L, gi_vset *F, gi_vset *N,
                       cudaGraphConditionalHandle h, cudaStream_t cs) {
  DecideParams p = decide_params(sc, 0, true);
  p.gm = L->gm;
  p.cond_handle = (unsigned long long)h;
  p.clear_bm = N->bitmap;  // N holds the frontier of two levels before: its queue lists its bits
  p.clear_q = N->queue;
  p.clear_qc = N->count;
  GI_TRY(frontier_decide(g, F, p, cs));
  gi_vset Fp = *F;  // the push sees |F| only when this level pushes
  Fp.count = L->gm + kGmPush;
  const OpBFSDev op{L->depth, L->parent, L->gm};
  GI_TRY(launch_push(g, op, kSrcQueue, &Fp, nullptr, out_of(N, false), sc, cs));
  if (g->has_csc) {
    const int32_t tw = sc.balance == GI_BAL_VERTEX ? INT32_MAX : (sc.t_warp > 0 ? sc.t_warp : 32);
    k_pull_bfs<<<grid_for(g, g->n, 256), 256, 0, cs>>>(g->in.ptr, g->in.idx, g->n,
                                                      FSet(static_cast<const uint32_t *>(F->bitmap)), nullptr,
                                                      L->depth, L->parent, 0, tw, N->bitmap, N->queue, N->count,
                                                      L->gm, nullptr, 0, L->unv);
    GI_LAUNCH_CHECK();
  }
  N->reps = GI_REP_SPARSE | GI_REP_BITMAP;
  return GI_OK;
}

static int graph_loop_build(gi_graph *g, const gi_schedule &sc, GraphLoop *L, cudaStream_t s) {
  GI_TRY(heavy_get(g, s));
  if (sc.dst_list && g->has_csc) GI_TRY(bfs_unv_get(g, s, &L->unv));
  GI_TRY(dev_alloc_n(&L->depth, g->n, s));
  GI_TRY(dev_alloc_n(&L->parent, g->n, s));
  GI_TRY(dev_alloc_n(&L->gm, kGmWords, s));
  GI_TRY(vset_alloc(g, &L->a, s));
  GI_TRY(vset_alloc(g, &L->b, s));
  GI_CUDA(cudaStreamSynchronize(s));
  GI_CUDA(cudaGraphCreate(&L->graph, 0));
  cudaGraphConditionalHandle h;
  GI_CUDA(cudaGraphConditionalHandleCreate(&h, L->graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t loop;
  GI_CUDA(cudaGraphAddNode(&loop, L->graph, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  cudaStream_t cs;
  GI_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  int st = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) == cudaSuccess
               ? GI_OK
               : cuda_fail(cudaGetLastError(), "begin capture", __FILE__, __LINE__);
  L->a.reps = L->b.reps = GI_REP_SPARSE | GI_REP_BITMAP;
  if (st == GI_OK) st = graph_level(g, sc, L, &L->a, &L->b, h, cs);
  if (st == GI_OK) st = graph_level(g, sc, L, &L->b, &L->a, h, cs);
  cudaGraph_t captured = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(cs, &captured);
  cudaStreamDestroy(cs);
  if (st == GI_OK && ec != cudaSuccess) st = cuda_fail(ec, "end capture", __FILE__, __LINE__);
  if (st == GI_OK && cudaGraphInstantiate(&L->exec, L->graph, 0) != cudaSuccess)
    st = cuda_fail(cudaGetLastError(), "graph instantiate", __FILE__, __LINE__);
  return st;
}

// BFS depths (and canonical parents, parent may be NULL) by the graph-driven
// loop; levels = number of levels
// the graph's cached BFS loop for `sched`, built (or rebuilt) if needed
static int graph_loop_get(gi_graph *g, const gi_schedule &sched, cudaStream_t s, GraphLoop **out) {
  gi_schedule sc = sched;
  sc.balance = sc.balance == GI_BAL_EDGE_PARALLEL ? GI_BAL_EDGE_AWARE : sc.balance;  // needs a host-known |F|
  if (!g->has_csc) sc.direction = GI_DIR_SPARSE_PUSH;
  const int use_sel = selector_loaded() ? 1 : 0;
  GraphLoop *L = static_cast<GraphLoop *>(g->graph_loop);
  if (L && (std::memcmp(&L->sc, &sc, sizeof(sc)) != 0 || L->use_selector != use_sel)) {
    graph_loop_free(g);
    L = nullptr;
  }
  if (!L) {
    L = new GraphLoop();
    L->sc = sc;
    L->use_selector = use_sel;
    g->graph_loop = L;
    const int st = graph_loop_build(g, sc, L, s);
    if (st != GI_OK) {
      graph_loop_free(g);
      return st;
    }
  }
  *out = L;
  return GI_OK;
}

static int run_graph_bfs(gi_graph *g, int32_t src, int32_t *depth, int32_t *parent, const gi_schedule &sched,
                         int32_t *levels, cudaStream_t s) {
  GraphLoop *L = nullptr;
  GI_TRY(graph_loop_get(g, sched, s, &L));
  k_bfs_init<<<grid_for(g, g->n, 256), 256, 0, s>>>(L->depth, L->parent, g->n, src, L->unv.st);
  k_gm_init<<<1, 32, 0, s>>>(L->gm, (int32_t)(g->n + 1 < INT32_MAX ? g->n + 1 : INT32_MAX));
  GI_TRY(launch_status(2));
  GI_TRY(front_init(g, &L->a, src, s));
  GI_TRY(vset_clear(&L->b, s));  // the loop empties b through its queue from then on
  GI_TRY(ctrl_init(g, g->n, g->m, s));
  GI_CUDA(cudaGraphLaunch(L->exec, s));
  GI_CUDA(cudaMemcpyAsync(depth, L->depth, sizeof(int32_t) * (size_t)g->n, cudaMemcpyDeviceToDevice, s));
  if (parent) {
    k_parent_copy_fix<<<grid_for(g, g->n, 256), 256, 0, s>>>(parent, L->parent, g->n);
    GI_TRY(launch_status(1));
  }
  int32_t gm[kGmWords];
  GI_CUDA(cudaMemcpyAsync(gm, L->gm, sizeof(gm), cudaMemcpyDeviceToHost, s));
  GI_CUDA(cudaStreamSynchronize(s));
  if (gm[kGmErr]) {
    set_error("graph-driven BFS reached its level cap");
    return GI_ERR_TIMEOUT;
  }
  *levels = gm[kGmNext];
  return GI_OK;
}

}  // namespace gi

// ===================================================================== BFS ==
extern "C" int gi_bfs(gi_graph *g, int32_t src, int32_t *depth, int32_t *parent, const gi_schedule *sched,
                      gi_trace *trace, void *stream) {
  GI_ARG(g != nullptr, "graph is NULL");
  GI_TRY(check_schedule(sched));
  GI_ARG(src >= 0 && src < g->n, "source out of range");
  GI_ARG(depth != nullptr, "depth is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const gi_schedule sc = *sched;
  if (forced_direction(sc.direction) >= 0) GI_TRY(pull_available(g, forced_direction(sc.direction)));
  if (sc.persistent == 2) {
    // the graph-driven loop keeps depths and canonical parents itself
    int32_t levels = 0;
    GI_TRY(run_graph_bfs(g, src, depth, parent, sc, &levels, s));
    if (trace) trace->iterations = levels;
    return GI_OK;
  }
  if (sc.persistent == 1) {
    // depths and canonical parents in one persistent launch of the batched engine
    return run_persistent(g, GI_ALGO_BFS, src, depth, sc, trace, s, parent);
  }
  GI_TRY(ensure_tiles(g, sc, s));
  BfsUnv U;
  if (sc.dst_list && g->has_csc) GI_TRY(bfs_unv_get(g, s, &U));
  VsetPair P;
  int st = pair_alloc(g, P, s);
  if (st == GI_OK) {
    k_bfs_init<<<grid_for(g, g->n, 256), 256, 0, s>>>(depth, parent, g->n, src, U.st);
    st = launch_status(1);
  }
  g->bfs_unv_query = U;  // this query's pull levels walk the compacted list
  if (st == GI_OK) st = front_init(g, P.F, src, s);
  if (st == GI_OK) st = ctrl_init(g, g->n, g->m, s);
  if (st == GI_OK)
    st = frontier_loop(g, P, sc, true, trace, s, [&](int32_t it, int32_t dir) {
      // the canonical parent in every direction: pull levels stop at the
      // first (smallest-id) frontier in-neighbour; push levels lower parent[v]
      // with atomicMin from every frontier in-neighbour of a vertex found at
      // this level (after a plain read shows the id is smaller).  A pass over
      // the in-edges after the loop instead scanned hub rows serially for
      // their parent (R-MAT 24: 6.8 ms per query against < 0.1 ms here).
      gi_bfs_args a{depth, parent, it + 1};
      return apply_dispatch(g, P.F, nullptr, dir, sc, GI_K_BFS, &a, P.N, GI_NO_DEDUP, s);
    });
  g->bfs_unv_query = BfsUnv{};
  if (st == GI_OK && parent) {
    k_parent_fix<<<grid_for(g, g->n, 256), 256, 0, s>>>(parent, g->n);
    st = launch_status(1);
  }
  pair_free(P, s);
  if (st == GI_OK && cudaStreamSynchronize(s) != cudaSuccess)
    st = cuda_fail(cudaGetLastError(), "bfs", __FILE__, __LINE__);
  return st;
}

// =========================================================== SSSP and CC ==
// Synchronous rounds on x[] (dist or label): snap[] holds the start-of-round
// value of frontier members (INT32_MAX elsewhere) and is what every source
// reads, so push and pull rounds compute the same thing.
static int minlabel_run(gi_graph *g, int32_t *x, int32_t kernel_id, int32_t src, const gi_schedule &sc,
                        gi_trace *trace, cudaStream_t s) {
  GI_TRY(ensure_tiles(g, sc, s));
  VsetPair P;
  int32_t *snap = nullptr, *seg_acc = nullptr;
  int st = pair_alloc(g, P, s);
  if (st == GI_OK) st = dev_alloc_n(&snap, g->n, s);
  if (st == GI_OK && sc.num_segments > 1 && g->has_csc) {
    if (g->segs.num != sc.num_segments || g->segs.strategy != sc.seg_strategy)
      st = gi_graph_build_segments(g, sc.num_segments, sc.seg_strategy, s);
    if (st == GI_OK) st = dev_alloc_n(&seg_acc, g->n, s);
    if (st == GI_OK) {
      k_fill_i32<<<grid_for(g, g->n, 256), 256, 0, s>>>(seg_acc, g->n, INT32_MAX);
      st = launch_status(1);
    }
  }
  if (st == GI_OK) {
    if (kernel_id == GI_K_CC) {
      k_iota2<<<grid_for(g, g->n, 256), 256, 0, s>>>(x, snap, g->n);
    } else {
      k_fill_i32<<<grid_for(g, g->n, 256), 256, 0, s>>>(x, g->n, INT32_MAX);
      k_fill_i32<<<grid_for(g, g->n, 256), 256, 0, s>>>(snap, g->n, INT32_MAX);
      k_set_one<<<1, 1, 0, s>>>(x, src, 0);
      k_set_one<<<1, 1, 0, s>>>(snap, src, 0);
    }
    st = launch_status(kernel_id == GI_K_CC ? 1 : 4);
  }
  if (st == GI_OK) st = front_init(g, P.F, kernel_id == GI_K_CC ? -1 : src, s);
  if (st == GI_OK) st = ctrl_init(g, 0, 0, s);
  if (st == GI_OK)
    st = frontier_loop(g, P, sc, false, trace, s, [&](int32_t, int32_t dir) -> int {
      int r;
      if (dir == GI_DIR_DENSE_PULL && seg_acc) {
        // cache-partitioned pull: one source segment at a time folds its
        // minimum into seg_acc (no atomics: each destination row belongs to
        // one tile), then one vertex pass applies and marks
        GI_TRY(vset_clear(P.N, s));
        for (int sid = 0; sid < g->segs.num; ++sid) {
          OpMinInt op{seg_acc, snap, kernel_id == GI_K_CC ? nullptr : g->segs.seg[sid].wt};
          GI_TRY(launch_pull_tiled(g, op, g->segs.seg[sid], g->segs.tiles[sid], nullptr, nullptr, OutSet(), s,
                                   kClassMinPull));
        }
        k_min_apply<<<grid_for(g, g->n, 256), 256, 0, s>>>(x, seg_acc, g->n, P.N->bitmap, P.N->queue, P.N->count);
        r = launch_status(1);
        P.N->reps = GI_REP_SPARSE | GI_REP_BITMAP;
      } else if (dir == GI_DIR_DENSE_PULL) {
        // snap holds INT32_MAX outside the frontier, so the pull needs no
        // frontier test: a non-member contributes the identity of min
        GI_TRY(vset_clear(P.N, s));
        OpMinInt op{x, snap, kernel_id == GI_K_CC ? nullptr : g->in.wt};
        r = launch_pull_tiled(g, op, g->in, g->in_tiles, nullptr, nullptr, out_of(P.N), s, kClassMinPull,
                              sc.balance == GI_BAL_VERTEX, sc.hot_cache);
        P.N->reps = GI_REP_SPARSE | GI_REP_BITMAP;
      } else if (kernel_id == GI_K_CC) {
        gi_cc_args a{x, snap};
        r = apply_dispatch(g, P.F, nullptr, dir, sc, GI_K_CC, &a, P.N, 0, s);
      } else {
        gi_sssp_args a{x, snap};
        r = apply_dispatch(g, P.F, nullptr, dir, sc, GI_K_SSSP, &a, P.N, 0, s);
      }
      if (r != GI_OK) return r;
      int grid = g->num_sms * 4;
      k_snap_reset<<<grid, 256, 0, s>>>(P.F->queue, P.F->count, snap);
      k_snap_set<<<grid, 256, 0, s>>>(P.N->queue, P.N->count, snap, x);
      return launch_status(2);
    }, /*pull_ok=*/kernel_id == GI_K_CC || g->symmetric || g->in.wt != nullptr);
  dev_free(snap, s);
  dev_free(seg_acc, s);
  pair_free(P, s);
  if (st == GI_OK && cudaStreamSynchronize(s) != cudaSuccess)
    st = cuda_fail(cudaGetLastError(), "minlabel", __FILE__, __LINE__);
  return st;
}

// ========================================================= delta-stepping ==
// gi_schedule.delta > 0: SSSP by delta-stepping (Meyer & Sanders) in
// synchronous rounds, an ordering of the same label-correcting relaxations
// that Sec. 6's asyncMin leaves free (the final distances do not depend on
// it).  Arcs lighter than delta ("light") are relaxed inside the bucket
// [k*delta, (k+1)*delta) until it stops changing; the bucket's vertices are
// then final and their heavy arcs are relaxed once.  Each row's arcs are split
// by class into two CSRs, built once per graph and delta, so a round streams
// only the arcs it relaxes.  Every round is a SparsePush over the round's
// sources or a DensePull whose per-source values are the start-of-round
// distances of those sources (INT32_MAX elsewhere); on symmetric graphs the
// light and heavy CSRs are also their own in-edge views, so both directions
// relax exactly the same arcs and leave the same state.
namespace gi {

struct DeltaSplit {
  int32_t delta = 0;
  int32_t tile_edges = 0;
  Csr light, heavy;  // same vertices, arcs split by w < delta
  bool light_alias = false;  // every arc is light: light is the graph's own CSR (not owned)
  int32_t *deg_l = nullptr, *deg_h = nullptr;
  // The pulls' views (symmetric graphs, block tiles): only the rows that have
  // arcs of the class (rows_l / rows_h; their offsets in light_c / heavy_c,
  // whose arcs are light's / heavy's), so a pull skips the empty rows; with
  // warp tiles they are light / heavy themselves (compacted false).
  bool compacted = false;
  Csr light_c, heavy_c;
  int32_t *rows_l = nullptr, *rows_h = nullptr;
  TileSet tl, th;    // pull tiles (symmetric graphs) over light_c / heavy_c
  int64_t m_light = 0;
  void *loop = nullptr;  // cached graph-driven loop over this split (DsLoop)
  // the CSR a pull of the class reads: the compacted view with the tiles, the
  // full rows for the vertex-parallel pull (one thread per vertex)
  const Csr &pull_csr(bool light_class, bool vertex_parallel) const {
    if (vertex_parallel || !compacted) return light_class ? light : heavy;
    return light_class ? light_c : heavy_c;
  }
};

static void dsloop_free(DeltaSplit *D);

void dstep_free(gi_graph *g, cudaStream_t s) {
  DeltaSplit *D = static_cast<DeltaSplit *>(g->dstep);
  if (!D) return;
  dsloop_free(D);
  if (D->light_alias) {  // the light arcs are the graph's own; only its row offsets are ours
    dev_free(D->light.ptr, s);
    D->light = Csr();
  }
  for (Csr *c : {&D->light, &D->heavy}) {
    dev_free(c->ptr, s);
    dev_free(c->idx, s);
    dev_free(c->wt, s);
  }
  dev_free(D->deg_l, s);
  dev_free(D->deg_h, s);
  if (D->compacted) {  // the compacted views own their offsets and row lists only
    dev_free(D->light_c.ptr, s);
    dev_free(D->heavy_c.ptr, s);
    dev_free(D->rows_l, s);
    dev_free(D->rows_h, s);
  }
  free_tiles(&D->tl, s);
  free_tiles(&D->th, s);
  delete D;
  g->dstep = nullptr;
}

__global__ void k_nonempty(const int32_t *__restrict__ deg, int64_t n, int32_t *flag) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    flag[v] = deg[v] > 0 ? 1 : 0;
}

// rows[pos[v]] = v and ptr_c[pos[v]] = ptr[v] for the rows with arcs; the
// closing offset ptr_c[k] = ptr[n] (k = pos[n], the scan's total)
__global__ void k_compact_rows(const int32_t *__restrict__ deg, const int32_t *__restrict__ pos,
                               const int32_t *__restrict__ ptr, int64_t n, int32_t *rows, int32_t *ptr_c) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += (int64_t)gridDim.x * blockDim.x) {
    if (v == n) {
      ptr_c[pos[n]] = ptr[n];
    } else if (deg[v] > 0) {
      rows[pos[v]] = (int32_t)v;
      ptr_c[pos[v]] = ptr[v];
    }
  }
}

// The row-compacted view of class c (degrees deg): its rows with arcs and
// their offsets, and block tiles over them.
static int compact_class(gi_graph *g, const Csr &c, const int32_t *deg, int32_t te, Csr *cc, int32_t **rows,
                         TileSet *ts, cudaStream_t s) {
  const int64_t n = g->n;
  int32_t *flag = nullptr, *pos = nullptr;
  GI_TRY(ws_scratch(g, &flag, &pos, s));
  k_nonempty<<<grid_for(g, n, 256), 256, 0, s>>>(deg, n, flag);
  GI_TRY(launch_status(1));
  GI_TRY(scan_exclusive(g, flag, pos, n, s));
  int32_t k = 0;
  GI_CUDA(cudaMemcpyAsync(&k, pos + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  GI_CUDA(cudaStreamSynchronize(s));
  GI_TRY(dev_alloc_n(rows, k, s));
  GI_TRY(dev_alloc_n(&cc->ptr, (int64_t)k + 1, s));
  cc->idx = c.idx;
  cc->wt = c.wt;
  k_compact_rows<<<grid_for(g, n + 1, 256), 256, 0, s>>>(deg, pos, c.ptr, n, *rows, cc->ptr);
  GI_TRY(launch_status(1));
  GI_TRY(build_tiles(g, *cc, te, ts, s, k));
  ts->rows = *rows;
  return GI_OK;
}

// Rows with more than kDsLongRow arcs are split by a whole block instead of
// one warp (a hub row of 10^5-10^6 arcs walked by one warp took tens of ms);
// the warp kernels queue them (long[0] = count, long[1..] = rows).
constexpr int64_t kDsLongRow = 4096;

// light arcs per row, one warp per row; long rows queued for k_ds_count_long
__global__ void k_ds_count(const int32_t *__restrict__ ptr, const int32_t *__restrict__ wt, int64_t n, int32_t delta,
                           int32_t *cnt, int32_t *longq) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
    const int64_t a = __ldg(ptr + v), b = __ldg(ptr + v + 1);
    if (b - a > kDsLongRow) {
      if (lane == 0) longq[1 + atomicAdd(longq, 1)] = (int32_t)v;
      continue;
    }
    int32_t c = 0;
    for (int64_t e = a + lane; e < b; e += 32) c += __ldg(wt + e) < delta ? 1 : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) cnt[v] = c;
  }
}

// the queued long rows' light arcs, one block (256 threads) per row
__global__ void __launch_bounds__(256) k_ds_count_long(const int32_t *__restrict__ ptr,
                                                       const int32_t *__restrict__ wt, int32_t delta,
                                                       const int32_t *__restrict__ longq, int32_t *cnt) {
  __shared__ int32_t s_c[8];
  const int32_t nl = longq[0];
  for (int32_t j = blockIdx.x; j < nl; j += gridDim.x) {
    const int32_t v = longq[1 + j];
    const int64_t a = __ldg(ptr + v), b = __ldg(ptr + v + 1);
    int32_t c = 0;
    for (int64_t e = a + threadIdx.x; e < b; e += 256) c += __ldg(wt + e) < delta ? 1 : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) s_c[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
      int32_t t = 0;
      for (int w = 0; w < 8; ++w) t += s_c[w];
      cnt[v] = t;
    }
    __syncthreads();
  }
}

// heavy row offsets and both degree arrays: hptr[v] = ptr[v] - lptr[v]
__global__ void k_ds_offsets(const int32_t *__restrict__ ptr, const int32_t *__restrict__ lptr, int64_t n,
                             int32_t *hptr, int32_t *deg_l, int32_t *deg_h) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += (int64_t)gridDim.x * blockDim.x) {
    hptr[v] = ptr[v] - lptr[v];
    if (v < n) {
      const int32_t dl = lptr[v + 1] - lptr[v];
      deg_l[v] = dl;
      deg_h[v] = (ptr[v + 1] - ptr[v]) - dl;
    }
  }
}

// stable split of each row (one warp per row): light arcs to the light CSR,
// the others to the heavy CSR, both keeping the row's ascending order
__global__ void k_ds_fill(const int32_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                          const int32_t *__restrict__ wt, int64_t n, int32_t delta, const int32_t *__restrict__ lptr,
                          const int32_t *__restrict__ hptr, int32_t *lidx, int32_t *lwt, int32_t *hidx, int32_t *hwt) {
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
    const int64_t a = __ldg(ptr + v), b = __ldg(ptr + v + 1);
    if (b - a > kDsLongRow) continue;  // k_ds_fill_long
    int64_t lo = __ldg(lptr + v), ho = __ldg(hptr + v);
    for (int64_t e0 = a; e0 < b; e0 += 32) {
      const int64_t e = e0 + lane;
      const bool ok = e < b;
      const int32_t w = ok ? __ldg(wt + e) : 0, u = ok ? __ldg(idx + e) : 0;
      const bool li = ok && w < delta, hv = ok && !li;
      const unsigned bl = __ballot_sync(0xffffffffu, li), bh = __ballot_sync(0xffffffffu, hv);
      if (li) {
        const int64_t p = lo + __popc(bl & below);
        lidx[p] = u;
        lwt[p] = w;
      }
      if (hv) {
        const int64_t p = ho + __popc(bh & below);
        hidx[p] = u;
        hwt[p] = w;
      }
      lo += __popc(bl);
      ho += __popc(bh);
    }
  }
}

// the queued long rows' stable split, one block (256 threads) per row: each
// 256-arc chunk is placed by a block-wide prefix of its light (heavy) flags,
// chunks in order
__global__ void __launch_bounds__(256) k_ds_fill_long(const int32_t *__restrict__ ptr,
                                                      const int32_t *__restrict__ idx,
                                                      const int32_t *__restrict__ wt, int32_t delta,
                                                      const int32_t *__restrict__ lptr,
                                                      const int32_t *__restrict__ hptr,
                                                      const int32_t *__restrict__ longq, int32_t *lidx, int32_t *lwt,
                                                      int32_t *hidx, int32_t *hwt) {
  __shared__ int32_t s_l[8], s_h[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned below = (1u << lane) - 1u;
  const int32_t nl = longq[0];
  for (int32_t j = blockIdx.x; j < nl; j += gridDim.x) {
    const int32_t v = longq[1 + j];
    const int64_t a = __ldg(ptr + v), b = __ldg(ptr + v + 1);
    int64_t lo = __ldg(lptr + v), ho = __ldg(hptr + v);
    for (int64_t e0 = a; e0 < b; e0 += 256) {
      const int64_t e = e0 + threadIdx.x;
      const bool ok = e < b;
      const int32_t w = ok ? __ldg(wt + e) : 0, u = ok ? __ldg(idx + e) : 0;
      const bool li = ok && w < delta, hv = ok && !li;
      const unsigned bl = __ballot_sync(0xffffffffu, li), bh = __ballot_sync(0xffffffffu, hv);
      if (lane == 0) {
        s_l[warp] = __popc(bl);
        s_h[warp] = __popc(bh);
      }
      __syncthreads();
      int32_t pl = 0, ph = 0, tl = 0, th = 0;
      for (int k = 0; k < 8; ++k) {
        if (k < warp) {
          pl += s_l[k];
          ph += s_h[k];
        }
        tl += s_l[k];
        th += s_h[k];
      }
      if (li) {
        const int64_t p = lo + pl + __popc(bl & below);
        lidx[p] = u;
        lwt[p] = w;
      }
      if (hv) {
        const int64_t p = ho + ph + __popc(bh & below);
        hidx[p] = u;
        hwt[p] = w;
      }
      lo += tl;
      ho += th;
      __syncthreads();
    }
  }
}

static int dstep_get(gi_graph *g, int32_t delta, int32_t tile_edges, cudaStream_t s, DeltaSplit **out) {
  DeltaSplit *D = static_cast<DeltaSplit *>(g->dstep);
  const int32_t te = tile_edges > 0 ? tile_edges : 2048;
  if (D && D->delta == delta && (!g->symmetric || D->tile_edges == te)) {
    *out = D;
    return GI_OK;
  }
  dstep_free(g, s);
  D = new DeltaSplit();
  g->dstep = D;
  D->delta = delta;
  D->tile_edges = te;
  const int64_t n = g->n;
  int st = dev_alloc_n(&D->light.ptr, n + 1, s);
  if (st == GI_OK) st = dev_alloc_n(&D->heavy.ptr, n + 1, s);
  if (st == GI_OK) st = dev_alloc_n(&D->deg_l, n, s);
  if (st == GI_OK) st = dev_alloc_n(&D->deg_h, n, s);
  const int wgrid = grid_for(g, n * 32, 256);
  int32_t *cnt = nullptr, *longq = nullptr;
  if (st == GI_OK) st = dev_alloc_n(&cnt, n, s);
  // at most m / kDsLongRow rows are long
  if (st == GI_OK) st = dev_alloc_n(&longq, 2 + g->m / kDsLongRow, s);
  if (st == GI_OK && cudaMemsetAsync(longq, 0, sizeof(int32_t), s) != cudaSuccess)
    st = cuda_fail(cudaGetLastError(), "long-row queue", __FILE__, __LINE__);
  if (st == GI_OK) {
    k_ds_count<<<wgrid, 256, 0, s>>>(g->out.ptr, g->out.wt, n, delta, cnt, longq);
    k_ds_count_long<<<g->num_sms * 8, 256, 0, s>>>(g->out.ptr, g->out.wt, delta, longq, cnt);
    st = launch_status(2);
  }
  if (st == GI_OK) st = scan_exclusive(g, cnt, D->light.ptr, n, s);
  dev_free(cnt, s);
  int32_t ml = 0;
  if (st == GI_OK) {
    k_ds_offsets<<<grid_for(g, n + 1, 256), 256, 0, s>>>(g->out.ptr, D->light.ptr, n, D->heavy.ptr, D->deg_l,
                                                          D->deg_h);
    st = launch_status(1);
  }
  if (st == GI_OK && (cudaMemcpyAsync(&ml, D->light.ptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s) !=
                          cudaSuccess ||
                      cudaStreamSynchronize(s) != cudaSuccess))
    st = cuda_fail(cudaGetLastError(), "light arc count", __FILE__, __LINE__);
  D->m_light = ml;
  const int64_t mh = g->m - ml;
  if (st == GI_OK && mh == 0) {
    // every arc is light (Bellman-Ford when delta exceeds every weight): the
    // light arcs are the graph's own arrays, no copy
    D->light_alias = true;
    D->light.idx = g->out.idx;
    D->light.wt = g->out.wt;
  } else {
    if (st == GI_OK) st = dev_alloc_n(&D->light.idx, ml, s);
    if (st == GI_OK) st = dev_alloc_n(&D->light.wt, ml, s);
    if (st == GI_OK) st = dev_alloc_n(&D->heavy.idx, mh, s);
    if (st == GI_OK) st = dev_alloc_n(&D->heavy.wt, mh, s);
    if (st == GI_OK) {
      k_ds_fill<<<wgrid, 256, 0, s>>>(g->out.ptr, g->out.idx, g->out.wt, n, delta, D->light.ptr, D->heavy.ptr,
                                      D->light.idx, D->light.wt, D->heavy.idx, D->heavy.wt);
      k_ds_fill_long<<<g->num_sms * 8, 256, 0, s>>>(g->out.ptr, g->out.idx, g->out.wt, delta, D->light.ptr,
                                                     D->heavy.ptr, longq, D->light.idx, D->light.wt, D->heavy.idx,
                                                     D->heavy.wt);
      st = launch_status(2);
    }
  }
  dev_free(longq, s);
  if (st == GI_OK && g->symmetric) {
    if (te != kWarpTileEdges) {
      D->compacted = true;
      st = compact_class(g, D->light, D->deg_l, te, &D->light_c, &D->rows_l, &D->tl, s);
      if (st == GI_OK) st = compact_class(g, D->heavy, D->deg_h, te, &D->heavy_c, &D->rows_h, &D->th, s);
    } else {
      st = build_tiles(g, D->light, te, &D->tl, s);
      if (st == GI_OK) st = build_tiles(g, D->heavy, te, &D->th, s);
    }
  }
  if (st != GI_OK) {
    dstep_free(g, s);
    return st;
  }
  *out = D;
  return GI_OK;
}

// Device words of delta-stepping (int32, in the graph's control block): the
// round's R and the bucket's S counts, the counts of the two far-pile
// buffers and the smallest distance in the far pile.
enum DsWord { kDsR = 0, kDsS = 1, kDsPile0 = 2, kDsPile1 = 3, kDsPileMin = 4, kDsHi = 5 };

__global__ void k_ds_round_init(int32_t *w) {
  if (threadIdx.x == 0) w[kDsR] = 0;
}

// Splits the vertices whose distance changed last round (P): those below hi
// form this round's R (snap = their distance), join the bucket's settled list
// S once and leave the far pile if they were in it; the rest join the far
// pile once and lower its recorded minimum.
// P holds each vertex once, so the S and pile membership flags (bucket
// number s_mark[v], byte pile_in[v]) are plain reads and writes.
__global__ void k_ds_split(const int32_t *__restrict__ P, const int32_t *__restrict__ Pc,
                           const int32_t *__restrict__ x, int32_t hi, int32_t *Rq, int32_t *snap, int32_t *s_mark,
                           int32_t epoch, int32_t *Sq, uint8_t *pile_in, int32_t *pile, int32_t *pile_count,
                           int32_t *w) {
  const int lane = threadIdx.x & 31;
  const int32_t c = *Pc;
  const int32_t stride = gridDim.x * blockDim.x;
  int32_t fmin = INT32_MAX;
  for (int32_t i0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < c; i0 += stride) {
    const int32_t i = i0 + lane;
    int32_t v = -1, d = INT32_MAX, sm = epoch;
    uint8_t pin = 0;
    if (i < c) {
      v = P[i];
      d = x[v];  // with the membership words, in one round trip
      sm = s_mark[v];
      pin = pile_in[v];
    }
    const bool near = v >= 0 && d < hi, far = v >= 0 && !near;
    bool snew = false, pnew = false;
    if (near) {
      snap[v] = d;
      if (pin) pile_in[v] = 0;  // its pile entry is now stale
      if (sm != epoch) {
        s_mark[v] = epoch;
        snew = true;
      }
    }
    if (far) {
      fmin = min(fmin, d);
      if (!pin) {
        pile_in[v] = 1;
        pnew = true;
      }
    }
    warp_append3(Rq, w + kDsR, near, Sq, w + kDsS, snew, pile, pile_count, pnew, v);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) fmin = min(fmin, __shfl_xor_sync(0xffffffffu, fmin, o));
  if (lane == 0 && fmin < INT32_MAX) atomicMin(w + kDsPileMin, fmin);
}

// Next bucket: the far pile's live entries (pile_in still set) below hi
// leave it for the pending set P (queue only; P is empty here and nothing
// reads its bitmap before it is cleared), the rest are compacted into the
// other pile buffer, whose minimum is recomputed.
__global__ void k_ds_pile_split(const int32_t *__restrict__ pile, const int32_t *__restrict__ pile_count,
                                const int32_t *__restrict__ x, int32_t hi, uint8_t *pile_in, int32_t *Pq,
                                int32_t *Pc, int32_t *pile2, int32_t *pile2_count, int32_t *w) {
  const int lane = threadIdx.x & 31;
  const int32_t c = *pile_count;
  const int32_t stride = gridDim.x * blockDim.x;
  int32_t fmin = INT32_MAX;
  for (int32_t i0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < c; i0 += stride) {
    const int32_t i = i0 + lane;
    int32_t v = -1, d = INT32_MAX;
    if (i < c) {
      v = pile[i];
      const uint8_t pin = pile_in[v];
      const int32_t dv = x[v];  // loaded with the flag, one round trip
      if (!pin) v = -1;  // left the pile after it was queued
      else d = dv;
    }
    const bool near = v >= 0 && d < hi, far = v >= 0 && !near;
    if (near) pile_in[v] = 0;
    if (far) fmin = min(fmin, d);
    warp_append3(Pq, Pc, near, pile2, pile2_count, far, nullptr, nullptr, false, v);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) fmin = min(fmin, __shfl_xor_sync(0xffffffffu, fmin, o));
  if (lane == 0 && fmin < INT32_MAX) atomicMin(w + kDsPileMin, fmin);
}

// before a pile split: the target buffer empty, its minimum to be recomputed
// a new bucket ending at hi: the next pile buffer emptied, its minimum reset
__global__ void k_ds_pile_prep(int32_t *w, int32_t target, int32_t hi) {
  if (threadIdx.x == 0) {
    w[target] = 0;
    w[kDsPileMin] = INT32_MAX;
    w[kDsHi] = hi;
  }
}

__global__ void k_ds_zero_s(int32_t *w) {
  if (threadIdx.x == 0) w[kDsS] = 0;
}

}  // namespace gi

// Per-round timing of both directions from the same state (selector training
// data, gi_selector_profile): for round i < cap, features[16 i..] and
// times_ms[3 i..] = {SparsePush, -1 (DensePush is not offered), DensePull}.
struct DsProfile {
  int32_t cap = 0;
  float *features = nullptr;
  float *times_ms = nullptr;
  int32_t rounds = 0;
};

// Host loop of delta-stepping.  Each round: split the changed vertices into
// this bucket's R and the far pile (one kernel), statistics and direction for
// R (one kernel and one host read-back), then the light relaxation of R.  When
// R is empty the bucket's settled list S gets its heavy round; when S is empty
// too, the far pile's entries of the next non-empty bucket become the pending
// set.  Far vertices wait in the pile instead of being re-read every round.
static int deltastep_run(gi_graph *g, int32_t *x, int32_t src, const gi_schedule &sc, gi_trace *trace,
                         cudaStream_t s, DsProfile *prof = nullptr) {
  DeltaSplit *D = nullptr;
  GI_TRY(dstep_get(g, sc.delta, sc.tile_edges, s, &D));
  const int64_t n = g->n;
  const bool pull_ok = g->symmetric;
  VsetPair P;
  gi_vset R{}, S{};
  int32_t *snap = nullptr, *Rq = nullptr, *Sq = nullptr, *pile[2] = {nullptr, nullptr}, *s_mark = nullptr;
  uint8_t *pile_in = nullptr;
  int32_t epoch = 0;  // bucket number
  // the words live in the graph's control block, so the fetch of the
  // statistics brings them to the host in the same pinned copy
  int32_t *w = reinterpret_cast<int32_t *>(g->ctrl + kDsSlots);
  const int32_t *hw = reinterpret_cast<const int32_t *>(g->ctrl_host + kDsSlots);
  int st = pair_alloc(g, P, s);
  if (st == GI_OK) st = dev_alloc_n(&snap, n, s);
  if (st == GI_OK) st = dev_alloc_n(&Rq, n, s);
  if (st == GI_OK) st = dev_alloc_n(&Sq, n, s);
  if (st == GI_OK) st = dev_alloc_n(&pile[0], n, s);
  if (st == GI_OK) st = dev_alloc_n(&pile[1], n, s);
  if (st == GI_OK) st = dev_alloc_n(&s_mark, n, s);
  if (st == GI_OK) st = dev_alloc_n(&pile_in, n, s);
  int32_t *prof_keep = nullptr;
  cudaEvent_t prof_ev[2] = {nullptr, nullptr};
  if (prof) {
    if (st == GI_OK) st = dev_alloc_n(&prof_keep, n, s);
    if (st == GI_OK && (cudaEventCreate(&prof_ev[0]) != cudaSuccess || cudaEventCreate(&prof_ev[1]) != cudaSuccess))
      st = cuda_fail(cudaGetLastError(), "event create", __FILE__, __LINE__);
  }
  if (st == GI_OK) {
    k_fill_i32<<<grid_for(g, n, 256), 256, 0, s>>>(x, n, INT32_MAX);
    k_fill_i32<<<grid_for(g, n, 256), 256, 0, s>>>(snap, n, INT32_MAX);
    k_fill_i32<<<grid_for(g, n, 256), 256, 0, s>>>(s_mark, n, -1);
    k_set_one<<<1, 1, 0, s>>>(x, src, 0);
    st = launch_status(4);
  }
  if (st == GI_OK && cudaMemsetAsync(pile_in, 0, (size_t)(n > 0 ? n : 1), s) != cudaSuccess)
    st = cuda_fail(cudaGetLastError(), "delta-stepping init", __FILE__, __LINE__);
  if (st == GI_OK) st = front_init(g, P.F, src, s);
  if (st == GI_OK) st = ctrl_init(g, 0, 0, s);  // also zeroes the words
  if (st == GI_OK) {
    // pile minimum = INT32_MAX, first bucket [0, delta)
    k_ds_pile_prep<<<1, 32, 0, s>>>(w, kDsPile0, sc.delta);
    st = launch_status(1);
  }
  // R and S are vertex sets with the queue form only; their counters are words
  R.g = S.g = g;
  R.n = S.n = n;
  R.queue = Rq;
  R.count = w + kDsR;
  R.reps = GI_REP_SPARSE;
  S.queue = Sq;
  S.count = w + kDsS;
  S.reps = GI_REP_SPARSE;
  int64_t hi = sc.delta;  // end of the current bucket (distance of src = 0)
  int cur = 0;            // far-pile buffer in use
  const int grid = g->num_sms * 8;
  int32_t it = 0;
  while (st == GI_OK) {
    k_ds_round_init<<<1, 32, 0, s>>>(w);
    k_ds_split<<<g->num_sms * 8, 256, 0, s>>>(P.F->queue, P.F->count, x, (int32_t)(hi < INT32_MAX ? hi : INT32_MAX),
                                              Rq, snap, s_mark, epoch, Sq, pile_in, pile[cur], w + kDsPile0 + cur, w);
    if ((st = launch_status(2)) != GI_OK) break;
    DecideParams p = decide_params(sc, it, false);
    if ((st = frontier_decide(g, &R, p, s, D->deg_l)) != GI_OK) break;
    if ((st = ctrl_fetch(g, s)) != GI_OK) break;
    const bool light = hw[kDsR] > 0;
    if (!light && hw[kDsS] == 0) {
      if (hw[kDsPile0 + cur] == 0) break;  // nothing pending: done
      // the bucket is finished and its heavy arcs relaxed: the far pile's
      // entries of the next bucket become the pending set
      hi = ((int64_t)hw[kDsPileMin] / sc.delta + 1) * sc.delta;
      if ((st = vset_clear(P.F, s)) != GI_OK) break;
      k_ds_pile_prep<<<1, 32, 0, s>>>(w, kDsPile0 + (cur ^ 1), (int32_t)(hi < INT32_MAX ? hi : INT32_MAX));
      k_ds_pile_split<<<grid, 256, 0, s>>>(pile[cur], w + kDsPile0 + cur, x, (int32_t)(hi < INT32_MAX ? hi : INT32_MAX),
                                           pile_in, P.F->queue, P.F->count, pile[cur ^ 1], w + kDsPile0 + (cur ^ 1),
                                           w);
      if ((st = launch_status(2)) != GI_OK) break;
      P.F->reps = GI_REP_SPARSE | GI_REP_BITMAP;
      cur ^= 1;
      continue;
    }
    gi_vset *Fr = light ? &R : &S;
    const Csr &arcs = light ? D->light : D->heavy;
    if (!light) {
      // heavy round of the finished bucket: its vertices are final
      k_snap_set<<<grid, 256, 0, s>>>(Sq, S.count, snap, x);
      if ((st = launch_status(1)) != GI_OK) break;
      if ((st = frontier_decide(g, &S, p, s, D->deg_h)) != GI_OK) break;
      if ((st = ctrl_fetch(g, s)) != GI_OK) break;
    }
    int32_t dir = (int32_t)g->ctrl_host[kDecision];
    if (dir == GI_DIR_DENSE_PUSH || (dir == GI_DIR_DENSE_PULL && !pull_ok)) dir = GI_DIR_SPARSE_PUSH;
    g->ctrl_host[kDecision] = dir;
    const int64_t nf = g->ctrl_host[kNf], mf = g->ctrl_host[kMf];
    // a heavy round without heavy arcs only empties S: not a relaxation round
    const bool counted = light || mf > 0;
    if (counted) trace_put(trace, it, g->ctrl_host, light ? 0 : 1);
    auto relax = [&](int32_t d) -> int {
      GI_TRY(vset_clear(P.N, s));
      if (mf == 0) return GI_OK;
      OpMinInt op{x, snap, arcs.wt};
      if (d == GI_DIR_DENSE_PULL) {
        const Csr &pc = D->pull_csr(light, sc.balance == GI_BAL_VERTEX);
        const bool vp = sc.balance == GI_BAL_VERTEX;
        if (light)
          return launch_pull_tiled(g, op, pc, D->tl, FSet(), nullptr, out_of(P.N), s, kClassMinPull, vp);
        // heavy round: rows at or below the bucket's end are not pulled
        const OpMinIntBounded opb{op, w + kDsHi, 0};
        return launch_pull_tiled(g, opb, pc, D->th, FSet(), nullptr, out_of(P.N), s, kClassMinPull, vp);
      }
      g->hint_vset = Fr;
      g->hint_nf = nf;
      g->hint_mf = mf;
      const int r = launch_push(g, op, kSrcQueue, Fr, nullptr, out_of(P.N), sc, s, &arcs);
      g->hint_vset = nullptr;
      g->hint_nf = g->hint_mf = -1;
      return r;
    };
    if (prof && counted && pull_ok && prof->rounds < prof->cap) {
      // both directions from the same state, timed; the pull's result stays
      const float *f = reinterpret_cast<const float *>(g->ctrl_host + kFeat);
      for (int k = 0; k < 16; ++k) prof->features[16 * prof->rounds + k] = f[k];
      float *t3 = prof->times_ms + 3 * prof->rounds;
      t3[1] = -1.0f;
      const int32_t dirs[2] = {GI_DIR_SPARSE_PUSH, GI_DIR_DENSE_PULL};
      for (int k = 0; k < 2 && st == GI_OK; ++k) {
        if (k == 0 && cudaMemcpyAsync(prof_keep, x, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s) !=
                          cudaSuccess)
          st = cuda_fail(cudaGetLastError(), "snapshot", __FILE__, __LINE__);
        if (k > 0 && cudaMemcpyAsync(x, prof_keep, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s) !=
                         cudaSuccess)
          st = cuda_fail(cudaGetLastError(), "restore", __FILE__, __LINE__);
        if (st != GI_OK) break;
        cudaEventRecord(prof_ev[0], s);
        st = relax(dirs[k]);
        cudaEventRecord(prof_ev[1], s);
        if (st == GI_OK && cudaEventSynchronize(prof_ev[1]) != cudaSuccess)
          st = cuda_fail(cudaGetLastError(), "profile sync", __FILE__, __LINE__);
        float ms = 0.0f;
        if (st == GI_OK) cudaEventElapsedTime(&ms, prof_ev[0], prof_ev[1]);
        t3[k == 0 ? 0 : 2] = ms;
      }
      ++prof->rounds;
    } else {
      st = relax(dir);
    }
    if (st != GI_OK) break;
    k_snap_reset<<<grid, 256, 0, s>>>(Fr->queue, Fr->count, snap);
    int launched = 1;
    if (!light) {  // the bucket's settled list is done with
      k_ds_zero_s<<<1, 32, 0, s>>>(w);
      ++epoch;
      launched += 1;
    }
    if ((st = launch_status(launched)) != GI_OK) break;
    P.N->reps = GI_REP_SPARSE | GI_REP_BITMAP;
    P.swap();
    if (counted) ++it;
  }
  if (trace) trace->iterations = it;
  if (prof_ev[0]) cudaEventDestroy(prof_ev[0]);
  if (prof_ev[1]) cudaEventDestroy(prof_ev[1]);
  dev_free(prof_keep, s);
  dev_free(snap, s);
  dev_free(Rq, s);
  dev_free(Sq, s);
  dev_free(pile[0], s);
  dev_free(pile[1], s);
  dev_free(s_mark, s);
  dev_free(pile_in, s);
  pair_free(P, s);
  if (st == GI_OK && cudaStreamSynchronize(s) != cudaSuccess)
    st = cuda_fail(cudaGetLastError(), "delta-stepping", __FILE__, __LINE__);
  return st;
}

// ================================================== graph-driven SSSP ==
// gi_sssp with gi_schedule.persistent = 2: the delta-stepping rounds run as a
// CUDA graph, a WHILE node whose body holds two rounds (the pending sets a and
// b swap roles).  Each round is one kernel that splits the changed vertices
// into R, S and the far pile, empties their set and decides the round
// (statistics of R or S, direction, mode), then a SWITCH node that runs only
// the round's relaxation (light or heavy arcs, push or pull) or the far
// pile's next bucket.  No host round trip per round.
// The snapshots (snap for R, snap_h for S) are not reset after a round: an
// entry, once set, equals its vertex's distance at the last split (a vertex
// whose distance drops is pending at the next split, is near and gets a new
// entry), and its arcs of that class were relaxed from that value in the
// round that set it (light) or in its bucket's heavy round (heavy).  A pull
// that reads such an entry again improves nothing, so every round changes
// exactly the vertices it changes with the entries reset, push or pull.
// Bellman-Ford (delta = 0) is the same loop with one bucket holding every
// arc (delta beyond every weight), which gives its synchronous rounds exactly.
namespace gi {

// next bucket: live pile entries below hi -> the pending set N (cleared
// before), the rest -> the pile buffer in use from now on (kDgCur, which the
// split kernel has just switched; its count was zeroed there) with a fresh
// minimum
__global__ void k_dsg_pile_split(const int32_t *__restrict__ x, int32_t *dw, uint8_t *pile_in, int32_t *pile0,
                                 int32_t *pile1, int32_t *Nq, int32_t *Nc) {
  const int lane = threadIdx.x & 31;
  const int32_t cur = dw[kDgCur] ^ 1, hi = dw[kDgHi];  // cur: the buffer being thinned
  const int32_t *pile = cur ? pile1 : pile0;
  int32_t *pile2 = cur ? pile0 : pile1;
  const int32_t c = dw[kDgPile0 + cur];
  const int32_t stride = gridDim.x * blockDim.x;
  int32_t fmin = INT32_MAX;
  for (int32_t i0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < c; i0 += stride) {
    const int32_t i = i0 + lane;
    int32_t v = -1, d = INT32_MAX;
    if (i < c) {
      v = pile[i];
      const uint8_t pin = pile_in[v];
      const int32_t dv = x[v];  // loaded with the flag, one round trip
      if (!pin) v = -1;  // left the pile after it was queued
      else d = dv;
    }
    const bool near = v >= 0 && d < hi, far = v >= 0 && !near;
    if (near) pile_in[v] = 0;
    if (far) fmin = min(fmin, d);
    warp_append3(Nq, Nc, near, pile2, dw + kDgPile0 + (cur ^ 1), far, nullptr, nullptr, false, v);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) fmin = min(fmin, __shfl_xor_sync(0xffffffffu, fmin, o));
  if (lane == 0 && fmin < INT32_MAX) atomicMin(dw + kDgPmin, fmin);
}

__global__ void k_dsg_init(int32_t *dw, int32_t delta, int32_t cap) {
  if (threadIdx.x < kDgWords) {
    int32_t v = 0;
    if (threadIdx.x == kDgHi) v = delta;
    if (threadIdx.x == kDgPmin) v = INT32_MAX;
    if (threadIdx.x == kDgCap) v = cap;
    dw[threadIdx.x] = v;
  }
}

struct DsLoop {
  gi_schedule sc{};
  int use_selector = -1;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int32_t *x = nullptr, *snap = nullptr, *snap_h = nullptr, *Rq = nullptr, *Sq = nullptr,
          *pile[2] = {nullptr, nullptr}, *s_mark = nullptr;
  int32_t *dw = nullptr;
  uint8_t *pile_in = nullptr;
  gi_vset a, b;
};

static void dsloop_free(DeltaSplit *D) {
  DsLoop *L = static_cast<DsLoop *>(D->loop);
  if (!L) return;
  if (L->exec) cudaGraphExecDestroy(L->exec);
  if (L->graph) cudaGraphDestroy(L->graph);
  for (gi_vset *v : {&L->a, &L->b}) {
    dev_free(v->queue, nullptr);
    dev_free(v->count, nullptr);
    dev_free(v->bitmap, nullptr);
    dev_free(v->boolmap, nullptr);
  }
  for (void *p : {(void *)L->x, (void *)L->snap, (void *)L->snap_h, (void *)L->Rq, (void *)L->Sq, (void *)L->pile[0],
                  (void *)L->pile[1], (void *)L->dw, (void *)L->s_mark, (void *)L->pile_in})
    dev_free(p, nullptr);
  delete L;
  D->loop = nullptr;
}

// one round F -> N captured on cs into `body`: split + decision (one kernel),
// switch over the round's relaxation, epilogue (which also empties F, the
// next round's output set; N was emptied the same way a round before)
static int dsg_round(gi_graph *g, DeltaSplit *D, DsLoop *L, const gi_schedule &sc, gi_vset *F, gi_vset *N,
                     cudaGraph_t body, cudaGraphConditionalHandle hw, cudaStream_t cs) {
  const int grid = g->num_sms * 8;
  const bool pull_ok = g->symmetric;
  cudaGraphConditionalHandle hs;
  GI_CUDA(cudaGraphConditionalHandleCreate(&hs, body, kDgDone, cudaGraphCondAssignDefault));
  DsgBuffers B{F->queue, F->count, F->bitmap, L->x, L->dw, L->Rq, L->snap, L->snap_h, L->Sq, L->pile[0], L->pile[1],
               L->s_mark, L->pile_in, D->deg_l, D->deg_h};
  DecideParams p = decide_params(sc, 0, false);
  GI_TRY(dsg_step_launch(g, B, p, sc.delta, pull_ok, (unsigned long long)hs, (unsigned long long)hw, cs));
  // the switch node after what was captured so far
  cudaStreamCaptureStatus cst;
  const cudaGraphNode_t *deps = nullptr;
  size_t ndeps = 0;
  GI_CUDA(cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps));
  std::vector<cudaGraphNode_t> dv(deps, deps + ndeps);
  cudaGraph_t seg = nullptr;  // capturing into `body`: the same graph comes back
  GI_CUDA(cudaStreamEndCapture(cs, &seg));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = hs;
  cp.conditional.type = cudaGraphCondTypeSwitch;
  cp.conditional.size = 5;
  cudaGraphNode_t sw;
  GI_CUDA(cudaGraphAddNode(&sw, body, dv.data(), nullptr, dv.size(), &cp));
  // branches: light push, light pull, heavy push, heavy pull, next bucket
  gi_vset Rv{}, Sv{};
  Rv.g = Sv.g = g;
  Rv.n = Sv.n = g->n;
  Rv.queue = L->Rq;
  Rv.count = L->dw + kDgPushL;
  Rv.reps = GI_REP_SPARSE;
  Sv.queue = L->Sq;
  Sv.count = L->dw + kDgPushH;
  Sv.reps = GI_REP_SPARSE;
  for (int k = 0; k < 5; ++k) {
    GI_CUDA(cudaStreamBeginCaptureToGraph(cs, cp.conditional.phGraph_out[k], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeRelaxed));
    int st = GI_OK;
    const bool light = k < 2;
    const Csr &arcs = light ? D->light : D->heavy;
    OpMinInt op{L->x, light ? L->snap : L->snap_h, arcs.wt};
    if (k == kDgLightPush || k == kDgHeavyPush) {
      st = launch_push(g, op, kSrcQueue, light ? &Rv : &Sv, nullptr, out_of(N), sc, cs, &arcs);
    } else if (k == kDgLightPull || k == kDgHeavyPull) {
      const Csr &pc = D->pull_csr(light, sc.balance == GI_BAL_VERTEX);
      if (!light) {
        // heavy round: rows at or below the bucket's end are not pulled
        const OpMinIntBounded opb{op, L->dw + kDgHi, 0};
        st = launch_pull_tiled(g, opb, pc, light ? D->tl : D->th, FSet(), nullptr, out_of(N), cs, kClassMinPull,
                               sc.balance == GI_BAL_VERTEX);
      } else {
        st = launch_pull_tiled(g, op, pc, light ? D->tl : D->th, FSet(), nullptr, out_of(N), cs, kClassMinPull,
                               sc.balance == GI_BAL_VERTEX);
      }
    } else {
      k_dsg_pile_split<<<grid, 256, 0, cs>>>(L->x, L->dw, L->pile_in, L->pile[0], L->pile[1], N->queue, N->count);
      st = launch_status(1);
    }
    cudaGraph_t got = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cs, &got);
    GI_TRY(st);
    if (e != cudaSuccess) return cuda_fail(e, "branch capture", __FILE__, __LINE__);
  }
  // the next round's kernels follow the switch node
  GI_CUDA(cudaStreamBeginCaptureToGraph(cs, body, &sw, nullptr, 1, cudaStreamCaptureModeRelaxed));
  N->reps = GI_REP_SPARSE | GI_REP_BITMAP;
  return GI_OK;
}

static int dsloop_build(gi_graph *g, DeltaSplit *D, const gi_schedule &sc, DsLoop *L, cudaStream_t s) {
  const int64_t n = g->n;
  GI_TRY(heavy_get(g, s));
  for (int32_t **p : {&L->x, &L->snap, &L->snap_h, &L->Rq, &L->Sq, &L->pile[0], &L->pile[1], &L->s_mark})
    GI_TRY(dev_alloc_n(p, n, s));
  GI_TRY(dev_alloc_n(&L->dw, kDgWords, s));
  GI_TRY(dev_alloc_n(&L->pile_in, n, s));
  GI_TRY(vset_alloc(g, &L->a, s));
  GI_TRY(vset_alloc(g, &L->b, s));
  GI_CUDA(cudaStreamSynchronize(s));
  GI_CUDA(cudaGraphCreate(&L->graph, 0));
  cudaGraphConditionalHandle hw;
  GI_CUDA(cudaGraphConditionalHandleCreate(&hw, L->graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = hw;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t loop;
  GI_CUDA(cudaGraphAddNode(&loop, L->graph, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  cudaStream_t cs;
  GI_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  int st = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) == cudaSuccess
               ? GI_OK
               : cuda_fail(cudaGetLastError(), "begin capture", __FILE__, __LINE__);
  L->a.reps = L->b.reps = GI_REP_SPARSE | GI_REP_BITMAP;
  if (st == GI_OK) st = dsg_round(g, D, L, sc, &L->a, &L->b, body, hw, cs);
  if (st == GI_OK) st = dsg_round(g, D, L, sc, &L->b, &L->a, body, hw, cs);
  cudaGraph_t captured = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(cs, &captured);
  cudaStreamDestroy(cs);
  if (st == GI_OK && ec != cudaSuccess) st = cuda_fail(ec, "end capture", __FILE__, __LINE__);
  if (st == GI_OK && cudaGraphInstantiate(&L->exec, L->graph, 0) != cudaSuccess)
    st = cuda_fail(cudaGetLastError(), "graph instantiate", __FILE__, __LINE__);
  return st;
}

}  // namespace gi

// SSSP distances by the graph-driven loop; rounds = relaxation rounds run
// the graph's cached delta-stepping split and graph-driven loop for `sched`,
// built (or rebuilt) if needed; *sc_out receives the loop's normalized schedule
static int dsloop_get(gi_graph *g, const gi_schedule &sched, cudaStream_t s, DsLoop **out, gi_schedule *sc_out) {
  gi_schedule sc = sched;
  sc.balance = sc.balance == GI_BAL_EDGE_PARALLEL ? GI_BAL_EDGE_AWARE : sc.balance;  // needs a host-known |F|
  sc.persistent = 2;
  sc.delta = sc.delta > 0 ? sc.delta : INT32_MAX;  // Bellman-Ford: one bucket, every arc light
  DeltaSplit *D = nullptr;
  GI_TRY(dstep_get(g, sc.delta, sc.tile_edges, s, &D));
  const int use_sel = selector_loaded() ? 1 : 0;
  DsLoop *L = static_cast<DsLoop *>(D->loop);
  if (L && (std::memcmp(&L->sc, &sc, sizeof(sc)) != 0 || L->use_selector != use_sel)) {
    dsloop_free(D);
    L = nullptr;
  }
  if (!L) {
    L = new DsLoop();
    L->sc = sc;
    L->use_selector = use_sel;
    D->loop = L;
    const int st = dsloop_build(g, D, sc, L, s);
    if (st != GI_OK) {
      dsloop_free(D);
      return st;
    }
  }
  *out = L;
  if (sc_out) *sc_out = sc;
  return GI_OK;
}

static int run_graph_sssp(gi_graph *g, int32_t src, int32_t *dist, const gi_schedule &sched, int32_t *rounds,
                          cudaStream_t s) {
  DsLoop *L = nullptr;
  gi_schedule sc;
  GI_TRY(dsloop_get(g, sched, s, &L, &sc));
  const int64_t n = g->n;
  k_fill_i32<<<grid_for(g, n, 256), 256, 0, s>>>(L->x, n, INT32_MAX);
  k_fill_i32<<<grid_for(g, n, 256), 256, 0, s>>>(L->snap, n, INT32_MAX);
  k_fill_i32<<<grid_for(g, n, 256), 256, 0, s>>>(L->snap_h, n, INT32_MAX);
  k_fill_i32<<<grid_for(g, n, 256), 256, 0, s>>>(L->s_mark, n, -1);
  k_set_one<<<1, 1, 0, s>>>(L->x, src, 0);
  const int64_t cap64 = 4 * n + 16;
  k_dsg_init<<<1, 32, 0, s>>>(L->dw, sc.delta, (int32_t)(cap64 < INT32_MAX ? cap64 : INT32_MAX));
  GI_TRY(launch_status(6));
  GI_CUDA(cudaMemsetAsync(L->pile_in, 0, (size_t)(n > 0 ? n : 1), s));
  GI_TRY(front_init(g, &L->a, src, s));
  GI_TRY(vset_clear(&L->b, s));
  GI_TRY(ctrl_init(g, 0, 0, s));
  GI_CUDA(cudaGraphLaunch(L->exec, s));
  GI_CUDA(cudaMemcpyAsync(dist, L->x, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
  int32_t dw[kDgWords];
  GI_CUDA(cudaMemcpyAsync(dw, L->dw, sizeof(dw), cudaMemcpyDeviceToHost, s));
  GI_CUDA(cudaStreamSynchronize(s));
  if (dw[kDgErr]) {
    set_error("graph-driven SSSP reached its round cap");
    return GI_ERR_TIMEOUT;
  }
  *rounds = dw[kDgRound];
  return GI_OK;
}

extern "C" int gi_sssp(gi_graph *g, int32_t src, int32_t *dist, const gi_schedule *sched, gi_trace *trace,
                       void *stream) {
  GI_ARG(g != nullptr, "graph is NULL");
  GI_TRY(check_schedule(sched));
  GI_ARG(src >= 0 && src < g->n, "source out of range");
  GI_ARG(dist != nullptr, "dist is NULL");
  GI_ARG(g->out.wt != nullptr, "SSSP needs edge weights");
  if (forced_direction(sched->direction) >= 0) GI_TRY(pull_available(g, forced_direction(sched->direction)));
  if (forced_direction(sched->direction) == GI_DIR_DENSE_PULL || sched->direction == GI_DIR_HYBRID_PULL) {
    GI_ARG(g->symmetric || g->in.wt != nullptr, "pull SSSP needs in-edge weights (gi_load_csc with weights)");
  }
  if (sched->persistent == 1) return run_persistent(g, GI_ALGO_SSSP, src, dist, *sched, trace, (cudaStream_t)stream);
  if (sched->persistent == 2) {
    int32_t rounds = 0;
    GI_TRY(run_graph_sssp(g, src, dist, *sched, &rounds, (cudaStream_t)stream));
    if (trace) trace->iterations = rounds;
    return GI_OK;
  }
  if (sched->delta > 0) return deltastep_run(g, dist, src, *sched, trace, (cudaStream_t)stream);
  return minlabel_run(g, dist, GI_K_SSSP, src, *sched, trace, (cudaStream_t)stream);
}

extern "C" int gi_prepare(gi_graph *g, int32_t algo, const gi_schedule *sched, void *stream) {
  GI_ARG(g != nullptr, "graph is NULL");
  GI_TRY(check_schedule(sched));
  GI_ARG(algo >= GI_ALGO_BFS && algo <= GI_ALGO_PAGERANK_DELTA, "unknown algo");
  cudaStream_t s = (cudaStream_t)stream;
  const gi_schedule &sc = *sched;
  GI_TRY(ensure_tiles(g, sc, s));
  if (algo == GI_ALGO_BFS) {
    if (sc.persistent == 2) {
      GraphLoop *L = nullptr;
      GI_TRY(graph_loop_get(g, sc, s, &L));
    } else if (sc.dst_list && g->has_csc && sc.persistent == 0) {
      BfsUnv U;
      GI_TRY(bfs_unv_get(g, s, &U));
    }
  } else if (algo == GI_ALGO_SSSP) {
    GI_ARG(g->out.wt != nullptr, "SSSP needs edge weights");
    if (sc.persistent == 2) {
      DsLoop *L = nullptr;
      GI_TRY(dsloop_get(g, sc, s, &L, nullptr));
    } else if (sc.delta > 0 && sc.persistent == 0) {
      DeltaSplit *D = nullptr;
      GI_TRY(dstep_get(g, sc.delta, sc.tile_edges, s, &D));
    }
  }
  GI_CUDA(cudaStreamSynchronize(s));
  return GI_OK;
}

extern "C" int gi_cc(gi_graph *g, int32_t *label, const gi_schedule *sched, gi_trace *trace, void *stream) {
  GI_ARG(g != nullptr, "graph is NULL");
  GI_TRY(check_schedule(sched));
  GI_ARG(label != nullptr, "label is NULL");
  if (forced_direction(sched->direction) >= 0) GI_TRY(pull_available(g, forced_direction(sched->direction)));
  if (g->n == 0) return GI_OK;
  return minlabel_run(g, label, GI_K_CC, 0, *sched, trace, (cudaStream_t)stream);
}

// ================================================================ PageRank ==
static int pr_normalize(gi_graph *g, float *rank, cudaStream_t s) {
  const int np = g->num_sms * 2;
  double *partial = nullptr;
  GI_TRY(dev_alloc_n(&partial, np, s));
  k_sum_f64<<<np, 256, 0, s>>>(rank, g->n, partial);
  k_scale_f64<<<grid_for(g, g->n, 256), 256, 0, s>>>(rank, g->n, partial, np);
  int st = launch_status(2);
  dev_free(partial, s);
  return st;
}

extern "C" int gi_pagerank(gi_graph *g, float damping, int32_t iters, float *rank, const gi_schedule *sched,
                           void *stream) {
  GI_ARG(g != nullptr, "graph is NULL");
  GI_TRY(check_schedule(sched));
  GI_ARG(rank != nullptr || g->n == 0, "rank is NULL");
  GI_ARG(iters >= 0, "iters must be >= 0");
  GI_ARG(damping >= 0.0f && damping <= 1.0f, "damping must be in [0,1]");
  if (g->n == 0) return GI_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const gi_schedule sc = *sched;
  const bool push = sc.direction == GI_DIR_DENSE_PUSH || sc.direction == GI_DIR_SPARSE_PUSH;
  if (!push) GI_TRY(pull_available(g, GI_DIR_DENSE_PULL));
  GI_TRY(ensure_tiles(g, sc, s));
  const bool segmented = !push && sc.num_segments > 1;
  if (segmented && (g->segs.num != sc.num_segments || g->segs.strategy != sc.seg_strategy))
    GI_TRY(gi_graph_build_segments(g, sc.num_segments, sc.seg_strategy, s));
  const float base = (1.0f - damping) / (float)g->n, init = 1.0f / (float)g->n;
  float *buf[2] = {nullptr, nullptr}, *acc = nullptr;
  double *acc64 = nullptr;
  int st = dev_alloc_n(&buf[0], g->n, s);
  if (st == GI_OK) st = dev_alloc_n(&buf[1], g->n, s);
  if (st == GI_OK && segmented) st = dev_alloc_n(&acc, g->n, s);
  if (st == GI_OK && push) st = dev_alloc_n(&acc64, g->n, s);
  if (st == GI_OK && acc) st = cudaMemsetAsync(acc, 0, sizeof(float) * g->n, s) == cudaSuccess ? GI_OK : GI_ERR_CUDA;
  if (st == GI_OK && acc64)
    st = cudaMemsetAsync(acc64, 0, sizeof(double) * g->n, s) == cudaSuccess ? GI_OK : GI_ERR_CUDA;
  if (st == GI_OK) {
    if (iters == 0) k_fill_f32<<<grid_for(g, g->n, 256), 256, 0, s>>>(rank, g->n, init);
    k_pr_init<<<grid_for(g, g->n, 256), 256, 0, s>>>(buf[0], g->inv_out_deg, g->n, init);
    st = launch_status(1 + (iters == 0 ? 1 : 0));
  }
  for (int32_t k = 0; k < iters && st == GI_OK; ++k) {
    const bool last = (k == iters - 1);
    float *cin = buf[k & 1], *cout = buf[(k + 1) & 1];
    if (push) {
      OpSumPush64 op{cin, acc64};
      st = launch_push(g, op, kSrcAll, nullptr, nullptr, OutSet(), sc, s);
      if (st == GI_OK) {
        k_pr_vertex<<<grid_for(g, g->n, 256), 256, 0, s>>>(acc64, last ? nullptr : cout, last ? rank : nullptr,
                                                           g->inv_out_deg, g->n, base, damping);
        st = launch_status(1);
      }
    } else if (segmented) {
      // one SSG at a time (Sec. 6): acc accumulates over segments without
      // atomics; the last segment applies the vertex update.
      for (int sid = 0; sid < g->segs.num && st == GI_OK; ++sid) {
        if (sid + 1 < g->segs.num) {
          OpSum op{cin, acc};
          st = launch_pull_tiled(g, op, g->segs.seg[sid], g->segs.tiles[sid], nullptr, nullptr, OutSet(), s);
        } else {
          OpSum op{cin, acc};
          st = launch_pull_tiled(g, op, g->segs.seg[sid], g->segs.tiles[sid], nullptr, nullptr, OutSet(), s);
          if (st == GI_OK) {
            k_pr_vertex<<<grid_for(g, g->n, 256), 256, 0, s>>>(acc, last ? nullptr : cout, last ? rank : nullptr,
                                                               g->inv_out_deg, g->n, base, damping);
            st = launch_status(1);
          }
        }
      }
    } else {
      OpPR op{cin, last ? nullptr : cout, last ? rank : nullptr, g->inv_out_deg, base, damping};
      st = launch_pull_tiled(g, op, g->in, g->in_tiles, nullptr, nullptr, OutSet(), s, kClassPrPull,
                             sc.balance == GI_BAL_VERTEX, sc.hot_cache);
    }
  }
  if (st == GI_OK) st = pr_normalize(g, rank, s);
  dev_free(buf[0], s);
  dev_free(buf[1], s);
  dev_free(acc, s);
  dev_free(acc64, s);
  if (st == GI_OK && cudaStreamSynchronize(s) != cudaSuccess)
    st = cuda_fail(cudaGetLastError(), "pagerank", __FILE__, __LINE__);
  return st;
}

// =========================================================== PageRankDelta ==
extern "C" int gi_pagerank_delta(gi_graph *g, float damping, float eps, int32_t iters, float *rank,
                                 const gi_schedule *sched, gi_trace *trace, void *stream) {
  GI_ARG(g != nullptr, "graph is NULL");
  GI_TRY(check_schedule(sched));
  GI_ARG(rank != nullptr || g->n == 0, "rank is NULL");
  GI_ARG(iters >= 0, "iters must be >= 0");
  GI_ARG(eps >= 0.0f, "eps must be >= 0");
  if (g->n == 0) return GI_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const gi_schedule sc = *sched;
  if (forced_direction(sc.direction) >= 0) GI_TRY(pull_available(g, forced_direction(sc.direction)));
  GI_TRY(ensure_tiles(g, sc, s));
  const float inv_n = 1.0f / (float)g->n, first_base = (1.0f - damping) / (float)g->n;
  VsetPair P;
  float *cb[2] = {nullptr, nullptr}, *seg_sum = nullptr;
  double *dsum = nullptr;
  int st = pair_alloc(g, P, s);
  if (st == GI_OK) st = dev_alloc_n(&cb[0], g->n, s);
  if (st == GI_OK) st = dev_alloc_n(&cb[1], g->n, s);
  if (st == GI_OK) st = dev_alloc_n(&dsum, g->n, s);
  const bool segmented = sc.num_segments > 1 && g->has_csc;
  if (st == GI_OK && segmented) {
    if (g->segs.num != sc.num_segments || g->segs.strategy != sc.seg_strategy)
      st = gi_graph_build_segments(g, sc.num_segments, sc.seg_strategy, s);
    if (st == GI_OK) st = dev_alloc_n(&seg_sum, g->n, s);
    if (st == GI_OK && cudaMemsetAsync(seg_sum, 0, sizeof(float) * g->n, s) != cudaSuccess)
      st = cuda_fail(cudaGetLastError(), "memset", __FILE__, __LINE__);
  }
  if (st == GI_OK) {
    k_fill_f32<<<grid_for(g, g->n, 256), 256, 0, s>>>(rank, g->n, 0.0f);
    k_pr_init<<<grid_for(g, g->n, 256), 256, 0, s>>>(cb[0], g->inv_out_deg, g->n, inv_n);
    st = launch_status(2);
    if (st == GI_OK && cudaMemsetAsync(dsum, 0, sizeof(double) * g->n, s) != cudaSuccess)
      st = cuda_fail(cudaGetLastError(), "memset", __FILE__, __LINE__);
  }
  if (st == GI_OK) st = front_init(g, P.F, -1, s);
  if (st == GI_OK) st = ctrl_init(g, 0, 0, s);
  int cur = 0;
  for (int32_t round = 1; round <= iters && st == GI_OK; ++round) {
    DecideParams p = decide_params(sc, round - 1, false);
    if ((st = frontier_decide(g, P.F, p, s)) != GI_OK) break;
    if ((st = ctrl_fetch(g, s)) != GI_OK) break;
    if (g->ctrl_host[kNf] == 0 && round > 1) {
      if (trace) trace->iterations = round - 1;
      break;  // nothing active: Delta = 0 from now on, ranks stay
    }
    int32_t dir = (int32_t)g->ctrl_host[kDecision];
    if (dir == GI_DIR_DENSE_PULL && !g->has_csc) dir = GI_DIR_DENSE_PUSH;
    trace_put(trace, round - 1, g->ctrl_host);
    if ((st = vset_clear(P.N, s)) != GI_OK) break;
    float *cin = cb[cur], *cout = cb[cur ^ 1];
    g->hint_vset = P.F;
    g->hint_nf = g->ctrl_host[kNf];
    g->hint_mf = g->ctrl_host[kMf];
    if (dir == GI_DIR_DENSE_PULL && segmented) {
      // cache-partitioned pull: segments add into seg_sum, then the vertex filter
      for (int sid = 0; sid < g->segs.num && st == GI_OK; ++sid) {
        OpSum op{cin, seg_sum};
        st = launch_pull_tiled(g, op, g->segs.seg[sid], g->segs.tiles[sid], nullptr, nullptr, OutSet(), s,
                               kClassPrdPull);
      }
      if (st == GI_OK) {
        k_prd_vertex<<<grid_for(g, g->n, 256), 256, 0, s>>>(seg_sum, rank, cout, g->inv_out_deg, g->n, damping,
                                                            first_base, inv_n, eps, round == 1 ? 1 : 0, P.N->bitmap,
                                                            P.N->queue, P.N->count);
        st = launch_status(1);
      }
    } else if (dir == GI_DIR_DENSE_PULL) {
      OpPRD op{cin, cout, rank, g->inv_out_deg, damping, first_base, inv_n, eps, round == 1 ? 1 : 0};
      st = launch_pull_tiled(g, op, g->in, g->in_tiles, nullptr, nullptr, out_of(P.N), s, kClassPrdPull,
                             sc.balance == GI_BAL_VERTEX, sc.hot_cache);
    } else {
      OpSumPush64 op{cin, dsum};
      st = launch_push(g, op, dir == GI_DIR_SPARSE_PUSH ? kSrcQueue : kSrcBitmap, P.F, nullptr, OutSet(), sc, s);
      if (st == GI_OK) {
        k_prd_vertex<<<grid_for(g, g->n, 256), 256, 0, s>>>(dsum, rank, cout, g->inv_out_deg, g->n, damping,
                                                            first_base, inv_n, eps, round == 1 ? 1 : 0, P.N->bitmap,
                                                            P.N->queue, P.N->count);
        st = launch_status(1);
      }
    }
    g->hint_vset = nullptr;
    g->hint_nf = -1;
    g->hint_mf = -1;
    P.N->reps = GI_REP_SPARSE | GI_REP_BITMAP;
    P.swap();
    cur ^= 1;
  }
  dev_free(cb[0], s);
  dev_free(cb[1], s);
  dev_free(dsum, s);
  dev_free(seg_sum, s);
  pair_free(P, s);
  if (st == GI_OK && cudaStreamSynchronize(s) != cudaSuccess)
    st = cuda_fail(cudaGetLastError(), "prdelta", __FILE__, __LINE__);
  return st;
}

// ==================================================== Betweenness Centrality ==
// Single-source dependencies (Brandes), run as the paper runs BC (Sec. 7):
// synchronously, with two edgeset applies per level.
//   s1 (forward): path-counting BFS; a vertex found at level d+1 receives
//     sigma[v] = sum of sigma[u] over its in-neighbours u in F_d.  Push adds
//     with FP64 atomics (sums of integers: exact below 2^53), pull gathers.
//   s2 (backward): levels from the deepest up; w[v] = (1 + delta[v]) / sigma[v]
//     is set on level d+1 and zero everywhere else, so for u in level d
//     delta[u] = sigma[u] * sum of w over u's out-neighbours.  Either a
//     SparsePull over level d's queue along the out-edges (thread / warp /
//     block per vertex) or, for large levels of symmetric graphs, the tiled
//     pull over all rows with the level as destination filter.  Both sum in
//     a fixed order, without atomics.
namespace gi {

struct OpBCFwd {
  using V = double;
  static constexpr bool kSkipZeroTerms = true;
  int32_t *depth;
  double *sigma;
  int32_t level;  // depth of the vertices found in this step
  __device__ static V identity() { return 0.0; }
  __device__ static V combine(V a, V b) { return a + b; }
  __device__ V edge_val(int32_t u, int32_t) const { return sigma[u]; }
  __device__ bool dst_ok(int32_t v) const { return depth[v] == -1; }
  __device__ bool finish(int32_t v, V s) const {
    if (s > 0.0) {
      depth[v] = level;
      sigma[v] = s;
      return true;
    }
    return false;
  }
  __device__ bool push(int32_t u, int32_t v, int32_t) const {
    const int32_t d = *(volatile int32_t *)(depth + v);
    if (d != -1 && d != level) return false;
    bool won = false;
    if (d == -1) {
      const int32_t old = atomicCAS(depth + v, -1, level);
      won = (old == -1);
      if (!won && old != level) return false;
    }
    atomicAdd(sigma + v, sigma[u]);
    return won;
  }
};

struct OpBCBack {
  using V = double;
  static constexpr bool kSkipZeroTerms = true;
  const double *w;
  double *delta;
  const double *sigma;
  const int32_t *depth;
  int32_t level;  // rows (sources of the out-arcs) being accumulated
  __device__ static V identity() { return 0.0; }
  __device__ static V combine(V a, V b) { return a + b; }
  __device__ V edge_val(int32_t v, int32_t) const { return __ldg(w + v); }
  __device__ bool dst_ok(int32_t u) const { return depth[u] == level; }
  __device__ bool finish(int32_t u, V s) const {
    delta[u] = sigma[u] * s;
    return false;
  }
  __device__ bool push(int32_t, int32_t, int32_t) const { return false; }
};

// w[v] = (1 + delta[v]) / sigma[v] on the level below the one accumulated
// next (q_set); w back to 0 on the level that was below it before (q_clear).
__global__ void k_bc_weights(const int32_t *__restrict__ q_set, int64_t n_set, const int32_t *__restrict__ q_clear,
                             int64_t n_clear, const double *__restrict__ delta, const double *__restrict__ sigma,
                             double *w) {
  const int64_t nmax = n_set > n_clear ? n_set : n_clear;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nmax; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n_clear) w[q_clear[i]] = 0.0;
    if (i < n_set) {
      const int32_t v = q_set[i];
      w[v] = (1.0 + delta[v]) / sigma[v];
    }
  }
}

__global__ void k_bc_init(int32_t *depth, double *sigma, double *delta, double *w, int64_t n, int32_t src) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    depth[i] = i == src ? 0 : -1;
    sigma[i] = i == src ? 1.0 : 0.0;
    delta[i] = 0.0;
    w[i] = 0.0;
  }
}

// dependency[v] (+)= delta[v], with delta[src] = 0 (src is no interior vertex)
__global__ void k_bc_out(const double *__restrict__ delta, double *dep, int64_t n, int32_t src, int32_t accumulate) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = i == src ? 0.0 : delta[i];
    dep[i] = accumulate ? dep[i] + x : x;
  }
}

// one forward step (s1) from F into N at level `level`
static int bc_forward(gi_graph *g, VsetPair &P, int32_t dir, const gi_schedule &sc, int32_t *depth, double *sigma,
                      int32_t level, cudaStream_t s) {
  GI_TRY(vset_clear(P.N, s));
  const OutSet o = out_of(P.N, true);
  const OpBCFwd op{depth, sigma, level};
  if (dir == GI_DIR_DENSE_PULL) {
    GI_TRY(vset_ensure_bitmap(P.F, s));
    GI_TRY(launch_pull_tiled(g, op, g->in, g->in_tiles, FSet(static_cast<const uint32_t *>(P.F->bitmap)), nullptr,
                             o, s, kClassOtherPull, sc.balance == GI_BAL_VERTEX));
  } else if (dir == GI_DIR_SPARSE_PUSH) {
    GI_TRY(vset_ensure_queue(P.F, s));
    GI_TRY(launch_push(g, op, kSrcQueue, P.F, nullptr, o, sc, s));
  } else {
    GI_TRY(vset_ensure_bitmap(P.F, s));
    GI_TRY(launch_push(g, op, kSrcBitmap, P.F, nullptr, o, sc, s));
  }
  P.N->reps = GI_REP_SPARSE | GI_REP_BITMAP;
  return GI_OK;
}

}  // namespace gi

extern "C" int gi_bc(gi_graph *g, int32_t src, double *dependency, double *sigma_out, int32_t accumulate,
                     const gi_schedule *sched, gi_trace *trace, void *stream) {
  GI_ARG(g != nullptr, "graph is NULL");
  GI_TRY(check_schedule(sched));
  GI_ARG(src >= 0 && src < g->n, "source out of range");
  GI_ARG(dependency != nullptr, "dependency is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const gi_schedule sc = *sched;
  if (forced_direction(sc.direction) >= 0) GI_TRY(pull_available(g, forced_direction(sc.direction)));
  GI_TRY(ensure_tiles(g, sc, s));
  const int64_t n = g->n;
  VsetPair P;
  int32_t *depth = nullptr, *levels = nullptr;
  double *sigma = sigma_out, *own_sigma = nullptr, *delta = nullptr, *w = nullptr;
  int st = pair_alloc(g, P, s);
  if (st == GI_OK) st = dev_alloc_n(&depth, n, s);
  if (st == GI_OK) st = dev_alloc_n(&levels, n, s);
  if (st == GI_OK && !sigma) st = dev_alloc_n(&own_sigma, n, s), sigma = own_sigma;
  if (st == GI_OK) st = dev_alloc_n(&delta, n, s);
  if (st == GI_OK) st = dev_alloc_n(&w, n, s);
  if (st == GI_OK) {
    k_bc_init<<<grid_for(g, n, 256), 256, 0, s>>>(depth, sigma, delta, w, n, src);
    st = launch_status(1);
  }
  if (st == GI_OK) st = front_init(g, P.F, src, s);
  if (st == GI_OK) st = ctrl_init(g, g->n, g->m, s);
  // level d's vertices: levels[off[d] .. off[d+1]); its frontier statistics in nf/mf
  std::vector<int64_t> off{0}, nf, mf;
  if (st == GI_OK)
    st = frontier_loop(g, P, sc, true, trace, s, [&](int32_t it, int32_t dir) -> int {
      const int64_t k = g->ctrl_host[kNf];
      nf.push_back(k);
      mf.push_back(g->ctrl_host[kMf]);
      GI_TRY(vset_ensure_queue(P.F, s));
      GI_CUDA(cudaMemcpyAsync(levels + off.back(), P.F->queue, sizeof(int32_t) * (size_t)k,
                              cudaMemcpyDeviceToDevice, s));
      off.push_back(off.back() + k);
      return bc_forward(g, P, dir, sc, depth, sigma, it + 1, s);
    });
  const int32_t D = (int32_t)nf.size();
  for (int32_t d = D - 2; d >= 1 && st == GI_OK; --d) {
    const int64_t n_set = nf[d + 1], n_clear = d + 2 < D ? nf[d + 2] : 0;
    k_bc_weights<<<grid_for(g, n_set > n_clear ? n_set : n_clear, 256), 256, 0, s>>>(
        levels + off[d + 1], n_set, levels + off[d + 2 < D ? d + 2 : d + 1], n_clear, delta, sigma, w);
    st = launch_status(1);
    if (st != GI_OK) break;
    // s2's direction: SparsePull over level d's queue, or the dense pull over
    // all rows; forced by the schedule, else Ligra's rule on level d
    const int32_t fd = forced_direction(sc.direction);
    bool dense;
    if (sc.direction == GI_DIR_SPARSE_PULL || fd == GI_DIR_SPARSE_PUSH || fd == GI_DIR_DENSE_PUSH) dense = false;
    else if (fd == GI_DIR_DENSE_PULL) dense = true;
    else dense = (nf[d] + mf[d]) > g->m / 20;
    dense = dense && g->symmetric && sc.balance != GI_BAL_VERTEX;
    const OpBCBack op{w, delta, sigma, depth, d};
    if (dense)
      st = launch_pull_tiled(g, op, g->in, g->in_tiles, FSet(), nullptr, OutSet(), s, kClassOtherPull);
    else
      st = launch_pull_sparse(g, op, g->out, levels + off[d], nullptr, nf[d], FSet(), OutSet(), sc, s);
  }
  if (st == GI_OK) {
    k_bc_out<<<grid_for(g, n, 256), 256, 0, s>>>(delta, dependency, n, src, accumulate);
    st = launch_status(1);
  }
  dev_free(depth, s);
  dev_free(levels, s);
  dev_free(own_sigma, s);
  dev_free(delta, s);
  dev_free(w, s);
  pair_free(P, s);
  if (st == GI_OK && cudaStreamSynchronize(s) != cudaSuccess)
    st = cuda_fail(cudaGetLastError(), "bc", __FILE__, __LINE__);
  return st;
}

// ======================================================= selector profiling ==
// Training data for the learned selector: at every level of a BFS or SSSP run
// the state is kept, each of SparsePush / DensePush / DensePull runs from it
// and is timed with CUDA events, and the run continues from the (identical)
// result.  The level's features are those the selector sees at inference;
// "was_pull" follows the Beamer / Ligra rule's choice.
extern "C" int gi_selector_profile(gi_graph *g, int32_t kernel_id, int32_t src, const gi_schedule *sched, int32_t cap,
                                   float *features, float *times_ms, int32_t *levels, void *stream) {
  GI_ARG(g != nullptr, "graph is NULL");
  GI_TRY(check_schedule(sched));
  GI_ARG(kernel_id == GI_K_BFS || kernel_id == GI_K_SSSP, "profiling supports GI_K_BFS and GI_K_SSSP");
  GI_ARG(src >= 0 && src < g->n, "source out of range");
  GI_ARG(cap >= 0 && features != nullptr && times_ms != nullptr && levels != nullptr, "NULL output");
  if (kernel_id == GI_K_SSSP) GI_ARG(g->out.wt != nullptr, "SSSP needs edge weights");
  if (!g->has_csc) {
    set_error("profiling runs DensePull and needs the in-edges");
    return GI_ERR_UNSUPPORTED;
  }
  cudaStream_t s = (cudaStream_t)stream;
  gi_schedule sc = *sched;
  sc.direction = GI_DIR_HYBRID_PULL;
  if (kernel_id == GI_K_SSSP && sc.delta > 0) {
    // delta-stepping rounds: SparsePush and DensePull timed from each state
    if (!g->symmetric) {
      set_error("delta-stepping profiles need a symmetric graph (the pull relaxes the split arcs as in-edges)");
      return GI_ERR_UNSUPPORTED;
    }
    int32_t *x = nullptr;
    GI_TRY(dev_alloc_n(&x, g->n, s));
    DsProfile prof;
    prof.cap = cap;
    prof.features = features;
    prof.times_ms = times_ms;
    const int st = deltastep_run(g, x, src, sc, nullptr, s, &prof);
    dev_free(x, s);
    *levels = prof.rounds;
    return st;
  }
  GI_TRY(ensure_tiles(g, sc, s));
  const bool bfs = kernel_id == GI_K_BFS;
  VsetPair P;
  int32_t *x = nullptr, *snap = nullptr, *keep = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  int st = pair_alloc(g, P, s);
  if (st == GI_OK) st = dev_alloc_n(&x, g->n, s);
  if (st == GI_OK) st = dev_alloc_n(&keep, g->n, s);
  if (st == GI_OK && !bfs) st = dev_alloc_n(&snap, g->n, s);
  if (st == GI_OK && (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess))
    st = cuda_fail(cudaGetLastError(), "event create", __FILE__, __LINE__);
  BfsUnv U;
  if (st == GI_OK && bfs && sc.dst_list) st = bfs_unv_get(g, s, &U);
  if (st == GI_OK) {
    if (bfs) {
      // every level's pull runs last, from the state the pushes were timed
      // on, so the compacted list advances exactly as in gi_bfs
      k_bfs_init<<<grid_for(g, g->n, 256), 256, 0, s>>>(x, nullptr, g->n, src, U.st);
      st = launch_status(1);
      g->bfs_unv_query = U;
    } else {
      k_fill_i32<<<grid_for(g, g->n, 256), 256, 0, s>>>(x, g->n, INT32_MAX);
      k_fill_i32<<<grid_for(g, g->n, 256), 256, 0, s>>>(snap, g->n, INT32_MAX);
      k_set_one<<<1, 1, 0, s>>>(x, src, 0);
      k_set_one<<<1, 1, 0, s>>>(snap, src, 0);
      st = launch_status(4);
    }
  }
  if (st == GI_OK) st = front_init(g, P.F, src, s);
  if (st == GI_OK) st = ctrl_init(g, bfs ? g->n : 0, bfs ? g->m : 0, s);
  int32_t lv = 0;
  for (int32_t it = 0; st == GI_OK && lv < cap; ++it) {
    DecideParams p = decide_params(sc, it, bfs);
    if ((st = frontier_decide(g, P.F, p, s)) != GI_OK) break;
    if ((st = ctrl_fetch(g, s)) != GI_OK) break;
    if (g->ctrl_host[kNf] == 0) break;
    const float *f = reinterpret_cast<const float *>(g->ctrl_host + kFeat);
    for (int k = 0; k < 16; ++k) features[16 * lv + k] = f[k];
    if (cudaMemcpyAsync(keep, x, sizeof(int32_t) * g->n, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
      st = cuda_fail(cudaGetLastError(), "snapshot", __FILE__, __LINE__);
      break;
    }
    const int32_t dirs[3] = {GI_DIR_SPARSE_PUSH, GI_DIR_DENSE_PUSH, GI_DIR_DENSE_PULL};
    for (int k = 0; k < 3 && st == GI_OK; ++k) {
      if (k > 0 && cudaMemcpyAsync(x, keep, sizeof(int32_t) * g->n, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
        st = cuda_fail(cudaGetLastError(), "restore", __FILE__, __LINE__);
        break;
      }
      cudaEventRecord(ev[0], s);
      if (bfs) {
        gi_bfs_args a{x, nullptr, it + 1};
        st = apply_dispatch(g, P.F, nullptr, dirs[k], sc, GI_K_BFS, &a, P.N, GI_NO_DEDUP, s);
      } else {
        gi_sssp_args a{x, snap};
        st = apply_dispatch(g, P.F, nullptr, dirs[k], sc, GI_K_SSSP, &a, P.N, 0, s);
      }
      cudaEventRecord(ev[1], s);
      if (st != GI_OK) break;
      if (cudaEventSynchronize(ev[1]) != cudaSuccess) {
        st = cuda_fail(cudaGetLastError(), "profile sync", __FILE__, __LINE__);
        break;
      }
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, ev[0], ev[1]);
      times_ms[3 * lv + k] = ms;
    }
    if (st != GI_OK) break;
    if (!bfs) {
      int grid = g->num_sms * 4;
      k_snap_reset<<<grid, 256, 0, s>>>(P.F->queue, P.F->count, snap);
      k_snap_set<<<grid, 256, 0, s>>>(P.N->queue, P.N->count, snap, x);
      if ((st = launch_status(2)) != GI_OK) break;
    }
    P.swap();
    ++lv;
  }
  *levels = lv;
  g->bfs_unv_query = BfsUnv{};
  if (ev[0]) cudaEventDestroy(ev[0]);
  if (ev[1]) cudaEventDestroy(ev[1]);
  dev_free(x, s);
  dev_free(keep, s);
  dev_free(snap, s);
  pair_free(P, s);
  if (st == GI_OK && cudaStreamSynchronize(s) != cudaSuccess)
    st = cuda_fail(cudaGetLastError(), "profile", __FILE__, __LINE__);
  return st;
}
