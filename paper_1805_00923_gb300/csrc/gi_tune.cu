// Autotuner for schedule parameters (the paper tunes schedules with OpenTuner,
// Sec. 6 "Autotuning"; this is a small search written for the GPU knobs).
//
// Search: the start schedule, then random candidates, then hill climbing (one
// parameter moved to a neighbouring value of the best so far).  Every
// candidate is timed with CUDA events (best of `reps` runs after one warm-up)
// and is rejected when its output differs from the start schedule's output
// (integers bit-exact, ranks within 1e-4 relative) -- the paper's tuner
// likewise discards invalid schedules.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <functional>
#include <random>
#include <vector>

#include "gi_internal.cuh"

namespace gi {

struct Knob {
  std::function<int32_t(const gi_schedule &)> get;
  std::function<void(gi_schedule &, int32_t)> set;
  std::vector<int32_t> values;
};

template <class F>
Knob knob(F gi_schedule::*field, std::vector<int32_t> values) {
  return Knob{[field](const gi_schedule &s) { return (int32_t)(s.*field); },
              [field](gi_schedule &s, int32_t v) { s.*field = (F)v; }, std::move(values)};
}

__global__ void k_count_diff_i32(const int32_t *__restrict__ a, const int32_t *__restrict__ b, int64_t n,
                                 unsigned long long *out) {
  unsigned long long c = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    c += a[i] != b[i];
  if (c) atomicAdd(out, c);
}

__global__ void k_count_far_f32(const float *__restrict__ a, const float *__restrict__ b, int64_t n, float rtol,
                                unsigned long long *out) {
  unsigned long long c = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float d = fabsf(a[i] - b[i]), r = fabsf(b[i]);
    c += !(d <= rtol * r + 1e-30f);
  }
  if (c) atomicAdd(out, c);
}

struct Runner {
  gi_graph *g;
  int32_t algo, src;
  cudaStream_t s;
  void *out = nullptr;      // current output
  void *ref = nullptr;      // start schedule's output
  unsigned long long *diff = nullptr;

  int run(const gi_schedule &sc) {
    switch (algo) {
      case GI_ALGO_BFS: return gi_bfs(g, src, (int32_t *)out, nullptr, &sc, nullptr, s);
      case GI_ALGO_SSSP: return gi_sssp(g, src, (int32_t *)out, &sc, nullptr, s);
      case GI_ALGO_CC: return gi_cc(g, (int32_t *)out, &sc, nullptr, s);
      case GI_ALGO_PAGERANK: return gi_pagerank(g, 0.85f, 20, (float *)out, &sc, s);
      case GI_ALGO_PAGERANK_DELTA: return gi_pagerank_delta(g, 0.85f, 1e-7f, 10, (float *)out, &sc, nullptr, s);
    }
    return GI_ERR_INVALID_ARG;
  }

  bool is_float() const { return algo == GI_ALGO_PAGERANK || algo == GI_ALGO_PAGERANK_DELTA; }

  // 0 = same as reference, 1 = differs, <0 error
  int compare() {
    if (cudaMemsetAsync(diff, 0, sizeof(unsigned long long), s) != cudaSuccess) return GI_ERR_CUDA;
    if (is_float())
      k_count_far_f32<<<grid_for(g, g->n, 256), 256, 0, s>>>((const float *)out, (const float *)ref, g->n, 1e-4f,
                                                             diff);
    else
      k_count_diff_i32<<<grid_for(g, g->n, 256), 256, 0, s>>>((const int32_t *)out, (const int32_t *)ref, g->n,
                                                              diff);
    GI_TRY(launch_status(1));
    unsigned long long h = 0;
    GI_CUDA(cudaMemcpyAsync(&h, diff, sizeof(h), cudaMemcpyDeviceToHost, s));
    GI_CUDA(cudaStreamSynchronize(s));
    return h ? 1 : 0;
  }

  // best-of-reps milliseconds after one warm-up run
  int time(const gi_schedule &sc, int reps, double *ms) {
    GI_TRY(run(sc));
    cudaEvent_t a, b;
    GI_CUDA(cudaEventCreate(&a));
    GI_CUDA(cudaEventCreate(&b));
    double best = 1e300;
    int st = GI_OK;
    for (int r = 0; r < reps && st == GI_OK; ++r) {
      cudaEventRecord(a, s);
      st = run(sc);
      cudaEventRecord(b, s);
      if (st == GI_OK && cudaEventSynchronize(b) == cudaSuccess) {
        float t = 0.0f;
        cudaEventElapsedTime(&t, a, b);
        best = t < best ? t : best;
      }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *ms = best;
    return st;
  }
};

}  // namespace gi

using namespace gi;

extern "C" int gi_autotune(gi_graph *g, int32_t algo, int32_t src, const gi_schedule *start, int32_t budget,
                           uint64_t seed, gi_schedule *best, double *best_ms, double *start_ms, void *stream) {
  GI_ARG(g != nullptr && start != nullptr && best != nullptr, "NULL argument");
  GI_TRY(check_schedule(start));
  GI_ARG(algo >= GI_ALGO_BFS && algo <= GI_ALGO_PAGERANK_DELTA, "unknown algorithm");
  GI_ARG(budget >= 1 && budget <= 100000, "budget must be in [1, 100000]");
  if (algo == GI_ALGO_BFS || algo == GI_ALGO_SSSP) GI_ARG(src >= 0 && src < g->n, "source out of range");
  if (algo == GI_ALGO_SSSP) GI_ARG(g->out.wt != nullptr, "SSSP needs edge weights");
  if (g->n == 0) {
    *best = *start;
    if (best_ms) *best_ms = 0.0;
    if (start_ms) *start_ms = 0.0;
    return GI_OK;
  }
  cudaStream_t s = (cudaStream_t)stream;
  Runner R{g, algo, src, s};
  int st = dev_alloc(&R.out, 4 * (size_t)g->n, s);
  if (st == GI_OK) st = dev_alloc(&R.ref, 4 * (size_t)g->n, s);
  if (st == GI_OK) st = dev_alloc_n(&R.diff, 1, s);
  std::vector<Knob> knobs = {
      knob(&gi_schedule::tile_edges, {256, 512, 1024, 2048, 4096, 8192}),
      knob(&gi_schedule::t_warp, {8, 16, 32, 64}),
      knob(&gi_schedule::t_cta, {256, 512, 1024, 2048, 4096}),
      knob(&gi_schedule::t_heavy, {256, 512, 1024, 2048, 4096, 16384, INT32_MAX}),
      knob(&gi_schedule::block, {128, 256, 512}),
  };
  if (algo == GI_ALGO_PAGERANK && start->direction == GI_DIR_DENSE_PULL) {
    knobs.push_back(knob(&gi_schedule::num_segments, {1, 2, 4, 8}));
    knobs.push_back(knob(&gi_schedule::seg_strategy, {GI_SEG_FVC, GI_SEG_EVC}));
  }
  if (algo != GI_ALGO_BFS) knobs.push_back(knob(&gi_schedule::hot_cache, {0, 1, 2}));
  // the dense frontier representation (bitvector or boolean map) of DensePush levels
  if (algo != GI_ALGO_PAGERANK)
    knobs.push_back(knob(&gi_schedule::dense_rep, {(int32_t)GI_REP_BITMAP, (int32_t)GI_REP_BOOL}));
  // SSSP: Bellman-Ford rounds (0) or delta-stepping with these bucket widths
  if (algo == GI_ALGO_SSSP) knobs.push_back(knob(&gi_schedule::delta, {0, 16, 32, 48, 64, 96, 128, 256}));
  // BFS pull levels over every vertex or over the compacted unvisited list
  if (algo == GI_ALGO_BFS) knobs.push_back(knob(&gi_schedule::dst_list, {0, 1}));
  std::mt19937_64 rng(seed);
  const int reps = 2;
  gi_schedule cur = *start, top = *start;
  double t_start = 0.0, t_top = 0.0;
  if (st == GI_OK) st = R.time(cur, reps, &t_start);
  if (st == GI_OK && cudaMemcpyAsync(R.ref, R.out, 4 * (size_t)g->n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    st = cuda_fail(cudaGetLastError(), "autotune reference", __FILE__, __LINE__);
  t_top = t_start;
  // Beamer constants are knobs for rule-based hybrids of BFS (float fields)
  const bool tune_ab = algo == GI_ALGO_BFS && (start->direction == GI_DIR_HYBRID_PULL ||
                                               start->direction == GI_DIR_HYBRID_DPUSH);
  const float alphas[] = {4.f, 8.f, 14.f, 24.f, 48.f}, betas[] = {8.f, 16.f, 24.f, 48.f, 96.f};
  int sweep_knob = 0, sweep_val = 0;  // position of the coordinate sweep
  for (int32_t trial = 1; trial < budget && st == GI_OK; ++trial) {
    gi_schedule cand = top;
    if (trial < budget / 3) {  // random phase
      for (auto &k : knobs) k.set(cand, k.values[rng() % k.values.size()]);
      if (tune_ab) {
        cand.alpha = alphas[rng() % 5];
        cand.beta = betas[rng() % 5];
      }
    } else {
      // coordinate sweep around the best: one knob at a time (the
      // algorithm-specific ones, pushed last, first), each of its other
      // values in turn, then the next knob (a knob's values are all tried
      // before another knob moves, so interacting knobs keep their order)
      const int nk = (int)knobs.size() + (tune_ab ? 2 : 0);
      bool found = false;
      for (int guard = 0; guard < 2 * nk && !found; ++guard) {
        const int which = nk - 1 - (sweep_knob % nk);
        const int nv = which < (int)knobs.size() ? (int)knobs[which].values.size() : 5;
        if (sweep_val >= nv) {
          ++sweep_knob;
          sweep_val = 0;
          continue;
        }
        const int pos = sweep_val++;
        if (which < (int)knobs.size()) {
          auto &k = knobs[which];
          if (k.values[pos] == k.get(top)) continue;
          k.set(cand, k.values[pos]);
        } else {
          const float *vals = which == (int)knobs.size() ? alphas : betas;
          float &f = which == (int)knobs.size() ? cand.alpha : cand.beta;
          if (vals[pos] == f) continue;
          f = vals[pos];
        }
        found = true;
      }
      if (!found) continue;
    }
    if (cand.t_cta < cand.t_warp) cand.t_cta = cand.t_warp;
    double t = 0.0;
    st = R.time(cand, reps, &t);
    if (st != GI_OK) break;
    const int d = R.compare();
    if (d < 0) {
      st = d;
      break;
    }
    if (d == 0 && t < t_top) {
      top = cand;
      t_top = t;
    }
  }
  dev_free(R.out, s);
  dev_free(R.ref, s);
  dev_free(R.diff, s);
  if (st == GI_OK && cudaStreamSynchronize(s) != cudaSuccess)
    st = cuda_fail(cudaGetLastError(), "autotune", __FILE__, __LINE__);
  if (st != GI_OK) return st;
  *best = top;
  if (best_ms) *best_ms = t_top;
  if (start_ms) *start_ms = t_start;
  return GI_OK;
}

// =========================================================== batched engine ==
// The same search for the batched engine's launch options: CTAs per query
// (cluster_size), the expansion bins (t_warp, t_cta), the SSSP bucket step
// (sssp_delta) and the claim order; the start's selector and Beamer constants
// are kept.  Each candidate is a plan over the same queries writing into one
// contiguous buffer, so one kernel compares all outputs with the start's.

extern "C" int gi_batch_autotune(gi_graph *const *graphs, int32_t n_graphs, const int32_t *q_graph,
                                 const int32_t *q_src, const int32_t *q_algo, int32_t n_q, const gi_batch_opts *start,
                                 int32_t budget, uint64_t seed, gi_batch_opts *best, double *best_ms,
                                 double *start_ms, void *stream) {
  GI_ARG(graphs != nullptr && n_graphs > 0 && best != nullptr, "NULL argument");
  GI_ARG(n_q > 0 && q_graph && q_src && q_algo, "bad query arrays");
  GI_ARG(budget >= 1 && budget <= 100000, "budget must be in [1, 100000]");
  gi_batch_opts st0;
  gi_batch_opts_default(&st0);
  if (start) st0 = *start;
  st0.levels = nullptr;
  st0.parents = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int64_t> off(n_q + 1, 0);
  for (int i = 0; i < n_q; ++i) {
    GI_ARG(q_graph[i] >= 0 && q_graph[i] < n_graphs && graphs[q_graph[i]] != nullptr, "query graph out of range");
    off[i + 1] = off[i] + std::max<int64_t>(graphs[q_graph[i]]->n, 1);
  }
  const int64_t total = off[n_q];
  int32_t *out = nullptr, *ref = nullptr;
  unsigned long long *diff = nullptr;
  int st = dev_alloc_n(&out, total, s);
  if (st == GI_OK) st = dev_alloc_n(&ref, total, s);
  if (st == GI_OK) st = dev_alloc_n(&diff, 1, s);
  std::vector<int32_t *> outs(n_q);
  for (int i = 0; i < n_q; ++i) outs[i] = out + off[i];
  int dev = 0, sms = 0;
  if (st == GI_OK && (cudaGetDevice(&dev) != cudaSuccess ||
                      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess))
    st = cuda_fail(cudaGetLastError(), "device query", __FILE__, __LINE__);
  // best of two timed launches after one warm-up; *ms = 1e300 if the plan fails to build
  auto time_opts = [&](const gi_batch_opts &o, double *ms) -> int {
    gi_batch_plan *p = nullptr;
    int r = gi_batch_plan_create(graphs, n_graphs, q_graph, q_src, q_algo, n_q, outs.data(), &o, s, &p);
    if (r != GI_OK) return r;
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) r = GI_ERR_CUDA;
    double tbest = 1e300;
    for (int k = 0; k < 3 && r == GI_OK; ++k) {
      cudaEventRecord(a, s);
      r = gi_batch_plan_launch(p, s);
      cudaEventRecord(b, s);
      if (r == GI_OK) r = gi_batch_plan_results(p, nullptr, nullptr, s);
      float t = 0.0f;
      if (r == GI_OK && cudaEventElapsedTime(&t, a, b) == cudaSuccess && k > 0) tbest = t < tbest ? t : tbest;
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    const int r2 = gi_batch_plan_free(p);
    *ms = tbest;
    return r != GI_OK ? r : r2;
  };
  auto differs = [&]() -> int {
    GI_CUDA(cudaMemsetAsync(diff, 0, sizeof(unsigned long long), s));
    k_count_diff_i32<<<sms * 8, 256, 0, s>>>(out, ref, total, diff);
    GI_TRY(launch_status(1));
    unsigned long long h = 0;
    GI_CUDA(cudaMemcpyAsync(&h, diff, sizeof(h), cudaMemcpyDeviceToHost, s));
    GI_CUDA(cudaStreamSynchronize(s));
    return h ? 1 : 0;
  };
  double t_start = 0.0;
  if (st == GI_OK) st = time_opts(st0, &t_start);
  if (st == GI_OK && cudaMemcpyAsync(ref, out, sizeof(int32_t) * (size_t)total, cudaMemcpyDeviceToDevice, s) !=
                         cudaSuccess)
    st = cuda_fail(cudaGetLastError(), "batch autotune reference", __FILE__, __LINE__);
  const int32_t cs_vals[] = {1, 2, 4, 8}, tw_vals[] = {8, 16, 32}, tc_vals[] = {128, 256, 512, 1024, 4096},
                ord_vals[] = {0, 1};
  const float dl_vals[] = {0.5f, 1.0f, 2.0f, 4.0f, 8.0f};
  auto pos_of = [](const auto *vals, int nv, auto v) {
    for (int i = 0; i < nv; ++i)
      if (vals[i] == v) return i;
    return 0;
  };
  std::mt19937_64 rng(seed);
  gi_batch_opts top = st0;
  double t_top = t_start;
  for (int32_t trial = 1; trial < budget && st == GI_OK; ++trial) {
    gi_batch_opts c = top;
    if (trial < budget / 3) {
      c.cluster_size = cs_vals[rng() % 4];
      c.t_warp = tw_vals[rng() % 3];
      c.t_cta = tc_vals[rng() % 5];
      c.sssp_delta = dl_vals[rng() % 5];
      c.order = ord_vals[rng() % 2];
    } else {
      const int which = (int)(rng() % 5), dirn = (rng() & 1) ? 1 : -1;
      int p;
      switch (which) {
        case 0:
          p = pos_of(cs_vals, 4, c.cluster_size) + dirn;
          if (p < 0 || p >= 4) continue;
          c.cluster_size = cs_vals[p];
          break;
        case 1:
          p = pos_of(tw_vals, 3, c.t_warp) + dirn;
          if (p < 0 || p >= 3) continue;
          c.t_warp = tw_vals[p];
          break;
        case 2:
          p = pos_of(tc_vals, 5, c.t_cta) + dirn;
          if (p < 0 || p >= 5) continue;
          c.t_cta = tc_vals[p];
          break;
        case 3:
          p = pos_of(dl_vals, 5, c.sssp_delta) + dirn;
          if (p < 0 || p >= 5) continue;
          c.sssp_delta = dl_vals[p];
          break;
        default:
          c.order = 1 - c.order;
      }
    }
    if (c.cluster_size == 0) c.cluster_size = 4;
    c.clusters = 0;
    if (c.t_cta < c.t_warp) c.t_cta = c.t_warp;
    double t = 0.0;
    st = time_opts(c, &t);
    if (st != GI_OK) break;
    const int d = differs();
    if (d < 0) {
      st = d;
      break;
    }
    if (d == 0 && t < t_top) {
      top = c;
      t_top = t;
    }
  }
  dev_free(out, s);
  dev_free(ref, s);
  dev_free(diff, s);
  if (st == GI_OK && cudaStreamSynchronize(s) != cudaSuccess)
    st = cuda_fail(cudaGetLastError(), "batch autotune", __FILE__, __LINE__);
  if (st != GI_OK) return st;
  top.levels = start ? start->levels : nullptr;
  top.parents = start ? start->parents : nullptr;
  *best = top;
  if (best_ms) *best_ms = t_top;
  if (start_ms) *start_ms = t_start;
  return GI_OK;
}
