// Edge functions and traversal kernels (templates), shared by the edgeset
// apply entry point and the algorithm drivers.
//
// Directions follow Sec. 2 of the paper: SparsePush iterates the frontier's
// out-edges and updates destinations with atomics; DensePush scans every
// vertex, tests frontier membership and pushes like SparsePush; DensePull
// iterates destinations and reads in-edges, updating its own destination
// without atomics (the dependence rules of Sec. 6).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstddef>
#include <type_traits>

#include "gi_internal.cuh"

namespace gi {

// Where a traversal reports modified destinations (applyModified): the bit is
// set in `bm` and the vertex appended to `q` (count in *qc).  With dedup the
// append happens only for the call that set the bit.
struct OutSet {
  uint32_t *bm = nullptr;
  int32_t *q = nullptr;
  int32_t *qc = nullptr;
  bool dedup = true;
  __device__ __forceinline__ bool enabled() const { return bm != nullptr; }
};

__device__ __forceinline__ void out_mark(const OutSet &o, int32_t v) {
  bool fresh;
  if (o.dedup) {
    fresh = bit_test_and_set(o.bm, v);
  } else {
    atomicOr(o.bm + (v >> 5), 1u << (v & 31));
    fresh = true;
  }
  if (fresh) {
    int32_t pos = atomicAdd(o.qc, 1);
    o.q[pos] = v;
  }
}

__device__ __forceinline__ bool in_set(const uint32_t *bm, int32_t v) { return bm == nullptr || bit_test(bm, v); }

// Frontier as a traversal reads it (configApplyDenseVertexSet): a bitmap
// (bitvector), a boolean map (one byte per vertex), or neither (all vertices).
struct FSet {
  const uint32_t *bm = nullptr;
  const uint8_t *bytes = nullptr;
  __host__ __device__ FSet() {}
  __host__ __device__ FSet(std::nullptr_t) {}
  __host__ __device__ FSet(const uint32_t *b) : bm(b) {}
  __host__ __device__ FSet(const uint8_t *y) : bytes(y) {}
};

__device__ __forceinline__ bool in_set(const FSet &f, int32_t v) {
  if (f.bytes) return __ldg(f.bytes + v) != 0;
  return f.bm == nullptr || bit_test(f.bm, v);
}

// Whole-warp marking when lane l owns destination v0 + l (each destination is
// owned by one thread, so no test-and-set is needed): the ballot is split over
// the (at most two) bitmap words the 32 ids touch, and the queue append is
// one atomicAdd per warp.
__device__ __forceinline__ void mark_consecutive(const OutSet &o, int32_t v0, bool mod) {
  const unsigned ball = __ballot_sync(0xffffffffu, mod);
  if (!ball) return;
  const int lane = threadIdx.x & 31;
  const int32_t w_lo = v0 >> 5, sh = v0 & 31;
  if (lane == 0) {
    const unsigned lo = ball << sh;
    const unsigned hi = sh ? (ball >> (32 - sh)) : 0u;
    if (lo) atomicOr(o.bm + w_lo, lo);
    if (hi) atomicOr(o.bm + w_lo + 1, hi);
  }
  int32_t base = 0;
  if (lane == 0) base = atomicAdd(o.qc, __popc(ball));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (mod) o.q[base + __popc(ball & ((1u << lane) - 1u))] = v0 + lane;
}

// ------------------------------------------------------------ edge functions --
// Each op provides:
//   V, identity(), combine(a,b)         reduction used by pull
//   edge_val(u, e)                      value one selected in-edge contributes
//   finish(v, acc) -> bool              pull epilogue for destination v; true if modified
//   push(u, v, e) -> bool               atomic update for push; true if v modified
//   dst_ok(v)                           dstFilter (true = keep)

struct OpMinInt {  // CC (no weights) and SSSP (weights): x[v] = min(x[v], snap[u] + w)
  using V = int32_t;
  static constexpr bool kIdentityKeeps = true;  // finish(v, identity()) changes nothing
  int32_t *x;
  const int32_t *snap;
  const int32_t *wt;  // pull: in-edge weights; push: out-edge weights (same array for symmetric graphs)
  __device__ static V identity() { return INT32_MAX; }
  __device__ static V combine(V a, V b) { return a < b ? a : b; }
  __device__ V from_src(int32_t s, int32_t e) const {
    // the weight is loaded whatever s is, so its load is issued beside the
    // gather of s instead of after it (a pull round that the direction rule
    // takes uses most weights anyway)
    const int32_t w = wt ? __ldg(wt + e) : 0;
    if (s == INT32_MAX) return INT32_MAX;
    const long long t = (long long)s + w;
    return t < INT32_MAX ? (int32_t)t : INT32_MAX;
  }
  __device__ V edge_val(int32_t u, int32_t e) const { return from_src(__ldg(snap + u), e); }
  __host__ __device__ const int32_t *hot_source() const { return snap; }
  __device__ bool dst_ok(int32_t) const { return true; }
  __device__ bool finish(int32_t v, V acc) const {
    if (acc < x[v]) {
      x[v] = acc;
      return true;
    }
    return false;
  }
  __device__ bool push(int32_t u, int32_t v, int32_t e) const {
    V c = edge_val(u, e);
    if (c >= *(volatile int32_t *)(x + v)) return false;
    return c < atomicMin(x + v, c);
  }
};

// OpMinInt for rounds whose candidates have a floor: none that can lower a
// distance is below max(*bound - bound_off, 0), so rows whose distance is
// already at or below it are not pulled (dst_ok; long rows skip their
// gathers too).  Delta-stepping's heavy rounds: the floor is the bucket's
// end hi (S lies in [hi - delta, hi) and heavy arcs weigh at least delta).
// Light rounds (floor hi - delta) do without: their long rows are few, and
// the per-row test costs more than it saves.
struct OpMinIntBounded : OpMinInt {
  const int32_t *bound;
  int32_t bound_off;
  __device__ bool dst_ok(int32_t v) const {
    const int32_t b = *bound;
    return x[v] > (b > bound_off ? b - bound_off : 0);
  }
};

struct SumCount {
  float s;
  int32_t c;
};

struct OpSum {  // acc[v] += contrib[u]; modified = destinations with a selected in-edge
  using V = SumCount;
  const float *contrib;
  float *acc;
  __device__ static V identity() { return {0.0f, 0}; }
  __device__ static V combine(V a, V b) { return {a.s + b.s, a.c + b.c}; }
  __device__ V edge_val(int32_t u, int32_t) const { return {__ldg(contrib + u), 1}; }
  __device__ bool dst_ok(int32_t) const { return true; }
  __device__ bool finish(int32_t v, V a) const {
    if (a.c > 0) acc[v] += a.s;
    return a.c > 0;
  }
  __device__ bool push(int32_t u, int32_t v, int32_t) const {
    atomicAdd(acc + v, __ldg(contrib + u));
    return true;
  }
};

// Push accumulation for the PageRank drivers: FP64 atomics, because FP32
// atomic accumulation in arbitrary order onto a high in-degree vertex drifts
// beyond the 1e-4 bound (the pull direction sums in a fixed tree order).
struct OpSumPush64 {
  const float *contrib;
  double *acc;
  __device__ bool push(int32_t u, int32_t v, int32_t) const {
    atomicAdd(acc + v, (double)__ldg(contrib + u));
    return false;
  }
};

struct ProbeVal {
  int32_t c;
  unsigned long long s;
};

struct OpProbe {  // count[v] += 1, srcsum[v] += u+1 per selected edge (u,v)
  using V = ProbeVal;
  int32_t *count;
  unsigned long long *srcsum;
  __device__ static V identity() { return {0, 0ull}; }
  __device__ static V combine(V a, V b) { return {a.c + b.c, a.s + b.s}; }
  __device__ V edge_val(int32_t u, int32_t) const { return {1, (unsigned long long)u + 1ull}; }
  __device__ bool dst_ok(int32_t) const { return true; }
  __device__ bool finish(int32_t v, V a) const {
    if (a.c > 0) {
      count[v] += a.c;
      srcsum[v] += a.s;
    }
    return a.c > 0;
  }
  __device__ bool push(int32_t u, int32_t v, int32_t) const {
    atomicAdd(count + v, 1);
    atomicAdd(srcsum + v, (unsigned long long)u + 1ull);
    return true;
  }
};

// PageRank pull with the vertex update fused into the epilogue:
// r = base + d * sum; contrib_out[v] = r / outdeg (or rank_out[v] = r on the last iteration)
struct OpPR {
  using V = float;
  const float *contrib;
  float *contrib_out;
  float *rank_out;
  const float *inv_deg;
  float base, damping;
  __device__ static V identity() { return 0.0f; }
  __device__ static V combine(V a, V b) { return a + b; }
  __device__ V edge_val(int32_t u, int32_t) const { return __ldg(contrib + u); }
  __host__ __device__ const float *hot_source() const { return contrib; }
  __device__ V from_src(float x, int32_t) const { return x; }
  __device__ bool dst_ok(int32_t) const { return true; }
  __device__ bool finish(int32_t v, V s) const {
    float r = fmaf(damping, s, base);
    if (rank_out) rank_out[v] = r;
    else contrib_out[v] = r * __ldg(inv_deg + v);
    return false;
  }
  __device__ bool push(int32_t, int32_t, int32_t) const { return false; }
};

// PageRankDelta pull round with the vertex filter of Fig. 1 fused into the
// epilogue.  contrib[u] = Delta[u]/outdeg(u) for active u and 0 otherwise, so
// the sum over all in-edges equals the sum over frontier sources.
struct OpPRD {
  using V = float;
  const float *contrib;
  float *contrib_out;
  float *rank;
  const float *inv_deg;
  float damping, first_base, inv_n, eps;
  int32_t first_round;
  __device__ static V identity() { return 0.0f; }
  __device__ static V combine(V a, V b) { return a + b; }
  __device__ V edge_val(int32_t u, int32_t) const { return __ldg(contrib + u); }
  __host__ __device__ const float *hot_source() const { return contrib; }
  __device__ V from_src(float x, int32_t) const { return x; }
  __device__ bool dst_ok(int32_t) const { return true; }
  __device__ bool finish(int32_t v, V s) const {
    float delta, r = rank[v];
    if (first_round) {
      delta = fmaf(damping, s, first_base);
      r += delta;
      delta -= inv_n;
    } else {
      delta = damping * s;
      r += delta;
    }
    rank[v] = r;
    bool active = fabsf(delta) > eps * r;
    contrib_out[v] = active ? delta * __ldg(inv_deg + v) : 0.0f;
    return active;
  }
  __device__ bool push(int32_t, int32_t, int32_t) const { return false; }
};

struct OpBFS {  // dstFilter depth[v] == -1; depth[v] = level, parent[v] = min frontier in-neighbour
  int32_t *depth;
  int32_t *parent;
  int32_t level;
  __device__ bool push(int32_t u, int32_t v, int32_t) const {
    int32_t d = *(volatile int32_t *)(depth + v);
    if (d != -1 && d != level) return false;
    bool won = false;
    if (d == -1) {
      int32_t old = atomicCAS(depth + v, -1, level);
      won = (old == -1);
      if (!won && old != level) return false;
    }
    if (parent && u < *(volatile int32_t *)(parent + v)) atomicMin(parent + v, u);
    return won;
  }
};

// ------------------------------------------------------------------ reductions --
template <class V, class Op>
__device__ __forceinline__ V warp_reduce(V x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    V y;
    if constexpr (sizeof(V) == 4) {
      int32_t bits = __shfl_xor_sync(0xffffffffu, *reinterpret_cast<int32_t *>(&x), o);
      y = *reinterpret_cast<V *>(&bits);
    } else if constexpr (sizeof(V) == 8) {
      long long bits = __shfl_xor_sync(0xffffffffu, *reinterpret_cast<long long *>(&x), o);
      y = *reinterpret_cast<V *>(&bits);
    } else {
      static_assert(sizeof(V) == 16, "unsupported reduction type");
      int4 bits = *reinterpret_cast<int4 *>(&x);
      bits.x = __shfl_xor_sync(0xffffffffu, bits.x, o);
      bits.y = __shfl_xor_sync(0xffffffffu, bits.y, o);
      bits.z = __shfl_xor_sync(0xffffffffu, bits.z, o);
      bits.w = __shfl_xor_sync(0xffffffffu, bits.w, o);
      y = *reinterpret_cast<V *>(&bits);
    }
    x = Op::combine(x, y);
  }
  return x;
}

// ------------------------------------------------------------------ tiled pull --
// One block per tile (see TileSet).  Short tiles stage the selected in-edge
// values of all their rows in shared memory with coalesced loads, then reduce
// row by row (a thread per row below 32 arcs, the owning warp above); long
// rows are reduced by the whole block.  Pieces of split rows leave a partial
// value that k_pull_fixup combines in tile order (deterministic).
//
// Memory-level parallelism: each thread issues kBatch index loads, then the
// kBatch dependent gathers, before touching any result, so a tile costs about
// two memory round trips per kBatch arcs per thread instead of two per arc.
constexpr int kBatch = 8;

// Bytes of shared memory one tile reduction stages: the arc values (with
// room for a long row's piece) and the tile's row pointers.
template <class V>
__host__ __device__ constexpr size_t pull_stage_bytes(int tile_edges) {
  return sizeof(V) * (size_t)(tile_edges + tile_edges / kLongRowDiv) + sizeof(int32_t) * (kTileRows + 1);
}

// Loads of the L1-resident hot-source pull: hot values are cached in L1
// (ld.global.ca), cold gathers go to L2 only (ld.global.cg) and the index
// stream is marked evict-first (ld.global.cs), so neither displaces the hot
// lines.  (Measured on R-MAT 22: 0.424 ms against 0.433 ms with
// L1::evict_last / L1::no_allocate hints and 0.457 ms with plain loads.)
template <class T>
__device__ __forceinline__ T ld_hot(const T *p) {
  static_assert(sizeof(T) == 4, "hot values are 4-byte");
  uint32_t v;
  asm("ld.global.ca.b32 %0, [%1];" : "=r"(v) : "l"(p));
  T t;
  __builtin_memcpy(&t, &v, 4);
  return t;
}
template <class T>
__device__ __forceinline__ T ld_cold(const T *p) {
  static_assert(sizeof(T) == 4, "hot values are 4-byte");
  uint32_t v;
  asm("ld.global.cg.b32 %0, [%1];" : "=r"(v) : "l"(p));
  T t;
  __builtin_memcpy(&t, &v, 4);
  return t;
}
__device__ __forceinline__ int32_t ld_stream_i32(const int32_t *p) {
  int32_t v;
  asm("ld.global.cs.s32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

// Where a tile's arc values come from (kMode):
//   kGatherPlain: op.edge_val(u, e) for sources u in F;
//   kGatherHotSmem / kGatherHotL1: F is all vertices and the in-edge sources
//   were remapped by the graph's HotSet; a negative entry ~s reads slot s of
//   the hot sources' values.  kGatherHotL1 reads them from the dense global
//   array hot_g (cached in L1; the other loads bypass L1 or are marked
//   evict-first so they do not evict it).  kGatherHotSmem reads slots below
//   k1 (the hottest, slots being in descending degree) from the block's
//   shared-memory copy hot and the rest from hot_g as kGatherHotL1 does.  An
//   Op with a hot form exposes its per-source 4-byte values (hot_source())
//   and builds the arc value from one (from_src(value, e)).
constexpr int kGatherPlain = 0, kGatherHotSmem = 1, kGatherHotL1 = 2;

template <class Op>
using hot_src_t = std::remove_cv_t<std::remove_pointer_t<decltype(std::declval<const Op &>().hot_source())>>;

template <class Op, int kMode>
struct Gather {
  const Op &op;
  FSet F;
  const float *hot_g;         // 4-byte slots in global memory (the hot modes)
  const float *hot = nullptr; // kGatherHotSmem: slots [0, k1) in shared memory
  int32_t k1 = 0;
  __device__ __forceinline__ int32_t src(const int32_t *p) const {
    if constexpr (kMode != kGatherPlain) return ld_stream_i32(p);
    else return __ldg(p);
  }
  __device__ __forceinline__ typename Op::V hot_val(int32_t u, int32_t e) const {
    using S = hot_src_t<Op>;
    S sv;
    if (u >= 0) sv = ld_cold(op.hot_source() + u);
    else if (kMode == kGatherHotSmem && ~u < k1) sv = reinterpret_cast<const S *>(hot)[~u];
    else sv = ld_hot(reinterpret_cast<const S *>(hot_g) + ~u);
    return op.from_src(sv, e);
  }
};

template <class Op, int kBlock, int kMode>
__device__ __forceinline__ void stage_batch(const Gather<Op, kMode> &G, const int32_t *__restrict__ idx,
                                            int32_t e0, int32_t k0, int32_t ne, typename Op::V *vals) {
  int32_t u[kBatch];
#pragma unroll
  for (int j = 0; j < kBatch; ++j) {
    const int32_t k = k0 + j * kBlock;
    u[j] = k < ne ? G.src(idx + e0 + k) : -1;
  }
#pragma unroll
  for (int j = 0; j < kBatch; ++j) {
    const int32_t k = k0 + j * kBlock;
    if constexpr (kMode != kGatherPlain) {
      if (k < ne) vals[k] = G.hot_val(u[j], e0 + k);
    } else {
      if (k < ne) vals[k] = (u[j] >= 0 && in_set(G.F, u[j])) ? G.op.edge_val(u[j], e0 + k) : Op::identity();
    }
  }
}

// Ops with FP64 sums (kSkipZeroTerms) skip terms whose bits are zero: on
// GB300 an FP64 add costs a slot of the narrow FP64 pipe while the integer
// test does not, and x + 0.0 == x for the non-negative sums they build.
template <class Op, class = void>
struct SkipZeroTerms : std::false_type {};
template <class Op>
struct SkipZeroTerms<Op, std::void_t<decltype(Op::kSkipZeroTerms)>> : std::bool_constant<Op::kSkipZeroTerms> {};

// Ops whose finish() with the identity (no candidate reached the row) changes
// nothing (min reductions): such rows skip finish() and its load of the
// vertex's current value.
template <class Op, class = void>
struct IdentityKeeps : std::false_type {};
template <class Op>
struct IdentityKeeps<Op, std::void_t<decltype(Op::kIdentityKeeps)>> : std::bool_constant<Op::kIdentityKeeps> {};

template <class Op>
__device__ __forceinline__ bool worth_finishing(typename Op::V acc) {
  if constexpr (IdentityKeeps<Op>::value) return acc != Op::identity();
  else return true;
}

// Output marks of one warp whose lanes hold ascending but not consecutive
// vertices (rows of a row-compacted tile set): one atomicOr per distinct
// bitmap word of the marked lanes, one queue append for the warp.
__device__ __forceinline__ void mark_rows(const OutSet &o, int32_t v, bool mod) {
  const unsigned ball = __ballot_sync(0xffffffffu, mod);
  if (!ball) return;
  const int lane = threadIdx.x & 31;
  const int32_t myw = v >> 5;
  unsigned todo = ball;
  while (todo) {
    const int l = __ffs(todo) - 1;
    const int32_t wl = __shfl_sync(0xffffffffu, myw, l);
    const bool mine = mod && myw == wl;
    const unsigned bits = __reduce_or_sync(0xffffffffu, mine ? (1u << (v & 31)) : 0u);
    todo &= ~__ballot_sync(0xffffffffu, mine);
    if (lane == l) atomicOr(o.bm + wl, bits);
  }
  int32_t base = 0;
  if (lane == 0) base = atomicAdd(o.qc, __popc(ball));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (mod) o.q[base + __popc(ball & ((1u << lane) - 1u))] = v;
}

template <class Op>
__device__ __forceinline__ typename Op::V combine_term(typename Op::V acc, typename Op::V x) {
  if constexpr (SkipZeroTerms<Op>::value) {
    static_assert(sizeof(typename Op::V) == 8, "zero-term skipping is for FP64 sums");
    return __double_as_longlong(x) == 0 ? acc : Op::combine(acc, x);
  } else {
    return Op::combine(acc, x);
  }
}

struct BlockSync {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

// Named barrier over the kThreads threads of one group (ids 1..15; 0 is __syncthreads).
template <int kThreads>
struct GroupSync {
  int id;
  __device__ __forceinline__ void operator()() const { asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(kThreads) : "memory"); }
};

// Reduction of tile t by the kBlock threads that call it (tid in [0, kBlock)),
// with `sync` a barrier over exactly those threads.  vals/rp: the group's
// staging area (pull_stage_bytes), s_red: kBlock/32 values.
template <class Op, int kBlock, int kMode, class Sync>
__device__ __forceinline__ void pull_tile(const Gather<Op, kMode> &G, const int4 T, int32_t t,
                                          const int32_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                                          const uint32_t *__restrict__ to, const OutSet &out,
                                          typename Op::V *partial, typename Op::V *vals, int32_t *rp,
                                          typename Op::V *s_red, const int tid, const Sync &sync,
                                          const int32_t *__restrict__ rows = nullptr) {
  using V = typename Op::V;
  const Op &op = G.op;
  const int lane = tid & 31, warp = tid >> 5;
  if (T.y > T.x) {
    // short tile: rows [r0, r0+R), arcs [T.z, T.w) = [ptr[r0], ptr[r0+R]).  The
    // row pointers and the arc sources are loaded together (one round trip),
    // then the gathers; one barrier before the row reductions.
    const int32_t r0 = T.x, R = T.y - T.x, e0 = T.z, ne = T.w - T.z;
    constexpr int kRp = (kTileRows + 1 + kBlock - 1) / kBlock;
    int32_t p[kRp];
#pragma unroll
    for (int j = 0; j < kRp; ++j) {
      const int i = tid + j * kBlock;
      p[j] = i <= R ? __ldg(ptr + r0 + i) : 0;
    }
    for (int32_t k0 = tid; k0 < ne; k0 += kBatch * kBlock) stage_batch<Op, kBlock, kMode>(G, idx, e0, k0, ne, vals);
#pragma unroll
    for (int j = 0; j < kRp; ++j) {
      const int i = tid + j * kBlock;
      if (i <= R) rp[i] = p[j];
    }
    sync();
    for (int i0 = 0; i0 < R; i0 += kBlock) {
      const int i = i0 + tid;
      const int32_t v = rows ? (i < R ? __ldg(rows + r0 + i) : -1) : r0 + i;
      // rows the destination filters reject are not reduced at all
      const bool want = i < R && in_set(to, v) && op.dst_ok(v);
      int32_t a = 0, b = 0;
      if (want) {
        a = rp[i] - e0;
        b = rp[i + 1] - e0;
      }
      const bool big = want && (b - a) >= 32;
      V acc = Op::identity();
      if (want && !big)
        for (int32_t k = a; k < b; ++k) acc = combine_term<Op>(acc, vals[k]);
      unsigned bal = __ballot_sync(0xffffffffu, big);
      while (bal) {
        const int l = __ffs(bal) - 1;
        bal &= bal - 1;
        const int32_t la = __shfl_sync(0xffffffffu, a, l), lb = __shfl_sync(0xffffffffu, b, l);
        V x = Op::identity();
        for (int32_t k = la + lane; k < lb; k += 32) x = combine_term<Op>(x, vals[k]);
        x = warp_reduce<V, Op>(x);
        if (lane == l) acc = x;
      }
      bool mod = false;
      if (want && worth_finishing<Op>(acc)) mod = op.finish(v, acc);
      if (out.enabled()) {
        if (rows) mark_rows(out, v, mod);
        else mark_consecutive(out, r0 + i0 + (tid & ~31), mod);
      }
    }
    sync();
  } else {
    // one long row (or a piece of it): nothing to gather when its destination is filtered out
    const int32_t r = T.x, e0 = T.z;
    const int32_t vr = rows ? __ldg(rows + r) : r;
    const int32_t ne = (in_set(to, vr) && op.dst_ok(vr)) ? T.w - T.z : 0;
    V x = Op::identity();
    for (int32_t k0 = tid; k0 < ne; k0 += kBatch * kBlock) {
      int32_t u[kBatch];
#pragma unroll
      for (int j = 0; j < kBatch; ++j) {
        const int32_t k = k0 + j * kBlock;
        u[j] = k < ne ? G.src(idx + e0 + k) : -1;
      }
#pragma unroll
      for (int j = 0; j < kBatch; ++j) {
        if constexpr (kMode != kGatherPlain) {
          if (k0 + j * kBlock < ne) x = Op::combine(x, G.hot_val(u[j], e0 + k0 + j * kBlock));
        } else {
          if (u[j] >= 0 && in_set(G.F, u[j])) x = combine_term<Op>(x, op.edge_val(u[j], e0 + k0 + j * kBlock));
        }
      }
    }
    x = warp_reduce<V, Op>(x);
    if (lane == 0) s_red[warp] = x;
    sync();
    if (tid == 0) {
      V y = Op::identity();
      for (int w = 0; w < kBlock / 32; ++w) y = Op::combine(y, s_red[w]);
      if (T.y == r) {
        if (ne > 0 && worth_finishing<Op>(y) && op.finish(vr, y) && out.enabled()) out_mark(out, vr);
      } else {
        partial[t] = y;
      }
    }
    sync();
  }
}

template <class Op, int kBlock, int kTE, int kMode = kGatherPlain>
__global__ void __launch_bounds__(kBlock) k_pull_tiled(Op op, const int32_t *__restrict__ ptr,
                                                       const int32_t *__restrict__ idx, const int4 *__restrict__ tiles,
                                                       int32_t num_tiles, FSet F,
                                                       const uint32_t *__restrict__ to, OutSet out,
                                                       typename Op::V *partial, const float *__restrict__ hot,
                                                       const int32_t *__restrict__ rows) {
  using V = typename Op::V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V *vals = reinterpret_cast<V *>(smem_raw);
  int32_t *rp = reinterpret_cast<int32_t *>(smem_raw + sizeof(V) * (size_t)(kTE + kTE / kLongRowDiv));
  __shared__ V s_red[kBlock / 32];
  static_assert(kMode == kGatherPlain || kMode == kGatherHotL1, "k_pull_tiled: plain or L1-hot gathers");
  const Gather<Op, kMode> G{op, F, hot};
  for (int32_t t = blockIdx.x; t < num_tiles; t += gridDim.x)
    pull_tile<Op, kBlock, kMode>(G, tiles[t], t, ptr, idx, to, out, partial, vals, rp, s_red, threadIdx.x,
                                 BlockSync{}, rows);
}

// Hot-source pull (GPU form of the cache partitioning of Sec. 2) with a
// two-level cache: two persistent blocks of kGroups x 256 threads per SM
// (the plain kernel's warp count) each copy the k1 hottest slots of the
// HotSet (as many as fit beside the groups' staging areas) into shared
// memory; the remaining hot slots are read through L1 from the dense hot
// array and the cold sources from L2, as in the L1 form.  Each 256-thread
// group reduces every (gridDim.x*kGroups)-th tile with the same tile
// algorithm as k_pull_tiled, synchronised by its own named barrier, so the
// tiles and the order of every reduction are those of k_pull_tiled and the
// results are bit-identical to it.
template <class Op, int kTE, int kGroups>
__global__ void __launch_bounds__(256 * kGroups, 2) k_pull_hot(Op op, const int32_t *__restrict__ ptr,
                                                               const int32_t *__restrict__ hidx,
                                                               const int4 *__restrict__ tiles, int32_t num_tiles,
                                                               const float *__restrict__ hot_vals, int32_t k1,
                                                               const uint32_t *__restrict__ to, OutSet out,
                                                               typename Op::V *partial) {
  using V = typename Op::V;
  static_assert(sizeof(hot_src_t<Op>) == 4, "hot slots are 4-byte");
  static_assert(kGroups >= 1 && kGroups <= 4, "named barriers 1..kGroups");
  constexpr int kB = 256;
  constexpr size_t kStage = (pull_stage_bytes<V>(kTE) + 15) & ~(size_t)15;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float *s_hot = reinterpret_cast<float *>(smem_raw);
  {
    const float4 *src4 = reinterpret_cast<const float4 *>(hot_vals);
    float4 *dst4 = reinterpret_cast<float4 *>(s_hot);
    for (int i = threadIdx.x; i < k1 / 4; i += blockDim.x) dst4[i] = __ldg(src4 + i);
  }
  __syncthreads();
  __shared__ V s_red[kGroups][kB / 32];
  const int grp = threadIdx.x / kB;
  unsigned char *stage = smem_raw + sizeof(float) * (size_t)k1 + kStage * grp;
  V *vals = reinterpret_cast<V *>(stage);
  int32_t *rp = reinterpret_cast<int32_t *>(stage + sizeof(V) * (size_t)(kTE + kTE / kLongRowDiv));
  Gather<Op, kGatherHotSmem> G{op, FSet(), hot_vals};
  G.hot = s_hot;
  G.k1 = k1;
  const GroupSync<kB> sync{1 + grp};
  const int32_t stride = (int32_t)gridDim.x * kGroups;
  for (int32_t t = (int32_t)blockIdx.x * kGroups + grp; t < num_tiles; t += stride)
    pull_tile<Op, kB, kGatherHotSmem>(G, tiles[t], t, ptr, hidx, to, out, partial, vals, rp, s_red[grp],
                                      (int)(threadIdx.x % kB), sync);
}

// hot_vals[s] = values[src[s]]: the hot sources' values for one launch
template <class S>
static __global__ void k_hot_gather(const S *__restrict__ contrib, const int32_t *__restrict__ src, int32_t k,
                                    S *__restrict__ vals) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < k) vals[i] = __ldg(contrib + __ldg(src + i));
}

// Warp tiles (tile_edges = 256): every warp owns whole tiles and no block
// barrier is ever taken, so the SM overlaps the memory latency of up to 64
// independent warps.  A short warp tile holds <= 64 complete rows of <= 128
// arcs and < 384 arcs in all: the lanes stage the arc values (12 index loads,
// then 12 gathers, per lane) in the warp's shared-memory slice, then each lane
// sums its rows serially.  Long-row pieces (<= 256 arcs) are reduced across
// the warp.  Split rows leave partials for k_pull_fixup as with block tiles.
constexpr int kWarpsPerBlock = 8;

template <class Op>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) k_pull_warp(Op op, const int32_t *__restrict__ ptr,
                                                                   const int32_t *__restrict__ idx,
                                                                   const int4 *__restrict__ tiles, int32_t num_tiles,
                                                                   FSet F,
                                                                   const uint32_t *__restrict__ to, OutSet out,
                                                                   typename Op::V *partial) {
  using V = typename Op::V;
  constexpr int kCap = kWarpTileEdges + kWarpTileEdges / kLongRowDiv;
  constexpr int kPer = kCap / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  V *wb = reinterpret_cast<V *>(smem_raw) + warp * kCap;
  const int32_t stride = gridDim.x * kWarpsPerBlock;
  for (int32_t t = blockIdx.x * kWarpsPerBlock + warp; t < num_tiles; t += stride) {
    const int4 T = tiles[t];
    if (T.y > T.x) {
      const int32_t r0 = T.x, R = T.y - T.x, e0 = T.z, ne = T.w - T.z;
      // row bounds of this lane's rows (issued before the arc loads)
      int32_t ra[kWarpTileRows / 32], rb[kWarpTileRows / 32];
#pragma unroll
      for (int j = 0; j < kWarpTileRows / 32; ++j) {
        const int i = lane + 32 * j;
        ra[j] = i < R ? __ldg(ptr + r0 + i) - e0 : 0;
        rb[j] = i < R ? __ldg(ptr + r0 + i + 1) - e0 : 0;
      }
      int32_t u[kPer];
#pragma unroll
      for (int j = 0; j < kPer; ++j) {
        const int32_t k = lane + 32 * j;
        u[j] = k < ne ? __ldg(idx + e0 + k) : -1;
      }
#pragma unroll
      for (int j = 0; j < kPer; ++j) {
        const int32_t k = lane + 32 * j;
        if (k < ne) wb[k] = (u[j] >= 0 && in_set(F, u[j])) ? op.edge_val(u[j], e0 + k) : Op::identity();
      }
      __syncwarp();
#pragma unroll
      for (int j = 0; j < kWarpTileRows / 32; ++j) {
        if (32 * j >= R) break;
        const int i = lane + 32 * j;
        const bool valid = i < R;
        V acc = Op::identity();
        if (valid)
          for (int32_t k = ra[j]; k < rb[j]; ++k) acc = Op::combine(acc, wb[k]);
        const int32_t v = r0 + i;
        bool mod = false;
        if (valid && in_set(to, v) && op.dst_ok(v)) mod = op.finish(v, acc);
        if (out.enabled()) mark_consecutive(out, r0 + 32 * j, mod);
      }
      __syncwarp();
    } else {
      const int32_t r = T.x, e0 = T.z, ne = T.w - T.z;
      V x = Op::identity();
      for (int32_t k0 = lane; k0 < ne; k0 += 32 * kBatch) {
        int32_t uu[kBatch];
#pragma unroll
        for (int j = 0; j < kBatch; ++j) {
          const int32_t k = k0 + 32 * j;
          uu[j] = k < ne ? __ldg(idx + e0 + k) : -1;
        }
#pragma unroll
        for (int j = 0; j < kBatch; ++j)
          if (uu[j] >= 0 && in_set(F, uu[j])) x = Op::combine(x, op.edge_val(uu[j], e0 + k0 + 32 * j));
      }
      x = warp_reduce<V, Op>(x);
      if (lane == 0) {
        if (T.y == r) {
          if (in_set(to, r) && op.dst_ok(r) && op.finish(r, x) && out.enabled()) out_mark(out, r);
        } else {
          partial[t] = x;
        }
      }
    }
  }
}

// Vertex-parallel DensePull (configApplyParallelization's vertex-parallel
// mode): one thread per destination, in-edges scanned serially with 4 loads in
// flight.  Consecutive destinations sit in consecutive lanes, so the modified
// set is marked one bitmap word per warp.
template <class Op>
__global__ void __launch_bounds__(256) k_pull_vertex(Op op, const int32_t *__restrict__ ptr,
                                                     const int32_t *__restrict__ idx, int64_t n,
                                                     FSet F, const uint32_t *__restrict__ to,
                                                     OutSet out) {
  using V = typename Op::V;
  const int64_t nw = (n + 31) >> 5;
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nw;
       w += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t v = w * 32 + (threadIdx.x & 31);
    bool mod = false;
    if (v < n && in_set(to, (int32_t)v) && op.dst_ok((int32_t)v)) {
      const int32_t a = __ldg(ptr + v), b = __ldg(ptr + v + 1);
      V acc = Op::identity();
      for (int32_t e = a; e < b; e += 4) {
        int32_t u[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) u[j] = e + j < b ? __ldg(idx + e + j) : -1;
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (u[j] >= 0 && in_set(F, u[j])) acc = Op::combine(acc, op.edge_val(u[j], e + j));
      }
      mod = op.finish((int32_t)v, acc);
    }
    if (out.enabled()) mark_consecutive(out, (int32_t)(w * 32), mod);
  }
}

template <class Op>
__global__ void k_pull_fixup(Op op, const int4 *__restrict__ splits, int32_t num_splits,
                             const typename Op::V *__restrict__ partial, const uint32_t *__restrict__ to, OutSet out,
                             const int32_t *__restrict__ rows = nullptr) {
  using V = typename Op::V;
  for (int32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < num_splits; s += gridDim.x * blockDim.x) {
    const int4 S = splits[s];
    const int32_t v = rows ? __ldg(rows + S.x) : S.x;
    V y = Op::identity();
    for (int32_t k = 0; k < S.z; ++k) y = Op::combine(y, partial[S.y + k]);
    if (in_set(to, v) && op.dst_ok(v) && worth_finishing<Op>(y) && op.finish(v, y) && out.enabled())
      out_mark(out, v);
  }
}

// Instrumentation (gi_stats_pull_arcs): the arcs the block tiles will gather,
// by pull_tile's rules -- every arc of a short tile, a long row's arcs only
// if its destination passes the filters -- evaluated before the pull changes
// any distance; one atomic per block.
template <class Op>
__global__ void k_pull_count(Op op, const int4 *__restrict__ tiles, int32_t num_tiles, const int32_t *__restrict__ rows,
                             const uint32_t *__restrict__ to, unsigned long long *ctr) {
  unsigned long long c = 0;
  for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < num_tiles; t += gridDim.x * blockDim.x) {
    const int4 T = tiles[t];
    if (T.y > T.x) {
      c += (unsigned long long)(T.w - T.z);
    } else {
      const int32_t vr = rows ? __ldg(rows + T.x) : T.x;
      if (in_set(to, vr) && op.dst_ok(vr)) c += (unsigned long long)(T.w - T.z);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  __shared__ unsigned long long s_c[8];
  if ((threadIdx.x & 31) == 0) s_c[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += s_c[w];
    if (b) atomicAdd(ctr, b);
  }
}

// ------------------------------------------------------------- BFS pull ------
// DensePull for BFS with early exit (Sec. 2): a warp owns 32 destinations.
// Unvisited destinations scan their in-neighbours in ascending order and
// stop at the first frontier member, which is the smallest-id parent.  Rows
// with at least t_warp arcs are scanned by the whole warp 32 arcs at a time
// (ballot picks the first hit).  The destinations are either all vertices
// (32 consecutive ones per warp: one output bitmap word) or, with U.st set,
// the entries of the compacted unvisited list (BfsUnv): then the vertices
// left unvisited are appended to the other list, and the found ones set
// their output bits by one atomicOr per distinct word of the warp.
static __global__ void __launch_bounds__(256) k_pull_bfs(const int32_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                                                  int64_t n, FSet F,
                                                  const uint32_t *__restrict__ to, int32_t *depth, int32_t *parent,
                                                  int32_t level, int32_t t_warp, uint32_t *out_bm, int32_t *out_q,
                                                  int32_t *out_qc, const int32_t *gm = nullptr,
                                                  void *defer = nullptr, int32_t defer_cap = 0,
                                                  BfsUnv U = BfsUnv{}) {
  if (gm) {  // graph-driven level: run only when this level pulls
    if (gm[kGmPull] == 0) return;
    level = gm[kGmLevel] + 1;
  }
  // found vertices are staged per warp in shared memory and appended to the
  // queue kQBuf - 32 or more at a time: one atomic per flush, not one per
  // 32 vertices, and no wait on its return in every iteration; so are the
  // vertices left for the next pull level (listed walk)
  constexpr int kQBuf = 128;
  __shared__ int32_t s_q[8][kQBuf];  // blockDim.x == 256
  __shared__ int32_t s_u[8][kQBuf];
  const int lane = threadIdx.x & 31;
  int32_t *wq = s_q[threadIdx.x >> 5];
  int32_t *wu = s_u[threadIdx.x >> 5];
  int32_t qn = 0, un = 0;  // staged entries (warp-uniform)
  const auto flush = [&](int32_t *buf, int32_t cnt, int32_t *dst, int32_t *dst_count) {
    __syncwarp();
    int32_t base = 0;
    if (lane == 0) base = atomicAdd(dst_count, cnt);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (int32_t j = lane; j < cnt; j += 32) dst[base + j] = buf[j];
    __syncwarp();
  };
  // the walk: every vertex, or the input list of the compacted walk
  const bool listed = U.st != nullptr;
  int32_t cur = -1;
  const int32_t *in_list = nullptr;
  int32_t *next_list = nullptr, *next_count = nullptr;
  int64_t items = n;
  if (listed) {
    cur = U.st[0];
    in_list = cur < 0 ? U.live : (cur == 0 ? U.list0 : U.list1);
    items = cur < 0 ? U.nlive : U.st[1 + cur];
    next_list = cur == 0 ? U.list1 : U.list0;
    next_count = U.st + (cur == 0 ? 2 : 1);
  }
  const int64_t nw = (items + 31) >> 5;
  const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
  // the vertex, depth word and row bounds of the warp's next 32 entries are
  // loaded while the current ones are probed (one round trip per iteration fewer)
  int32_t nv = -1, ndv = 0, na = 0, nb = 0;
  const auto fetch = [&](int64_t ww) {
    const int64_t ii = ww * 32 + lane;
    nv = -1;
    if (ww < nw && ii < items) {
      nv = listed ? in_list[ii] : (int32_t)ii;
      ndv = depth[nv];
      na = __ldg(ptr + nv);
      nb = __ldg(ptr + nv + 1);
    }
  };
  int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  fetch(w);
  for (; w < nw; w += wstride) {
    const int32_t v = nv;
    const int32_t dv = ndv;
    int32_t a = na, b = nb;
    fetch(w + wstride);
    const bool active = v >= 0 && dv == -1 && in_set(to, v);
    if (!active) b = a;
    int32_t found = -1;
    // every lane first probes the first 4 arcs of its own row: 4 independent
    // index loads, then 4 independent frontier-bit loads; the first hit in
    // order is the min id.  Rows of fewer than t_warp arcs go on 4 at a time;
    // longer rows without a hit in the probe are scanned by the whole warp.
    for (int32_t e = a; e < b && found < 0; e += 4) {
      int32_t u[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) u[j] = e + j < b ? __ldg(idx + e + j) : -1;
      bool h[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) h[j] = u[j] >= 0 && in_set(F, u[j]);
#pragma unroll
      for (int j = 3; j >= 0; --j)
        if (h[j]) found = u[j];
      if (b - a >= t_warp) break;
    }
    const bool big = active && found < 0 && (b - a) >= t_warp;
    unsigned bal = __ballot_sync(0xffffffffu, big);
    while (bal) {
      const int l = __ffs(bal) - 1;
      bal &= bal - 1;
      // the probe covered [a, a + 4)
      const int32_t lb = __shfl_sync(0xffffffffu, b, l), la0 = __shfl_sync(0xffffffffu, a, l);
      const int32_t la = la0 + (lb - la0 < 4 ? lb - la0 : 4);
      // a long row is scanned here for kBfsScanCap arcs at most; the rest,
      // if no frontier source turned up, is left to every block
      const int32_t stop = (defer != nullptr && lb - la > kBfsScanCap + kBfsDeferChunk) ? la + kBfsScanCap : lb;
      int32_t hit = -1;
      for (int32_t base = la; base < stop; base += 32) {
        const int32_t e = base + lane;
        int32_t u = e < stop ? __ldg(idx + e) : 0;
        unsigned h = __ballot_sync(0xffffffffu, e < stop && in_set(F, u));
        if (h) {
          hit = __shfl_sync(0xffffffffu, u, __ffs(h) - 1);
          break;
        }
      }
      if (hit < 0 && stop < lb && lane == l) {
        const BfsDefer D = bfs_defer_at(defer, defer_cap);
        const unsigned nch = (unsigned)((lb - stop + kBfsDeferChunk - 1) / kBfsDeferChunk);
        const unsigned long long old = atomicAdd(D.ctr, (1ull << 32) | nch);
        const int32_t j = (int32_t)(old >> 32);
        if (j < defer_cap) {  // always: each queued row holds more than m / defer_cap arcs
          D.row[j] = v;
          D.from[j] = stop;
          D.base[j] = (int32_t)(old & 0xffffffffull);
          D.best[j] = INT32_MAX;
        }
      }
      if (lane == l) found = hit;
    }
    const bool got = found >= 0;
    if (got) {
      depth[v] = level;
      if (parent) parent[v] = found;
    }
    if (listed) {
      // still unvisited (not reached, filtered out by `to`, or deferred):
      // walked again at the next pull level
      const bool keep = v >= 0 && dv == -1 && !got;
      const unsigned kw = __ballot_sync(0xffffffffu, keep);
      if (kw) {
        if (keep) wu[un + __popc(kw & ((1u << lane) - 1u))] = v;
        un += __popc(kw);
        if (un > kQBuf - 32) {
          flush(wu, un, next_list, next_count);
          un = 0;
        }
      }
    }
    const unsigned word = __ballot_sync(0xffffffffu, got);
    if (out_bm == nullptr || word == 0) continue;
    if (!listed) {
      if (lane == 0) out_bm[w] |= word;
    } else {
      // one atomicOr per distinct bitmap word among the found lanes
      const int32_t myw = v >> 5;
      unsigned todo = word;
      while (todo) {
        const int l = __ffs(todo) - 1;
        const int32_t wl = __shfl_sync(0xffffffffu, myw, l);
        const bool mine = got && myw == wl;
        const unsigned bits = __reduce_or_sync(0xffffffffu, mine ? (1u << (v & 31)) : 0u);
        todo &= ~__ballot_sync(0xffffffffu, mine);
        if (lane == l) atomicOr(out_bm + wl, bits);
      }
    }
    if (got) wq[qn + __popc(word & ((1u << lane) - 1u))] = v;
    qn += __popc(word);
    if (qn > kQBuf - 32) {
      flush(wq, qn, out_q, out_qc);
      qn = 0;
    }
  }
  if (out_bm != nullptr && qn > 0) flush(wq, qn, out_q, out_qc);
  if (!listed) return;
  if (un > 0) flush(wu, un, next_list, next_count);
  // the last block to finish makes the list just written the next input and
  // empties the one just read (every block has read the state before its ticket)
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(U.st + 3, 1) == (int32_t)gridDim.x - 1) {
      __threadfence();
      const int32_t nxt = cur == 0 ? 1 : 0;
      U.st[0] = nxt;
      U.st[1 + (nxt ^ 1)] = 0;
      U.st[3] = 0;
      __threadfence();
    }
  }
}

// The deferred rows of k_pull_bfs: block task c is chunk c of the queue (the
// last entry whose first chunk is <= c), kBfsDeferChunk arcs, 8 per thread.
// A chunk that starts after a hit already recorded for its row is skipped;
// otherwise the chunk's first frontier source (lowest position) goes into
// best[row] by atomicMin, so best ends as the row's first hit in order, the
// min-id parent.  The last block to finish writes depth / parent / output
// set for the rows that hit and empties the queue for the next level (every
// block has read the counter before it takes its ticket).
static __global__ void __launch_bounds__(256) k_pull_bfs_deferred(const int32_t *__restrict__ ptr,
                                                           const int32_t *__restrict__ idx, FSet F, void *defer,
                                                           int32_t defer_cap, int32_t *depth, int32_t *parent,
                                                           int32_t level, uint32_t *out_bm, int32_t *out_q,
                                                           int32_t *out_qc) {
  constexpr int kPer = kBfsDeferChunk / 256;
  const BfsDefer D = bfs_defer_at(defer, defer_cap);
  const unsigned long long c64 = *(volatile unsigned long long *)D.ctr;
  const int32_t H = (int32_t)(c64 >> 32) < defer_cap ? (int32_t)(c64 >> 32) : defer_cap;
  const int32_t C = (int32_t)(c64 & 0xffffffffull);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  __shared__ int32_t s_j, s_from, s_end, s_min[8];
  __shared__ bool s_last;
  for (int32_t c = blockIdx.x; c < C; c += gridDim.x) {
    if (tid == 0) {
      int32_t lo = 0, hi = H - 1;
      while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (D.base[mid] <= c) lo = mid;
        else hi = mid - 1;
      }
      const int32_t from = D.from[lo] + (c - D.base[lo]) * kBfsDeferChunk;
      const int32_t end = __ldg(ptr + D.row[lo] + 1);
      s_j = lo;
      s_from = from;
      // chunk ends and arc positions in 64 bits: from + kBfsDeferChunk may pass
      // INT32_MAX on graphs with m close to 2^31
      s_end = *(volatile int32_t *)(D.best + lo) < from
                  ? from
                  : (int32_t)min((int64_t)from + kBfsDeferChunk, (int64_t)end);
    }
    __syncthreads();
    const int32_t from = s_from, end = s_end;
    int32_t u[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int64_t e = (int64_t)from + tid + 256 * k;
      u[k] = e < end ? __ldg(idx + e) : -1;
    }
    int32_t mine = INT32_MAX;
#pragma unroll
    for (int k = kPer - 1; k >= 0; --k)
      if (u[k] >= 0 && in_set(F, u[k])) mine = (int32_t)((int64_t)from + tid + 256 * k);  // < end <= m
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mine = min(mine, __shfl_xor_sync(0xffffffffu, mine, o));
    if (lane == 0) s_min[warp] = mine;
    __syncthreads();
    if (tid == 0) {
      int32_t y = s_min[0];
      for (int w = 1; w < 8; ++w) y = min(y, s_min[w]);
      if (y < INT32_MAX) atomicMin(D.best + s_j, y);
    }
    __syncthreads();
  }
  if (tid == 0) {
    __threadfence();
    s_last = atomicAdd(D.ticket, 1) == (int32_t)gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int32_t j = tid; j < H; j += blockDim.x) {
    const int32_t pos = *(volatile int32_t *)(D.best + j);
    if (pos == INT32_MAX) continue;
    const int32_t v = D.row[j], u = __ldg(idx + pos);
    depth[v] = level;
    if (parent) parent[v] = u;
    if (out_bm) {
      atomicOr(out_bm + (v >> 5), 1u << (v & 31));
      out_q[atomicAdd(out_qc, 1)] = v;
    }
  }
  __syncthreads();
  if (tid == 0) {
    *D.ctr = 0ull;
    *D.ticket = 0;
    __threadfence();
  }
}

// ------------------------------------------------------------------- push ------

// A batch of N candidate arcs (u[j] -> v[j], arc e[j]; v[j] < 0: none): all
// N updates first, then all dedup tests, then one warp-aggregated append to
// the output queue.  Taken arc by arc, a ballot and two atomics whose results
// are waited for stood between consecutive updates, so the updates of one
// batch never overlapped.
template <int N, class Op>
__device__ __forceinline__ void push_batch(const Op &op, const int32_t (&u)[N], const int32_t (&v)[N],
                                           const int32_t (&e)[N], const uint32_t *__restrict__ to,
                                           const OutSet &out) {
  bool mod[N];
#pragma unroll
  for (int j = 0; j < N; ++j) mod[j] = v[j] >= 0 && in_set(to, v[j]) && op.push(u[j], v[j], e[j]);
  if (!out.enabled()) return;
  bool fresh[N];
#pragma unroll
  for (int j = 0; j < N; ++j) {
    fresh[j] = false;
    if (mod[j]) {
      if (out.dedup) {
        fresh[j] = bit_test_and_set(out.bm, v[j]);
      } else {
        atomicOr(out.bm + (v[j] >> 5), 1u << (v[j] & 31));
        fresh[j] = true;
      }
    }
  }
  const unsigned act = __activemask();
  unsigned ball[N];
  int32_t tot = 0;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    ball[j] = __ballot_sync(act, fresh[j]);
    tot += __popc(ball[j]);
  }
  if (tot == 0) return;
  const int lane = lane_id(), leader = __ffs(act) - 1;
  int32_t base = 0;
  if (lane == leader) base = atomicAdd(out.qc, tot);
  base = __shfl_sync(act, base, leader);
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    if (fresh[j]) out.q[base + __popc(ball[j] & lt)] = v[j];
    base += __popc(ball[j]);
  }
}

// arcs [a + k0, a + k0 + step, ...) of source u: kPushBatch destination loads
// in flight before the updates
constexpr int kPushBatch = 4;

template <class Op>
__device__ __forceinline__ void push_strided(const Op &op, int32_t u, int32_t a, int32_t deg, int32_t k0,
                                             int32_t step, const int32_t *__restrict__ idx,
                                             const uint32_t *__restrict__ to, const OutSet &out) {
  for (int32_t k = k0; k < deg; k += kPushBatch * step) {
    int32_t uu[kPushBatch], v[kPushBatch], e[kPushBatch];
#pragma unroll
    for (int j = 0; j < kPushBatch; ++j) {
      uu[j] = u;
      e[j] = a + k + j * step;
      v[j] = (k + j * step < deg) ? __ldg(idx + e[j]) : -1;
    }
    push_batch(op, uu, v, e, to, out);
  }
}

__device__ __forceinline__ int32_t block_excl_scan(int32_t v, int32_t *total, int32_t *sw) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sw[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int32_t w = lane < nw ? sw[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) sw[lane] = w;
  }
  __syncthreads();
  const int32_t off = (warp > 0 ? sw[warp - 1] : 0) + x - v;
  *total = sw[nw - 1];
  __syncthreads();
  return off;
}

// Push from a frontier given as a queue (SparsePush), a bitmap scanned over
// all vertices (DensePush) or all vertices (from = all).  Load balance
// (edge-aware mode, after Merrill et al.'s scan-based gathering): sources with
// >= t_cta arcs are expanded by the whole block, >= t_warp by their warp; the
// arcs of the remaining sources of the block are laid out back to back in
// shared memory (an owner byte per arc) and expanded one arc per thread.
// Vertex-parallel mode (t_warp = t_cta = INT32_MAX) expands each source's
// arcs serially in its own thread.
enum SrcMode { kSrcQueue = 0, kSrcBitmap = 1, kSrcAll = 2 };
constexpr int kPushBlock = 256;
constexpr int32_t kHeavyChunk = 4096;  // arcs per chunk of a deferred high-degree source
constexpr int kMaxTWarp = 64;  // owner table holds kPushBlock * (kMaxTWarp - 1) arcs

// Owner table of the scan-based gathering: one entry per arc of the block's
// small sources (below t_warp arcs each); 512-thread blocks need 16-bit owners
// and hold sources below 32 arcs, to stay within 48 KB of shared memory.
template <int kBlock>
struct PushOwners {
  using T = std::conditional_t<(kBlock > 256), uint16_t, uint8_t>;
  static constexpr int kMaxTW = kBlock > 256 ? 32 : kMaxTWarp;
};

template <class Op, int kMode, int kBlock = kPushBlock>
__global__ void __launch_bounds__(kBlock) k_push(Op op, const int32_t *__restrict__ ptr,
                                                     const int32_t *__restrict__ idx, const int32_t *__restrict__ q,
                                                     const int32_t *__restrict__ qcount, FSet Fbm, int64_t n,
                                                     const uint32_t *__restrict__ to, OutSet out, int32_t t_warp,
                                                     int32_t t_cta, int32_t t_heavy, void *heavy_mem) {
  __shared__ int32_t s_owner, s_u, s_a, s_deg;
  __shared__ int32_t s_src[kBlock], s_beg[kBlock], s_off[kBlock], s_sw[32];
  using Own = typename PushOwners<kBlock>::T;
  __shared__ Own s_own[kBlock * (PushOwners<kBlock>::kMaxTW - 1)];
  const int tid = threadIdx.x, lane = tid & 31;
  const bool fine = t_warp <= PushOwners<kBlock>::kMaxTW;  // scan-based gathering of small sources
  const int64_t total = (kMode == kSrcQueue) ? (int64_t)(*qcount) : n;
  for (int64_t base = (int64_t)blockIdx.x * kBlock; base < total; base += (int64_t)gridDim.x * kBlock) {
    const int64_t i = base + tid;
    int32_t u = -1, a = 0, deg = 0;
    if (i < total) {
      if (kMode == kSrcQueue) u = q[i];
      else if (kMode == kSrcBitmap) u = in_set(Fbm, (int32_t)i) ? (int32_t)i : -1;
      else u = (int32_t)i;
      if (u >= 0) {
        a = __ldg(ptr + u);
        deg = __ldg(ptr + u + 1) - a;
      }
    }
    // the largest sources are expanded afterwards by every block (k_push_heavy)
    if (deg >= t_heavy) {
      const HeavyList heavy = heavy_at(heavy_mem, n);
      const unsigned nch = (unsigned)((deg + kHeavyChunk - 1) / kHeavyChunk);
      const unsigned long long old = atomicAdd(heavy.ctr, (1ull << 32) | nch);
      const int32_t j = (int32_t)(old >> 32);
      heavy.src[j] = u;
      heavy.base[j] = (int32_t)(old & 0xffffffffull);
      deg = 0;
    }
    // block-cooperative expansion of very high-degree sources
    while (true) {
      if (tid == 0) s_owner = -1;
      __syncthreads();
      if (deg >= t_cta) s_owner = tid;
      __syncthreads();
      const int owner = s_owner;
      if (owner < 0) break;
      if (tid == owner) {
        s_u = u;
        s_a = a;
        s_deg = deg;
        deg = 0;
      }
      __syncthreads();
      push_strided(op, s_u, s_a, s_deg, tid, kBlock, idx, to, out);
      __syncthreads();
    }
    // warp-cooperative expansion
    while (true) {
      unsigned bal = __ballot_sync(0xffffffffu, deg >= t_warp);
      if (!bal) break;
      const int l = __ffs(bal) - 1;
      const int32_t wu = __shfl_sync(0xffffffffu, u, l), wa = __shfl_sync(0xffffffffu, a, l),
                    wd = __shfl_sync(0xffffffffu, deg, l);
      if (lane == l) deg = 0;
      push_strided(op, wu, wa, wd, lane, 32, idx, to, out);
    }
    if (fine) {
      int32_t T;
      const int32_t off = block_excl_scan(deg, &T, s_sw);
      s_src[tid] = u;
      s_beg[tid] = a;
      s_off[tid] = off;
      for (int32_t k = 0; k < deg; ++k) s_own[off + k] = (Own)tid;
      __syncthreads();
      for (int32_t j0 = tid; j0 < T; j0 += kPushBatch * kBlock) {
        int32_t uu[kPushBatch], ee[kPushBatch], vv[kPushBatch];
#pragma unroll
        for (int b = 0; b < kPushBatch; ++b) {
          const int32_t j = j0 + b * kBlock;
          if (j < T) {
            const int o = s_own[j];
            uu[b] = s_src[o];
            ee[b] = s_beg[o] + (j - s_off[o]);
            vv[b] = __ldg(idx + ee[b]);
          } else {
            uu[b] = -1;
            ee[b] = 0;
            vv[b] = -1;
          }
        }
        push_batch(op, uu, vv, ee, to, out);
      }
      __syncthreads();
    } else {
      push_strided(op, u, a, deg, 0, 1, idx, to, out);
    }
  }
}

}  // namespace gi

namespace gi {

// Sources with >= t_heavy arcs, deferred by k_push: their arcs are cut into
// chunks of kHeavyChunk, numbered across all deferred sources, and chunk c is
// expanded by block c mod gridDim (its source found by binary search over the
// entries' first chunks), so one hub no longer serialises a block and the
// work per block does not grow with the number of deferred sources.
template <class Op>
__global__ void __launch_bounds__(kPushBlock) k_push_heavy(Op op, const int32_t *__restrict__ ptr,
                                                           const int32_t *__restrict__ idx, void *heavy_mem,
                                                           int64_t n, const uint32_t *__restrict__ to, OutSet out) {
  const HeavyList heavy = heavy_at(heavy_mem, n);
  const unsigned long long c64 = *(volatile unsigned long long *)heavy.ctr;
  // nothing deferred: the list is already empty, and no block takes a ticket
  // (the expansion of an empty list otherwise costs a ticket per block)
  if (c64 == 0ull) return;
  const int32_t H = (int32_t)(c64 >> 32), C = (int32_t)(c64 & 0xffffffffull);
  for (int32_t c = blockIdx.x; c < C; c += gridDim.x) {
    int32_t lo = 0, hi = H - 1;  // last entry whose first chunk is <= c
    while (lo < hi) {
      const int32_t mid = (lo + hi + 1) >> 1;
      if (heavy.base[mid] <= c) lo = mid;
      else hi = mid - 1;
    }
    const int32_t u = heavy.src[lo];
    const int32_t a = __ldg(ptr + u), deg = __ldg(ptr + u + 1) - a;
    const int32_t k0 = (c - heavy.base[lo]) * kHeavyChunk;
    const int32_t len = min(kHeavyChunk, deg - k0);
    push_strided(op, u, a + k0, len, (int32_t)threadIdx.x, kPushBlock, idx, to, out);
  }
  // the last block to finish empties the list for the next push (every block
  // has read the counter before it takes its ticket)
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(heavy.ticket, 1) == (int32_t)gridDim.x - 1) {
      *heavy.ctr = 0ull;
      *heavy.ticket = 0;
      __threadfence();
    }
  }
}

// Edge-parallel SparsePush (balance GI_BAL_EDGE_PARALLEL): off[] is the
// exclusive scan of the frontier's out-degrees (off[nf] = m_f), so arc j of
// the frontier belongs to entry i = max{i : off[i] <= j}.  Each block takes
// kEdgeTile consecutive arcs: two threads locate the entry range it spans,
// the block copies that slice of off[] to shared memory (when it fits) and
// every thread finds its arcs' entries there; arcs of one source sit in
// consecutive threads, so the index loads coalesce.
constexpr int kEdgeTile = 1024;

static __global__ void k_front_deg(const int32_t *__restrict__ q, int64_t nf, const int32_t *__restrict__ ptr,
                            int32_t *fd) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = q[i];
    fd[i] = __ldg(ptr + u + 1) - __ldg(ptr + u);
  }
}

// largest i in [lo, hi] with off[i] <= j (off[lo] <= j holds)
__device__ __forceinline__ int32_t entry_of(const int32_t *off, int32_t lo, int32_t hi, int32_t j) {
  while (lo < hi) {
    const int32_t mid = (lo + hi + 1) >> 1;
    if (off[mid] <= j) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <class Op>
__global__ void __launch_bounds__(256) k_push_edges(Op op, const int32_t *__restrict__ q,
                                                    const int32_t *__restrict__ off, int32_t nf,
                                                    const int32_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                                                    const uint32_t *__restrict__ to, OutSet out) {
  constexpr int kPer = kEdgeTile / 256;
  __shared__ int32_t s_off[kEdgeTile + 1];
  __shared__ int32_t s_lo, s_hi;
  const int32_t total = off[nf];
  for (int64_t base = (int64_t)blockIdx.x * kEdgeTile; base < total; base += (int64_t)gridDim.x * kEdgeTile) {
    const int32_t j0 = (int32_t)base;
    const int32_t j1 = (int32_t)(base + kEdgeTile < (int64_t)total ? base + kEdgeTile : (int64_t)total) - 1;
    if (threadIdx.x == 0) s_lo = entry_of(off, 0, nf - 1, j0);
    if (threadIdx.x == 1) s_hi = entry_of(off, 0, nf - 1, j1);
    __syncthreads();
    const int32_t lo = s_lo, hi = s_hi, cnt = hi - lo + 1;
    const bool window = cnt <= kEdgeTile;  // zero-degree entries can widen the range
    if (window)
      for (int k = threadIdx.x; k < cnt; k += 256) s_off[k] = off[lo + k];
    __syncthreads();
    int32_t u[kPer], e[kPer], v[kPer];
#pragma unroll
    for (int p = 0; p < kPer; ++p) {
      const int32_t j = j0 + (int32_t)threadIdx.x + p * 256;
      u[p] = -1;
      e[p] = 0;
      v[p] = -1;
      if (j <= j1) {
        const int32_t i = window ? lo + entry_of(s_off, 0, cnt - 1, j) : entry_of(off, lo, hi, j);
        const int32_t oi = window ? s_off[i - lo] : off[i];
        u[p] = q[i];
        e[p] = __ldg(ptr + u[p]) + (j - oi);
        v[p] = __ldg(idx + e[p]);
      }
    }
    push_batch(op, u, v, e, to, out);
    __syncthreads();
  }
}

// SparsePull (Table 3's pull into a sparse output set): every destination v
// of a queue gathers over its in-arcs, combine over sources in F of
// op.edge_val, then op.finish(v, .) where op.dst_ok(v).  Rows of >= t_cta
// arcs are reduced by the whole block, >= t_warp by a warp, the rest by their
// own thread; each row's order of combination is fixed, so results do not
// depend on scheduling.  The queue's length is *qcount (device) or, when
// qcount is NULL, qn.
template <class Op>
__device__ __forceinline__ typename Op::V sparse_row(const Op &op, const int32_t *__restrict__ idx, const FSet &F,
                                                     int32_t a, int32_t deg, int32_t k0, int32_t step) {
  using V = typename Op::V;
  V x = Op::identity();
  for (int32_t k = k0; k < deg; k += 8 * step) {
    int32_t u[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) u[j] = k + j * step < deg ? __ldg(idx + a + k + j * step) : -1;
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (u[j] >= 0 && in_set(F, u[j])) x = combine_term<Op>(x, op.edge_val(u[j], a + k + j * step));
  }
  return x;
}

template <class Op>
__global__ void __launch_bounds__(256) k_pull_sparse(Op op, const int32_t *__restrict__ q,
                                                     const int32_t *__restrict__ qcount, int64_t qn,
                                                     const int32_t *__restrict__ ptr,
                                                     const int32_t *__restrict__ idx, FSet F, OutSet out,
                                                     int32_t t_warp, int32_t t_cta) {
  using V = typename Op::V;
  constexpr int kB = 256;
  __shared__ int32_t s_owner, s_a, s_deg;
  __shared__ V s_red[kB / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t cnt = qcount ? (int64_t)(*qcount) : qn;
  for (int64_t base = (int64_t)blockIdx.x * kB; base < cnt; base += (int64_t)gridDim.x * kB) {
    const int64_t i = base + tid;
    int32_t v = -1, a = 0, deg = 0;
    bool pending = false;
    V acc = Op::identity();
    if (i < cnt) {
      v = q[i];
      a = __ldg(ptr + v);
      deg = __ldg(ptr + v + 1) - a;
      pending = true;
    }
    while (true) {  // block-cooperative rows
      if (tid == 0) s_owner = -1;
      __syncthreads();
      if (deg >= t_cta) s_owner = tid;
      __syncthreads();
      const int owner = s_owner;
      if (owner < 0) break;
      if (tid == owner) {
        s_a = a;
        s_deg = deg;
      }
      __syncthreads();
      V x = warp_reduce<V, Op>(sparse_row(op, idx, F, s_a, s_deg, tid, kB));
      if (lane == 0) s_red[warp] = x;
      __syncthreads();
      if (tid == owner) {
        V y = Op::identity();
        for (int k = 0; k < kB / 32; ++k) y = Op::combine(y, s_red[k]);
        acc = y;
        deg = 0;
      }
      __syncthreads();
    }
    while (true) {  // warp-cooperative rows
      const unsigned bal = __ballot_sync(0xffffffffu, deg >= t_warp);
      if (!bal) break;
      const int l = __ffs(bal) - 1;
      const int32_t la = __shfl_sync(0xffffffffu, a, l), ld = __shfl_sync(0xffffffffu, deg, l);
      const V x = warp_reduce<V, Op>(sparse_row(op, idx, F, la, ld, lane, 32));
      if (lane == l) {
        acc = x;
        deg = 0;
      }
    }
    if (deg > 0) acc = sparse_row(op, idx, F, a, deg, 0, 1);
    if (pending && op.dst_ok(v) && op.finish(v, acc) && out.enabled()) out_mark(out, v);
  }
}

// BFS as a pull edge function (SparsePull): an unvisited destination with an
// in-neighbour in F takes depth = level and parent = the smallest such
// in-neighbour (the canonical parent).
struct OpBFSPull {
  using V = int32_t;
  int32_t *depth;
  int32_t *parent;
  int32_t level;
  __device__ static V identity() { return INT32_MAX; }
  __device__ static V combine(V a, V b) { return a < b ? a : b; }
  __device__ V edge_val(int32_t u, int32_t) const { return u; }
  __device__ bool dst_ok(int32_t v) const { return depth[v] == -1; }
  __device__ bool finish(int32_t v, V m) const {
    if (m == INT32_MAX) return false;
    depth[v] = level;
    if (parent) parent[v] = m;
    return true;
  }
};

}  // namespace gi

// =================================================================== host side ==
namespace gi {

template <class Op>
size_t pull_smem_bytes(int32_t tile_edges) {
  return pull_stage_bytes<typename Op::V>(tile_edges);
}

// Ops whose arc value is built from a per-source 4-byte value (hot_source()[u]) can use the hot-source pull.
template <class Op, class = void>
struct HotGatherable : std::false_type {};
template <class Op>
struct HotGatherable<Op, std::void_t<decltype(std::declval<const Op &>().hot_source())>> : std::true_type {};

template <class Op, int kTE>
int launch_pull_hot_te(gi_graph *g, const Op &op, const TileSet &ts, const uint32_t *to, const OutSet &out,
                       cudaStream_t s) {
  using V = typename Op::V;
  constexpr int kGroups = 4, kBlocksPerSm = 2;
  auto kern = k_pull_hot<Op, kTE, kGroups>;
  const int32_t k4 = (g->hot.k + 3) & ~3;
  const size_t stage = (pull_stage_bytes<V>(kTE) + 15) & ~(size_t)15;
  // shared memory for two blocks per SM: the per-SM capacity less the 1 KB
  // the runtime reserves per block and the kernel's static arrays
  int per_sm = 0, optin = 0;
  cudaFuncAttributes fa;
  GI_CUDA(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, g->device));
  GI_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, g->device));
  GI_CUDA(cudaFuncGetAttributes(&fa, kern));
  const int64_t budget = std::min<int64_t>(optin, per_sm / kBlocksPerSm - 1024) - (int64_t)fa.sharedSizeBytes;
  int64_t room = (budget - (int64_t)stage * kGroups) / (int64_t)sizeof(float);
  room = room < 0 ? 0 : (room & ~(int64_t)3);
  const int32_t k1 = (int32_t)std::min<int64_t>({(int64_t)k4, room, (int64_t)kHotSmemSlots});
  const size_t smem = sizeof(float) * (size_t)k1 + stage * kGroups;
  GI_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t full = (int64_t)g->num_sms * kBlocksPerSm;
  const int grid = (int)std::min<int64_t>(full, div_up(ts.num_tiles, kGroups));
  kern<<<grid, 256 * kGroups, smem, s>>>(op, g->in.ptr, g->hot.idx, ts.tiles, ts.num_tiles, g->hot.vals, k1, to, out,
                                         reinterpret_cast<V *>(ts.partial));
  return GI_OK;
}

template <class Op, int kTE, int kMode = kGatherPlain>
int launch_pull_tiled_te(const Op &op, const int32_t *ptr, const int32_t *idx, const TileSet &ts, FSet F,
                         const uint32_t *to, const OutSet &out, const float *hot, cudaStream_t s) {
  constexpr int kB = 256;
  const size_t smem = pull_smem_bytes<Op>(kTE);
  if (smem > 48 * 1024) {
    GI_CUDA(cudaFuncSetAttribute(k_pull_tiled<Op, kB, kTE, kMode>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
  }
  k_pull_tiled<Op, kB, kTE, kMode><<<ts.num_tiles, kB, smem, s>>>(op, ptr, idx, ts.tiles, ts.num_tiles, F, to, out,
                                                                  reinterpret_cast<typename Op::V *>(ts.partial), hot,
                                                                  ts.rows);
  return GI_OK;
}

// Hot-source pull (hot_mode 1: shared-memory cache, block tiles of 512..2048
// arcs; 2: L1-resident hot array, block tiles of 512..8192 arcs).  Returns
// false (nothing launched) where it does not apply.
template <class Op>
int launch_pull_hot(gi_graph *g, const Op &op, const TileSet &ts, const uint32_t *to, const OutSet &out,
                    cudaStream_t s, int kclass, int hot_mode, bool *done) {
  *done = false;
  const int te = ts.tile_edges;
  // the shared-memory form takes block tiles of <= 2048 arcs
  if (ts.num_tiles == 0 || te < 512 || (hot_mode == 1 && te > 2048)) return GI_OK;
  GI_TRY(hot_get(g, s));
  if (g->hot.k == 0) return GI_OK;
  const int tok = timing_begin(kclass, s);
  using S = hot_src_t<Op>;
  k_hot_gather<S><<<div_up(g->hot.k, 256), 256, 0, s>>>(op.hot_source(), g->hot.src, g->hot.k,
                                                        reinterpret_cast<S *>(g->hot.vals));
  GI_LAUNCH_CHECK();
  const float *hv = g->hot.vals;
  const int32_t *hp = g->in.ptr, *hi = g->hot.idx;
  if (hot_mode == 1) {
    switch (te) {
      case 512: GI_TRY((launch_pull_hot_te<Op, 512>(g, op, ts, to, out, s))); break;
      case 1024: GI_TRY((launch_pull_hot_te<Op, 1024>(g, op, ts, to, out, s))); break;
      default: GI_TRY((launch_pull_hot_te<Op, 2048>(g, op, ts, to, out, s))); break;
    }
  } else {
    switch (te) {
      case 512: GI_TRY((launch_pull_tiled_te<Op, 512, kGatherHotL1>(op, hp, hi, ts, FSet(), to, out, hv, s))); break;
      case 1024: GI_TRY((launch_pull_tiled_te<Op, 1024, kGatherHotL1>(op, hp, hi, ts, FSet(), to, out, hv, s))); break;
      case 2048: GI_TRY((launch_pull_tiled_te<Op, 2048, kGatherHotL1>(op, hp, hi, ts, FSet(), to, out, hv, s))); break;
      case 4096: GI_TRY((launch_pull_tiled_te<Op, 4096, kGatherHotL1>(op, hp, hi, ts, FSet(), to, out, hv, s))); break;
      default: GI_TRY((launch_pull_tiled_te<Op, 8192, kGatherHotL1>(op, hp, hi, ts, FSet(), to, out, hv, s))); break;
    }
  }
  timing_end(tok, s);
  GI_LAUNCH_CHECK();
  if (ts.num_splits > 0) {
    k_pull_fixup<Op><<<div_up(ts.num_splits, 128), 128, 0, s>>>(
        op, ts.splits, ts.num_splits, reinterpret_cast<const typename Op::V *>(ts.partial), to, out);
    GI_LAUNCH_CHECK();
  }
  *done = true;
  return GI_OK;
}

// Tiled pull over the in-edges `c` with tiles `ts` (the whole graph or one segment).
// hot_mode (gi_schedule.hot_cache) applies to whole-graph pulls from all sources
// of Ops whose arc values come from per-source 4-byte values (both forms
// take any such value: fp32 contributions, int32 labels or distances).
template <class Op>
int launch_pull_tiled(gi_graph *g, const Op &op, const Csr &c, const TileSet &ts, FSet F,
                      const uint32_t *to, const OutSet &out, cudaStream_t s, int kclass = kClassOtherPull,
                      bool vertex_parallel = false, int hot_mode = 0) {
  if constexpr (HotGatherable<Op>::value) {
    if (hot_mode != 0 && !vertex_parallel && F.bm == nullptr && F.bytes == nullptr && c.idx == g->in.idx &&
        ts.tiles == g->in_tiles.tiles) {
      bool done = false;
      GI_TRY(launch_pull_hot(g, op, ts, to, out, s, kclass, hot_mode, &done));
      if (done) return GI_OK;
    }
  }
  if (vertex_parallel) {
    const int tok = timing_begin(kclass, s);
    k_pull_vertex<Op><<<grid_for(g, g->n, 256), 256, 0, s>>>(op, c.ptr, c.idx, g->n, F, to, out);
    timing_end(tok, s);
    GI_LAUNCH_CHECK();
    return GI_OK;
  }
  if (ts.num_tiles == 0) return GI_OK;
  if (timing_on() && ts.tile_edges != kWarpTileEdges) {
    // instrumentation, outside the timed launch: the arcs the block tiles
    // are about to gather, by the pull's own tile and filter rules
    k_pull_count<Op><<<grid_for(g, ts.num_tiles, 256), 256, 0, s>>>(
        op, ts.tiles, ts.num_tiles, ts.rows, to, reinterpret_cast<unsigned long long *>(g->ctrl + kPullArcs));
    GI_LAUNCH_CHECK();
  }
  const int tok = timing_begin(kclass, s);
  if (ts.rows != nullptr && ts.tile_edges == kWarpTileEdges) {
    set_error("warp tiles over a row-compacted CSR are not supported");
    return GI_ERR_UNSUPPORTED;
  }
  switch (ts.tile_edges) {
    case kWarpTileEdges: {
      constexpr int kCap = kWarpTileEdges + kWarpTileEdges / kLongRowDiv;
      const size_t smem = sizeof(typename Op::V) * kCap * kWarpsPerBlock;
      if (smem > 48 * 1024)
        GI_CUDA(cudaFuncSetAttribute(k_pull_warp<Op>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      const int grid = (ts.num_tiles + kWarpsPerBlock - 1) / kWarpsPerBlock;
      k_pull_warp<Op><<<grid, 32 * kWarpsPerBlock, smem, s>>>(op, c.ptr, c.idx, ts.tiles, ts.num_tiles, F, to, out,
                                                              reinterpret_cast<typename Op::V *>(ts.partial));
      break;
    }
    case 512: GI_TRY((launch_pull_tiled_te<Op, 512>(op, c.ptr, c.idx, ts, F, to, out, nullptr, s))); break;
    case 1024: GI_TRY((launch_pull_tiled_te<Op, 1024>(op, c.ptr, c.idx, ts, F, to, out, nullptr, s))); break;
    case 2048: GI_TRY((launch_pull_tiled_te<Op, 2048>(op, c.ptr, c.idx, ts, F, to, out, nullptr, s))); break;
    case 4096: GI_TRY((launch_pull_tiled_te<Op, 4096>(op, c.ptr, c.idx, ts, F, to, out, nullptr, s))); break;
    case 8192: GI_TRY((launch_pull_tiled_te<Op, 8192>(op, c.ptr, c.idx, ts, F, to, out, nullptr, s))); break;
    default:
      set_error("unsupported tile size %d", ts.tile_edges);
      return GI_ERR_UNSUPPORTED;
  }
  timing_end(tok, s);
  GI_LAUNCH_CHECK();
  if (ts.num_splits > 0) {
    k_pull_fixup<Op><<<div_up(ts.num_splits, 128), 128, 0, s>>>(
        op, ts.splits, ts.num_splits, reinterpret_cast<const typename Op::V *>(ts.partial), to, out, ts.rows);
    GI_LAUNCH_CHECK();
  }
  return GI_OK;
}

// Edge-parallel SparsePush over from's queue (nf members, or read back when -1).
template <class Op>
int launch_push_edges(gi_graph *g, const Op &op, const gi_vset *from, int64_t nf, const uint32_t *to,
                      const OutSet &out, cudaStream_t s, const Csr &c) {
  if (nf < 0) {
    int32_t c = 0;
    GI_CUDA(cudaMemcpyAsync(&c, from->count, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    GI_CUDA(cudaStreamSynchronize(s));
    nf = c;
  }
  if (nf == 0) return GI_OK;
  int32_t *fd = nullptr, *off = nullptr;
  GI_TRY(ws_scratch(g, &fd, &off, s));
  k_front_deg<<<grid_for(g, nf, 256), 256, 0, s>>>(from->queue, nf, c.ptr, fd);
  GI_LAUNCH_CHECK();
  GI_TRY(scan_exclusive(g, fd, off, nf, s));
  const int tok = timing_begin(kClassPush, s);
  k_push_edges<Op><<<g->num_sms * 8, 256, 0, s>>>(op, from->queue, off, (int32_t)nf, c.ptr, c.idx, to, out);
  timing_end(tok, s);
  GI_LAUNCH_CHECK();
  return GI_OK;
}

// SparsePull over the queue q (length *qcount on the device, or qn when
// qcount is NULL), gathering along c's rows.
template <class Op>
int launch_pull_sparse(gi_graph *g, const Op &op, const Csr &c, const int32_t *q, const int32_t *qcount, int64_t qn,
                       FSet F, const OutSet &out, const gi_schedule &sc, cudaStream_t s, int kclass = kClassOtherPull) {
  const int32_t tw = sc.balance == GI_BAL_VERTEX ? INT32_MAX : (sc.t_warp > 0 ? sc.t_warp : 32);
  const int32_t tc = sc.balance == GI_BAL_VERTEX ? INT32_MAX : (sc.t_cta > 0 ? max(sc.t_cta, tw) : 1024);
  int grid = g->num_sms * 8;
  if (!qcount) {
    if (qn == 0) return GI_OK;
    grid = (int)std::min<int64_t>((qn + 255) / 256, (int64_t)grid);
  }
  const int tok = timing_begin(kclass, s);
  k_pull_sparse<Op><<<grid, 256, 0, s>>>(op, q, qcount, qn, c.ptr, c.idx, F, out, tw, tc);
  timing_end(tok, s);
  GI_LAUNCH_CHECK();
  return GI_OK;
}

// Push along the out-edges (csr: another arc set of the same vertices, e.g.
// the light or heavy arcs of delta-stepping; NULL = the graph's CSR).  mode:
// kSrcQueue (from's queue), kSrcBitmap (scan from's bitmap over all
// vertices), kSrcAll.
template <class Op>
int launch_push(gi_graph *g, const Op &op, int mode, const gi_vset *from, const uint32_t *to, const OutSet &out,
                const gi_schedule &sc, cudaStream_t s, const Csr *csr = nullptr) {
  const Csr &c = csr ? *csr : g->out;
  if (mode == kSrcQueue && sc.balance == GI_BAL_EDGE_PARALLEL)
    return launch_push_edges(g, op, from, from == g->hint_vset ? g->hint_nf : -1, to, out, s, c);
  int32_t tw = sc.balance == GI_BAL_VERTEX ? INT32_MAX : (sc.t_warp > 0 ? sc.t_warp : 32);
  int32_t tc = sc.balance == GI_BAL_VERTEX ? INT32_MAX : (sc.t_cta > 0 ? sc.t_cta : 1024);
  if (tw != INT32_MAX && tw > kMaxTWarp) tw = kMaxTWarp;
  if (tc < tw) tc = tw;
  const int32_t th = sc.balance == GI_BAL_VERTEX ? INT32_MAX : (sc.t_heavy > 0 ? max(sc.t_heavy, tc) : INT32_MAX);
  if (th != INT32_MAX) GI_TRY(heavy_get(g, s));
  void *heavy = g->heavy_mem;
  const int block = kPushBlock;
  int grid;
  const int tok = timing_begin(kClassPush, s);
  if (mode == kSrcQueue) {
    // SparsePush takes the schedule's block size (128, 256 or 512 threads);
    // the grid keeps 2048 threads per SM
    const int qb = sc.block == 128 || sc.block == 512 ? sc.block : 256;
    grid = g->num_sms * (2048 / qb);
    if (qb == 512 && tw != INT32_MAX && tw > PushOwners<512>::kMaxTW) tw = PushOwners<512>::kMaxTW;
    if (tc < tw) tc = tw;
    if (qb == 128)
      k_push<Op, kSrcQueue, 128><<<grid, 128, 0, s>>>(op, c.ptr, c.idx, from->queue, from->count, nullptr, g->n, to,
                                                      out, tw, tc, th, heavy);
    else if (qb == 512)
      k_push<Op, kSrcQueue, 512><<<grid, 512, 0, s>>>(op, c.ptr, c.idx, from->queue, from->count, nullptr, g->n, to,
                                                      out, tw, tc, th, heavy);
    else
      k_push<Op, kSrcQueue><<<grid, block, 0, s>>>(op, c.ptr, c.idx, from->queue, from->count, nullptr, g->n, to,
                                                   out, tw, tc, th, heavy);
  } else if (mode == kSrcBitmap) {
    grid = grid_for(g, g->n, block, 2048 / block);
    const FSet fs = (sc.dense_rep == GI_REP_BOOL && from->boolmap && (from->reps & GI_REP_BOOL))
                        ? FSet(static_cast<const uint8_t *>(from->boolmap))
                        : FSet(static_cast<const uint32_t *>(from->bitmap));
    k_push<Op, kSrcBitmap><<<grid, block, 0, s>>>(op, c.ptr, c.idx, nullptr, nullptr, fs, g->n, to, out, tw,
                                                  tc, th, heavy);
  } else {
    grid = grid_for(g, g->n, block, 2048 / block);
    k_push<Op, kSrcAll><<<grid, block, 0, s>>>(op, c.ptr, c.idx, nullptr, nullptr, nullptr, g->n, to, out,
                                               tw, tc, th, heavy);
  }
  GI_LAUNCH_CHECK();
  if (th != INT32_MAX && g->max_deg >= th) {  // otherwise no source can have been deferred
    k_push_heavy<Op><<<g->num_sms * 4, block, 0, s>>>(op, c.ptr, c.idx, heavy, g->n, to, out);
    GI_LAUNCH_CHECK();
  }
  timing_end(tok, s);
  return GI_OK;
}

inline OutSet out_of(gi_vset *v, bool dedup = true) {
  OutSet o;
  if (v) {
    o.bm = v->bitmap;
    o.q = v->queue;
    o.qc = v->count;
    o.dedup = dedup;
  }
  return o;
}

}  // namespace gi
