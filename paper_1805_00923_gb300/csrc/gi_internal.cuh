// Internal declarations shared by the library's translation units.
// Not part of the public ABI (see include/graphit_gb.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>

#include "../../include/graphit_gb.h"

// ------------------------------------------------------------------ errors --
namespace gi {

void set_error(const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what, const char *file, int line);

// launch accounting: every kernel launch is counted; launch_status counts n
// launches and reports a launch error as GI_ERR_CUDA.
void note_launch(int n);
int launch_status(int n);

// CUDA-event timing of selected kernel classes (gi_stats_*): returns a token
// for timing_end, or -1 when timing is off.
enum KernelClass { kClassPrPull = 0, kClassPrdPull = 1, kClassMinPull = 2, kClassPush = 3, kClassBfsPull = 4,
                   kClassOtherPull = 5, kClassBatch = 6, kNumClasses = 7 };
int timing_begin(int kclass, cudaStream_t s);
bool timing_on();  // per-launch event timing (gi_stats_enable) is on
void timing_end(int token, cudaStream_t s);

}  // namespace gi

#define GI_CUDA(call)                                                           \
  do {                                                                          \
    cudaError_t _e = (call);                                                    \
    if (_e != cudaSuccess) return gi::cuda_fail(_e, #call, __FILE__, __LINE__); \
  } while (0)

#define GI_LAUNCH_CHECK()                  \
  do {                                     \
    gi::note_launch(1);                    \
    GI_CUDA(cudaGetLastError());           \
  } while (0)

#define GI_ARG(cond, msg)                                   \
  do {                                                      \
    if (!(cond)) {                                          \
      gi::set_error("invalid argument: %s", msg);           \
      return GI_ERR_INVALID_ARG;                            \
    }                                                       \
  } while (0)

#define GI_TRY(expr)            \
  do {                          \
    int _s = (expr);            \
    if (_s != GI_OK) return _s; \
  } while (0)

namespace gi {

// ------------------------------------------------------------ constants --
constexpr int kLongRowDiv = 2;         // rows with degree > tile_edges/kLongRowDiv get their own tiles
constexpr int kTileRows = 512;         // at most this many rows per short block tile
constexpr int kWarpTileEdges = 256;    // tile_edges value that selects warp-sized tiles
constexpr int kWarpTileRows = 64;      // at most this many rows per short warp tile
inline int tile_rows_for(int tile_edges) { return tile_edges == kWarpTileEdges ? kWarpTileRows : kTileRows; }
constexpr int kCtrlWords = 64;         // int64 words in the per-graph control block

// Control-block slots (int64) written by the frontier-statistics kernel.
enum CtrlSlot {
  kNf = 0,        // |F|
  kMf = 1,        // sum of out-degrees over F
  kNu = 2,        // unvisited vertices (BFS)
  kMu = 3,        // sum of out-degrees over unvisited vertices
  kDecision = 4,  // chosen direction (GI_DIR_SPARSE_PUSH / DENSE_PUSH / DENSE_PULL)
  kWasPull = 5,
  kLevel = 6,
  kNfPrev = 7,
  kTicket = 8,    // last-block ticket of the statistics kernel
  kErr = 9,       // device-side error flag (bounded waits, bounds checks)
  kMfAcc = 10,    // m_f accumulator of the statistics kernel (its last block returns it to 0)
  kFeat = 16,     // 16 float features stored as float bits in 8 int64 words (slots 16..23)
  kDsSlots = 32,  // delta-stepping SSSP: 8 int32 round words in slots 32..35 (fetched with the rest)
  kPullArcs = 40, // arcs the block-tiled pulls gathered while timing was on (kept by ctrl_init)
  kSHeavyMf = 11, // graph-driven delta-stepping: heavy arcs of the bucket's settled list so far
};

// --------------------------------------------------------------- graph --
struct Csr {
  int32_t *ptr = nullptr;  // n+1
  int32_t *idx = nullptr;  // m
  int32_t *wt = nullptr;   // m or null
};

// Pull tile: {r0, r1, e0, e1}.
//   r1 >  r0 : short tile, rows [r0, r1), arcs [ptr[r0], ptr[r1])
//   r1 == r0 : one long row r0, arcs [e0, e1) = the whole row
//   r1 == -1 : piece [e0, e1) of long row r0 split over several tiles; the
//              partial result goes to slot = tile index, combined by a fix-up.
struct TileSet {
  int4 *tiles = nullptr;
  int4 *splits = nullptr;  // {row, first tile, piece count, 0}
  // tiles over a row-compacted CSR (only the rows that have arcs): row r of
  // the tiles is vertex rows[r] (not owned); nullptr: row r is vertex r
  const int32_t *rows = nullptr;
  int32_t num_tiles = 0;
  int32_t num_splits = 0;
  int32_t tile_edges = 0;
  void *partial = nullptr;  // 16 bytes per tile (largest reduction value)
};

struct Segments {
  int32_t num = 1;
  int32_t strategy = 0;       // GI_SEG_FVC or GI_SEG_EVC
  int32_t *bounds = nullptr;  // host array [num+1]: segment s holds sources [bounds[s], bounds[s+1])
  int64_t *arcs = nullptr;    // host array [num]: arcs of each segment
  Csr *seg = nullptr;         // host array of per-segment CSCs (device pointers)
  TileSet *tiles = nullptr;   // host array: tiles of each segment
};

// Hot-source cache for dense pulls over the whole graph: the sources of
// highest out-degree (out_deg >= min_deg, at most kHotMax of them) get slots
// in descending degree; `idx` is the in-edge column array with each hot
// source u replaced by ~slot(u) (negative), so a pull kernel that holds the
// hot sources' values on chip reads them there without a lookup.
constexpr int kHotMax = 24576;  // 96 KB of 4-byte values (fits beside the pull's staging in L1)
// cap on the slots the shared-memory form keeps in shared memory (the rest
// of the hot set is read through L1).  A larger shared-memory share shrinks
// L1, which the cold gathers need for their misses in flight: on R-MAT 22
// (2048-arc tiles) caps of 8,192 / 12,288 / 14,544 slots ran 0.479 / 0.649 /
// 0.635 ms per PageRank pull.
constexpr int kHotSmemSlots = 8192;
struct HotSet {
  bool built = false;
  int32_t k = 0;              // hot sources (0: the cache does not apply)
  int32_t min_deg = 0;
  int32_t *src = nullptr;     // k: slot -> vertex id
  int32_t *idx = nullptr;     // m: remapped in-edge sources
  float *vals = nullptr;      // round_up(k, 4): source values staged for one launch
};

struct Workspace;  // per-graph scratch (frontiers, buffers); defined in gi_core.cu

// The unvisited destinations of the early-exit BFS pull as a compacted list
// (the destination filter of Sec. 2 kept sparse).  `live` lists, ascending,
// the vertices with in-arcs (built once per graph: the others can never be
// reached); each pull level walks its input list and appends the vertices it
// leaves unvisited to the other list, so later pull levels touch only rows
// that can still be reached.  st[0] = the input of the next pull (-1: live;
// 0 / 1: list0 / list1), st[1] / st[2] = the counts of list0 / list1, st[3] =
// the walking launch's ticket (its last block flips st[0] and empties the
// next output).  A query starts at {-1, 0, 0, 0} (k_bfs_init).
struct BfsUnv {
  const int32_t *live = nullptr;
  int32_t *list0 = nullptr, *list1 = nullptr;
  int32_t *st = nullptr;  // nullptr: walk every vertex
  int32_t nlive = 0;
};
}  // namespace gi

struct gi_graph {
  int64_t n = 0, m = 0;
  int32_t max_deg = 0;
  double wt_mean = 0.0;          // mean arc weight (0 without weights)
  bool symmetric = false;
  bool has_csc = false;
  gi::Csr out;            // CSR (out-edges)
  gi::Csr in;             // CSC (in-edges); aliases `out` when symmetric
  int32_t *out_deg = nullptr;
  float *inv_out_deg = nullptr;  // 1/outdeg (0 for degree 0)
  gi::TileSet in_tiles;          // active tile set over the in-edges (a view into tile_cache)
  gi::TileSet tile_cache[6];     // owned tile sets for tile_edges 256, 512, ..., 8192 (built on first use)
  gi::Segments segs;
  gi::HotSet hot;                // built on first use of the hot-source pull
  // member count and out-degree sum of a frontier known on the host (set by
  // the drivers after their per-round statistics, cleared after the round);
  // -1 = unknown
  const gi_vset *hint_vset = nullptr;
  int64_t hint_nf = -1, hint_mf = -1;
  void *graph_loop = nullptr;    // cached CUDA graph of the graph-driven BFS (gi_schedule.persistent = 2)
  void *dstep = nullptr;         // cached light/heavy arc split of delta-stepping SSSP (gi_schedule.delta)
  int64_t *ctrl = nullptr;       // device control block (kCtrlWords)
  void *heavy_mem = nullptr;     // HeavyList storage (counter, ticket, 2n entries), allocated on first use
  void *bfs_defer = nullptr;     // BfsDefer storage of the early-exit BFS pull, allocated on first use
  void *bfs_unv = nullptr;       // BfsUnv storage (live list, two lists, state), built on first use
  int32_t bfs_unv_n = 0;         // its live-list length
  // BfsUnv state of the running gi_bfs query (st == nullptr outside one):
  // its DensePull levels walk the compacted unvisited list
  gi::BfsUnv bfs_unv_query;
  int64_t *ctrl_host = nullptr;  // pinned mirror
  gi::Workspace *ws = nullptr;
  int device = 0;
  int num_sms = 0;
};

struct gi_vset {
  gi_graph *g = nullptr;
  int64_t n = 0;
  uint32_t reps = 0;          // valid representations (GI_REP_*)
  int32_t *queue = nullptr;   // n entries
  int32_t *count = nullptr;   // device counter (int32) for the queue
  uint8_t *boolmap = nullptr; // n bytes (allocated on first use)
  uint32_t *bitmap = nullptr; // (n+31)/32 words
  int64_t words = 0;
};

namespace gi {

// ---------------------------------------------------------- allocation --
int dev_alloc(void **p, size_t bytes, cudaStream_t s);
void dev_free(void *p, cudaStream_t s);
template <class T>
inline int dev_alloc_n(T **p, int64_t n, cudaStream_t s) {
  return dev_alloc(reinterpret_cast<void **>(p), sizeof(T) * (size_t)(n > 0 ? n : 1), s);
}

// --------------------------------------------------------------- utils --
inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }
int grid_for(const gi_graph *g, int64_t work, int block, int per_sm = 8);
// Sources deferred by k_push to the all-block expansion k_push_heavy.  Each
// deferred source takes its entry and its range of chunks with one 64-bit
// atomicAdd on ctr ((entries << 32) | chunks), so base[] grows with the entry
// index and a chunk's source is found by binary search.  k_push_heavy's last
// block returns ctr and ticket to zero.
// Storage (one allocation): 8-byte ctr, 4-byte ticket, 4 bytes padding, then
// src[n] (deferred sources) and base[n] (first global chunk of src[j]).
struct HeavyList {
  unsigned long long *ctr;
  int32_t *ticket;
  int32_t *src;
  int32_t *base;
};
__host__ __device__ inline HeavyList heavy_at(void *mem, int64_t n) {
  unsigned char *b = static_cast<unsigned char *>(mem);
  HeavyList h;
  h.ctr = reinterpret_cast<unsigned long long *>(b);
  h.ticket = reinterpret_cast<int32_t *>(b + 8);
  h.src = reinterpret_cast<int32_t *>(b + 16);
  h.base = h.src + (n > 0 ? n : 1);
  return h;
}
int heavy_get(gi_graph *g, cudaStream_t s);  // allocates g->heavy_mem on first use

// Rows of the early-exit BFS pull that a warp scanned for kBfsScanCap arcs
// without meeting a frontier source, with more than kBfsDeferChunk arcs
// left, are queued here and finished by every block in chunks of
// kBfsDeferChunk arcs (k_pull_bfs_deferred); best[j] receives the position
// of the first frontier source in the rest of row j.  Each queued row has
// more than kBfsScanCap + kBfsDeferChunk arcs, so m / that + 1 entries hold
// them all.
constexpr int kBfsScanCap = 1024, kBfsDeferChunk = 2048;
struct BfsDefer {
  unsigned long long *ctr;  // (entries << 32) | chunks
  int32_t *ticket;
  int32_t *row, *from, *base, *best;
};
__host__ __device__ inline int32_t bfs_defer_cap(int64_t m) {
  return (int32_t)(m / (kBfsScanCap + kBfsDeferChunk) + 1);
}
__host__ __device__ inline BfsDefer bfs_defer_at(void *mem, int32_t cap) {
  unsigned char *b = static_cast<unsigned char *>(mem);
  BfsDefer d;
  d.ctr = reinterpret_cast<unsigned long long *>(b);
  d.ticket = reinterpret_cast<int32_t *>(b + 8);
  d.row = reinterpret_cast<int32_t *>(b + 16);
  d.from = d.row + cap;
  d.base = d.from + cap;
  d.best = d.base + cap;
  return d;
}
int bfs_defer_get(gi_graph *g, cudaStream_t s);  // allocates g->bfs_defer on first use

int bfs_unv_get(gi_graph *g, cudaStream_t s, BfsUnv *out);  // builds the lists on first use
void bfs_unv_free(gi_graph *g, cudaStream_t s);

// exclusive scan of n int32 counts into out[n+1] (out[n] = total); scratch owned by g's workspace
int scan_exclusive(gi_graph *g, const int32_t *in, int32_t *out, int64_t n, cudaStream_t s);
// the workspace's two (n+2)-entry int32 scratch arrays (transient: valid until the next call that uses them)
int ws_scratch(gi_graph *g, int32_t **a, int32_t **b, cudaStream_t s);

// tiles
// nrows < 0: the graph's n rows
int build_tiles(gi_graph *g, const Csr &c, int32_t tile_edges, TileSet *ts, cudaStream_t s, int64_t nrows = -1);
int use_tiles(gi_graph *g, int32_t tile_edges, cudaStream_t s);  // select (building once) the in-edge tiles
void free_tile_cache(gi_graph *g, cudaStream_t s);
void graph_loop_free(gi_graph *g);  // the cached graph-driven BFS (gi_algos.cu)
void dstep_free(gi_graph *g, cudaStream_t s);  // the cached light/heavy split of delta-stepping (gi_algos.cu)
void free_tiles(TileSet *ts, cudaStream_t s);
int hot_get(gi_graph *g, cudaStream_t s);  // build (once) g->hot from the in-edges
void hot_free(gi_graph *g, cudaStream_t s);

// vertexset internals
int vset_alloc(gi_graph *g, gi_vset *v, cudaStream_t s);
int vset_clear(gi_vset *v, cudaStream_t s);       // empty set, all reps valid (bitmap + queue)
int vset_ensure_bitmap(gi_vset *v, cudaStream_t s);
int vset_ensure_queue(gi_vset *v, cudaStream_t s);
int vset_ensure_bool(gi_vset *v, cudaStream_t s);

// frontier statistics + direction decision (fused); reads F's queue.
// mode: 0 = forced direction `forced`, 1 = rule (hybrid), 2 = learned.
// Device-side level control of the graph-driven drivers (int32 words): the
// statistics kernel reads the level from kGmNext, writes what each traversal
// kernel of the level needs, and sets the WHILE condition of the graph.
enum GmSlot {
  kGmPush = 0,   // queue length the push kernel sees (|F| if this level pushes, else 0)
  kGmPull = 1,   // 1 if this level pulls
  kGmLevel = 2,  // index of the level being expanded (its new vertices get depth kGmLevel + 1)
  kGmNext = 3,   // index of the next level
  kGmCap = 4,    // level cap: reaching it stops the loop with kGmErr set
  kGmErr = 5,
  kGmWords = 8
};

struct DecideParams {
  int32_t mode;
  int32_t forced;      // GI_DIR_* when mode == 0
  int32_t hybrid_kind; // GI_DIR_HYBRID_PULL or GI_DIR_HYBRID_DPUSH
  int32_t rule;
  float alpha, beta;
  int32_t track_unvisited;  // subtract |F|, m_f from n_u, m_u after deciding (BFS)
  int32_t level;
  int32_t *gm = nullptr;                     // graph-driven mode: GmSlot words (level read from there)
  unsigned long long cond_handle = 0;        // graph-driven mode: cudaGraphConditionalHandle of the loop
  // graph-driven mode: the set the level fills, emptied here (its bits are
  // exactly its queue's members: the frontier of two levels before)
  uint32_t *clear_bm = nullptr;
  const int32_t *clear_q = nullptr;
  int32_t *clear_qc = nullptr;
};
// deg: per-vertex arc counts summed into m_f (NULL = out-degrees)
int frontier_decide(gi_graph *g, gi_vset *F, const DecideParams &p, cudaStream_t s, const int32_t *deg = nullptr);

// Graph-driven delta-stepping (gi_sssp with gi_schedule.persistent = 2): the
// int32 words the per-round kernels share, and the round's mode, which is
// also the value of the switch node that runs the round's relaxation.
enum DsgWord {
  kDgHi = 0,      // end of the current bucket
  kDgMode = 1,    // DsgMode of the current round
  kDgRc = 2,      // |R| (this round's light sources)
  kDgSc = 3,      // |S| (the bucket's settled list)
  kDgPile0 = 4,   // counts of the two far-pile buffers
  kDgPile1 = 5,
  kDgPmin = 6,    // smallest distance recorded in the far pile
  kDgCur = 7,     // far-pile buffer in use
  kDgPushL = 8,   // queue length the light push sees (|R| when the round pushes light arcs, else 0)
  kDgPushH = 9,   // the same for the heavy push over S
  kDgRound = 10,  // relaxation rounds run
  kDgCap = 11,    // round cap: reaching it stops the loop with kDgErr set
  kDgErr = 12,
  kDgEpoch = 14,  // bucket number: S membership is s_mark[v] == epoch (no clearing between buckets)
  kDgWords = 16
};
enum DsgMode { kDgLightPush = 0, kDgLightPull = 1, kDgHeavyPush = 2, kDgHeavyPull = 3, kDgAdvance = 4, kDgDone = 5 };
// One graph-driven delta-stepping round's set-up, one launch on s: splits the
// vertices whose distance changed (P) into this round's light sources R
// (snap), the bucket's settled list S (snap_h keeps their latest distance)
// and the far pile, summing R's light and S's heavy arc counts as it goes,
// and empties P's set (bitmap words through its queue, then its count) for
// its next use as an output; its last block then picks the round: the light
// round over R if R is non-empty, else the bucket's heavy round over S, else
// the next bucket (advance) or the end, with its direction (rule or the MLP),
// resets the counters the round has consumed and sets the switch and loop
// conditions.
struct DsgBuffers {
  const int32_t *P;
  int32_t *Pc;
  uint32_t *Pbm;  // P's bitmap
  const int32_t *x;
  int32_t *dw, *Rq, *snap, *snap_h, *Sq, *pile0, *pile1;
  int32_t *s_mark;   // bucket number in which v last joined S
  uint8_t *pile_in;  // 1 while v waits in the far pile
  const int32_t *deg_l, *deg_h;
};
int dsg_step_launch(gi_graph *g, const DsgBuffers &b, const DecideParams &p, int32_t delta, bool pull_ok,
                    unsigned long long switch_handle, unsigned long long while_handle, cudaStream_t s);
int ctrl_init(gi_graph *g, int64_t nu, int64_t mu, cudaStream_t s);
int ctrl_fetch(gi_graph *g, cudaStream_t s);  // copies ctrl to pinned host + syncs

// The traversal a schedule's direction forces (SparsePull needs a `to` set;
// the drivers have none and run it as DensePull), or -1 when it is chosen
// per round (hybrids, learned).
inline int32_t forced_direction(int32_t d) {
  return d <= GI_DIR_DENSE_PULL ? d : (d == GI_DIR_SPARSE_PULL ? GI_DIR_DENSE_PULL : -1);
}

// selector weights (device memory) and state; the batched engine keeps its
// own copy of the weights, uploaded by gi_selector_load
bool selector_loaded();
int batch_selector_upload(const float *params, const float *mean, const float *inv_std);

// traversal entry (gi_traverse.cu)
int apply_dispatch(gi_graph *g, gi_vset *from, gi_vset *to, int32_t dir, const gi_schedule &sc, int32_t kernel_id,
                   const void *args, gi_vset *out, uint32_t flags, cudaStream_t s);

// schedule helpers (gi_traverse.cu)
int check_schedule(const gi_schedule *sc);
DecideParams decide_params(const gi_schedule &sc, int32_t level, bool track_unvisited);
int ensure_tiles(gi_graph *g, const gi_schedule &sc, cudaStream_t s);

}  // namespace gi

// ----------------------------------------------------------- device helpers --
namespace gi {

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ bool bit_test(const uint32_t *bm, int32_t v) {
  return (__ldg(bm + (v >> 5)) >> (v & 31)) & 1u;
}

// set bit; returns true if this call changed it from 0 to 1
__device__ __forceinline__ bool bit_test_and_set(uint32_t *bm, int32_t v) {
  uint32_t mask = 1u << (v & 31);
  uint32_t old = atomicOr(bm + (v >> 5), mask);
  return (old & mask) == 0;
}

// one warp appends the ids of its lanes with pred set to q (count *qc); all
// 32 lanes must call it
__device__ __forceinline__ void warp_append(int32_t *q, int32_t *qc, bool pred, int32_t v) {
  const unsigned b = __ballot_sync(0xffffffffu, pred);
  if (!b) return;
  const int lane = threadIdx.x & 31;
  int32_t base = 0;
  if (lane == 0) base = atomicAdd(qc, __popc(b));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (pred) q[base + __popc(b & ((1u << lane) - 1u))] = v;
}

// warp_append to up to three queues at once: the three reservations are
// issued back to back and their results awaited together (one atomic round
// trip per warp iteration instead of three); q2 may be unused (p2 false)
__device__ __forceinline__ void warp_append3(int32_t *q0, int32_t *c0, bool p0, int32_t *q1, int32_t *c1, bool p1,
                                             int32_t *q2, int32_t *c2, bool p2, int32_t v) {
  const unsigned b0 = __ballot_sync(0xffffffffu, p0), b1 = __ballot_sync(0xffffffffu, p1),
                 b2 = __ballot_sync(0xffffffffu, p2);
  if (!(b0 | b1 | b2)) return;
  const int lane = threadIdx.x & 31;
  int32_t x0 = 0, x1 = 0, x2 = 0;
  if (lane == 0) {
    if (b0) x0 = atomicAdd(c0, __popc(b0));
    if (b1) x1 = atomicAdd(c1, __popc(b1));
    if (b2) x2 = atomicAdd(c2, __popc(b2));
  }
  x0 = __shfl_sync(0xffffffffu, x0, 0);
  x1 = __shfl_sync(0xffffffffu, x1, 0);
  x2 = __shfl_sync(0xffffffffu, x2, 0);
  const unsigned lt = (1u << lane) - 1u;
  if (p0) q0[x0 + __popc(b0 & lt)] = v;
  if (p1) q1[x1 + __popc(b1 & lt)] = v;
  if (p2) q2[x2 + __popc(b2 & lt)] = v;
}


}  // namespace gi
