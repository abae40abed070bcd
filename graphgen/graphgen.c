/*
 * Seeded synthetic graph inputs shared by the oracle tests and the GPU path.
 *
 *   - R-MAT edge lists (recursive quadrant choice with probabilities a, b, c, d)
 *   - 2-D grids with 4-neighbour edges plus random local shortcuts
 *   - CSR assembly: drop self-loops, optionally symmetrize, sort each row, dedup
 *   - symmetric pair-hash edge weights and seeded source sampling
 *
 * Random numbers come from splitmix64 (Vigna's published mixer) applied to a
 * counter, so every value depends only on (seed, index) and the output is the
 * same for any thread count and on any host.  Nothing here computes any part
 * of a traversal: this module only produces inputs.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static inline uint64_t gg_mix(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

/* uniform double in [0,1) from the top 53 bits */
static inline double gg_unit(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

/* uniform integer in [0, n) by multiply-shift (n < 2^32) */
static inline uint64_t gg_below(uint64_t r, uint64_t n) { return ((r >> 32) * n) >> 32; }

uint64_t gg_splitmix64(uint64_t x) { return gg_mix(x); }

/*
 * R-MAT: edge i descends `scale` levels; at each level one draw picks the
 * quadrant (a: top-left, b: top-right, c: bottom-left, d: rest).  Bits are
 * assigned most-significant first.  No noise and no vertex relabelling, so the
 * highest-degree vertex is vertex 0.
 */
void gg_rmat_edges(int32_t scale, int64_t n_edges, double a, double b, double c, uint64_t seed,
                   int32_t *src, int32_t *dst) {
  const uint64_t base = gg_mix(seed ^ 0x5241544D45444745ull);
  const double ab = a + b, abc = a + b + c;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n_edges; ++i) {
    uint32_t s = 0, t = 0;
    for (int32_t lvl = 0; lvl < scale; ++lvl) {
      double u = gg_unit(gg_mix(base + (uint64_t)i * 64u + (uint64_t)lvl));
      uint32_t bit = 1u << (scale - 1 - lvl);
      if (u < a) {
      } else if (u < ab) {
        t |= bit;
      } else if (u < abc) {
        s |= bit;
      } else {
        s |= bit;
        t |= bit;
      }
    }
    src[i] = (int32_t)s;
    dst[i] = (int32_t)t;
  }
}

/* number of undirected 4-neighbour edges of a side x side grid */
int64_t gg_grid_base_edges(int32_t side) { return 2ll * side * (side - 1); }

/*
 * side x side grid, vertex id = y*side + x.  Writes the 4-neighbour edges
 * (each undirected edge once) followed by n_short shortcut edges: a uniform
 * endpoint and a uniform offset (dx, dy) with 2 <= |dx|+|dy| <= max_l1, redrawn
 * (up to 64 times) while the far end falls outside the grid.  Returns the
 * number of edges written (shortcuts that never fit are dropped).
 */
int64_t gg_grid_edges(int32_t side, int64_t n_short, int32_t max_l1, uint64_t seed, int32_t *src,
                      int32_t *dst) {
  int64_t k = 0;
  for (int32_t y = 0; y < side; ++y)
    for (int32_t x = 0; x < side; ++x) {
      int32_t v = y * side + x;
      if (x + 1 < side) { src[k] = v; dst[k] = v + 1; ++k; }
      if (y + 1 < side) { src[k] = v; dst[k] = v + side; ++k; }
    }
  /* offset table: all (dx,dy) with 2 <= |dx|+|dy| <= max_l1 */
  int32_t n_off = 0;
  int32_t *offs = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)(2 * max_l1 + 1) * (2 * max_l1 + 1));
  if (!offs) return -1;
  for (int32_t dy = -max_l1; dy <= max_l1; ++dy)
    for (int32_t dx = -max_l1; dx <= max_l1; ++dx) {
      int32_t l1 = (dx < 0 ? -dx : dx) + (dy < 0 ? -dy : dy);
      if (l1 >= 2 && l1 <= max_l1) { offs[2 * n_off] = dx; offs[2 * n_off + 1] = dy; ++n_off; }
    }
  const uint64_t base = gg_mix(seed ^ 0x4752494453484F52ull);
  const uint64_t nv = (uint64_t)side * (uint64_t)side;
  for (int64_t j = 0; j < n_short; ++j) {
    for (int32_t attempt = 0; attempt < 64; ++attempt) {
      uint64_t c0 = base + ((uint64_t)j * 64u + (uint64_t)attempt) * 2u;
      uint64_t u = gg_below(gg_mix(c0), nv);
      uint64_t o = gg_below(gg_mix(c0 + 1), (uint64_t)n_off);
      int64_t x = (int64_t)(u % side) + offs[2 * o], y = (int64_t)(u / side) + offs[2 * o + 1];
      if (x < 0 || y < 0 || x >= side || y >= side) continue;
      src[k] = (int32_t)u;
      dst[k] = (int32_t)(y * side + x);
      ++k;
      break;
    }
  }
  free(offs);
  return k;
}

static int gg_cmp_i32(const void *p, const void *q) {
  int32_t a = *(const int32_t *)p, b = *(const int32_t *)q;
  return (a > b) - (a < b);
}

static void gg_sort_row(int32_t *r, int64_t len) {
  if (len <= 32) {
    for (int64_t i = 1; i < len; ++i) {
      int32_t v = r[i];
      int64_t j = i - 1;
      while (j >= 0 && r[j] > v) { r[j + 1] = r[j]; --j; }
      r[j + 1] = v;
    }
  } else {
    qsort(r, (size_t)len, sizeof(int32_t), gg_cmp_i32);
  }
}

/*
 * CSR from an edge list.  Self-loops are dropped; with `symmetrize` every edge
 * (u,v) also yields (v,u); rows are sorted ascending and duplicates removed.
 * row_ptr has n+1 entries; col has room for `cap` entries.
 * Returns the arc count m, or -1 (out of host memory), -2 (cap too small),
 * -3 (m does not fit int32 offsets), -4 (vertex id out of range).
 */
int64_t gg_csr_from_edges(int64_t n, int64_t ne, const int32_t *src, const int32_t *dst, int32_t symmetrize,
                          int32_t *row_ptr, int32_t *col, int64_t cap) {
  int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  if (!cnt) return -1;
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (int64_t i = 0; i < ne; ++i) {
    int32_t s = src[i], t = dst[i];
    if (s < 0 || t < 0 || s >= n || t >= n) { bad |= 1; continue; }
    if (s == t) continue;
    __atomic_fetch_add(&cnt[s + 1], 1, __ATOMIC_RELAXED);
    if (symmetrize) __atomic_fetch_add(&cnt[t + 1], 1, __ATOMIC_RELAXED);
  }
  if (bad) { free(cnt); return -4; }
  for (int64_t v = 0; v < n; ++v) cnt[v + 1] += cnt[v];
  int64_t total = cnt[n];
  int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(total > 0 ? total : 1));
  int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!tmp || !cur) { free(cnt); free(tmp); free(cur); return -1; }
  memcpy(cur, cnt, sizeof(int64_t) * (size_t)n);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < ne; ++i) {
    int32_t s = src[i], t = dst[i];
    if (s == t) continue;
    tmp[__atomic_fetch_add(&cur[s], 1, __ATOMIC_RELAXED)] = t;
    if (symmetrize) tmp[__atomic_fetch_add(&cur[t], 1, __ATOMIC_RELAXED)] = s;
  }
  /* sort + dedup each row in place; cur[v] becomes the deduplicated length */
#pragma omp parallel for schedule(dynamic, 4096)
  for (int64_t v = 0; v < n; ++v) {
    int32_t *r = tmp + cnt[v];
    int64_t len = cnt[v + 1] - cnt[v], w = 0;
    gg_sort_row(r, len);
    for (int64_t i = 0; i < len; ++i)
      if (w == 0 || r[i] != r[w - 1]) r[w++] = r[i];
    cur[v] = w;
  }
  int64_t m = 0;
  for (int64_t v = 0; v < n; ++v) m += cur[v];
  if (m > cap) { free(cnt); free(tmp); free(cur); return -2; }
  if (m > 2147483647ll) { free(cnt); free(tmp); free(cur); return -3; }
  /* exclusive scan of the new lengths into row_ptr, then compact */
  int64_t acc = 0;
  for (int64_t v = 0; v < n; ++v) { row_ptr[v] = (int32_t)acc; acc += cur[v]; }
  row_ptr[n] = (int32_t)acc;
#pragma omp parallel for schedule(dynamic, 4096)
  for (int64_t v = 0; v < n; ++v)
    memcpy(col + row_ptr[v], tmp + cnt[v], sizeof(int32_t) * (size_t)cur[v]);
  free(cnt); free(tmp); free(cur);
  return m;
}

/*
 * Symmetric pair-hash weights: w(u,v) = lo + mix(mix(seed) ^ (min<<32 | max)) mod (hi-lo),
 * so both arcs of an undirected edge carry the same weight in [lo, hi).
 */
void gg_pair_weights(int64_t n, const int32_t *row_ptr, const int32_t *col, uint64_t seed, int32_t lo,
                     int32_t hi, int32_t *wt) {
  const uint64_t base = gg_mix(seed ^ 0x5745494748545321ull);
  const uint64_t span = (uint64_t)(hi - lo);
#pragma omp parallel for schedule(dynamic, 4096)
  for (int64_t u = 0; u < n; ++u)
    for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
      uint64_t a = (uint64_t)(u < col[e] ? u : col[e]), b = (uint64_t)(u < col[e] ? col[e] : u);
      wt[e] = lo + (int32_t)(gg_mix(base ^ ((a << 32) | b)) % span);
    }
}

/* k sources drawn uniformly (with replacement) among vertices with out-degree >= 1. */
int32_t gg_pick_sources(int64_t n, const int32_t *row_ptr, uint64_t seed, int32_t k, int32_t *out) {
  const uint64_t base = gg_mix(seed ^ 0x534F555243455321ull);
  uint64_t ctr = 0;
  for (int32_t i = 0; i < k; ++i) {
    int found = 0;
    for (int32_t tries = 0; tries < 1000000 && !found; ++tries) {
      uint64_t v = gg_below(gg_mix(base + ctr++), (uint64_t)n);
      if (row_ptr[v + 1] > row_ptr[v]) { out[i] = (int32_t)v; found = 1; }
    }
    if (!found) return i;
  }
  return k;
}
