/*
 * ORACLE -- test infrastructure only.
 *
 * Plain, slow, single-threaded C implementations of what the edgeset-apply hot
 * path computes, used to check the CUDA library.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load this file; the product
 * path never does.  It shares no code, header or constant with the CUDA side.
 *
 * Graphs are CSR arrays (rp[n+1], ci[m], optional wt[m]); "in" arrays are the
 * CSC (in-edges).  For symmetric graphs the caller passes the CSR twice.
 * Floating point is double throughout.
 *
 * Parity pins (tests/test_oracle_*.py): brute force on tiny graphs, SciPy's
 * textbook routines (BFS order, Dijkstra, connected components), closed forms
 * (grid Manhattan distances, uniform PageRank on regular graphs, the PageRank
 * mass recurrence), the worked from() example of Sec. 5, and central finite
 * differences for the MLP gradient, and for BC the pair-dependency definition
 * evaluated from all-pairs BFS on tiny graphs, path/star/cycle/complete-graph
 * closed forms, grid path counts (binomials) and NetworkX's betweenness.  The
 * schedule *choice* of the learned
 * selector is timing-dependent and has no pin ("parity unpinned"); only its
 * features and the outputs of whatever schedule it picks are pinned.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ CSR --- */

/*
 * Structural checks of an input graph: offsets start at 0, are monotone and end
 * at m; indices in range; each row strictly ascending (so no duplicates); no
 * self-loops; and, if asked, every arc (u,v) has its reverse (v,u).
 * Returns 0 if valid, else a positive code naming the first failed check.
 */
int or_validate_csr(int64_t n, int64_t m, const int32_t *rp, const int32_t *ci, int require_symmetric) {
  if (n < 0 || m < 0) return 1;
  if (rp[0] != 0 || rp[n] != m) return 2;
  for (int64_t v = 0; v < n; ++v)
    if (rp[v + 1] < rp[v]) return 3;
  for (int64_t v = 0; v < n; ++v)
    for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
      if (ci[e] < 0 || ci[e] >= n) return 4;
      if (ci[e] == v) return 5;
      if (e > rp[v] && ci[e] <= ci[e - 1]) return 6;
    }
  if (require_symmetric) {
    for (int64_t u = 0; u < n; ++u)
      for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
        int32_t v = ci[e];
        /* binary search for u in row v */
        int64_t lo = rp[v], hi = rp[v + 1];
        while (lo < hi) {
          int64_t mid = (lo + hi) / 2;
          if (ci[mid] < u) lo = mid + 1; else hi = mid;
        }
        if (lo >= rp[v + 1] || ci[lo] != u) return 7;
      }
  }
  return 0;
}

/* ------------------------------------------------ edgeset selection ---- */

/*
 * Table 2 operator semantics: edges.from(F).to(T).srcFilter(fs).dstFilter(fd)
 * selects {(u,v) : u in F, v in T, fs(u), fd(v)}; each selected edge is visited
 * once.  A NULL mask means "all".  The selected edges are written in push order
 * (u ascending, then v ascending as stored) up to cap; returns their count.
 */
int64_t or_edgeset_select(int64_t n, const int32_t *rp, const int32_t *ci, const uint8_t *from_mask,
                          const uint8_t *to_mask, const uint8_t *src_keep, const uint8_t *dst_keep,
                          int32_t *out_u, int32_t *out_v, int64_t cap) {
  int64_t k = 0;
  for (int64_t u = 0; u < n; ++u) {
    if (from_mask && !from_mask[u]) continue;
    if (src_keep && !src_keep[u]) continue;
    for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
      int32_t v = ci[e];
      if (to_mask && !to_mask[v]) continue;
      if (dst_keep && !dst_keep[v]) continue;
      if (k < cap) { out_u[k] = (int32_t)u; out_v[k] = v; }
      ++k;
    }
  }
  return k;
}

/* ----------------------------------------------------------------- BFS --- */

/*
 * Breadth-first search from src with a FIFO queue (depth[src] = 0, -1 when
 * unreached).  Parent follows a fixed canonical rule because the paper leaves
 * it open: parent[v] is the smallest-id in-neighbour w with
 * depth[w] = depth[v]-1; parent[src] = src; -1 when unreached.
 * level_sizes (optional, cap entries) receives the number of vertices at each
 * depth.  Returns the number of levels (max depth + 1), 0 if src is invalid.
 */
int32_t or_bfs(int64_t n, const int32_t *rp, const int32_t *ci, const int32_t *in_rp, const int32_t *in_ci,
               int32_t src, int32_t *depth, int32_t *parent, int64_t *level_sizes, int32_t cap) {
  for (int64_t v = 0; v < n; ++v) { depth[v] = -1; if (parent) parent[v] = -1; }
  if (src < 0 || src >= n) return 0;
  int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int64_t head = 0, tail = 0;
  queue[tail++] = src;
  depth[src] = 0;
  int32_t levels = 1;
  while (head < tail) {
    int32_t u = queue[head++];
    for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
      int32_t v = ci[e];
      if (depth[v] == -1) {
        depth[v] = depth[u] + 1;
        if (depth[v] + 1 > levels) levels = depth[v] + 1;
        queue[tail++] = v;
      }
    }
  }
  free(queue);
  if (level_sizes) {
    for (int32_t l = 0; l < cap; ++l) level_sizes[l] = 0;
    for (int64_t v = 0; v < n; ++v)
      if (depth[v] >= 0 && depth[v] < cap) level_sizes[depth[v]]++;
  }
  if (parent) {
    for (int64_t v = 0; v < n; ++v) {
      if (depth[v] <= 0) continue;
      for (int64_t e = in_rp[v]; e < in_rp[v + 1]; ++e) {
        int32_t w = in_ci[e];
        if (depth[w] == depth[v] - 1 && (parent[v] == -1 || w < parent[v])) parent[v] = w;
      }
    }
    parent[src] = src;
  }
  return levels;
}

/* ---------------------------------------------------------------- SSSP --- */

/*
 * Frontier-based Bellman-Ford on integer weights (Sec. 7 runs Bellman-Ford;
 * Sec. 6 allows asyncMin updates).  Rounds are synchronous: round r relaxes the
 * out-arcs of the vertices whose distance dropped in round r-1, each using its
 * distance as it stood at the start of the round; the vertices whose distance
 * dropped form the next frontier.  dist = INT32_MAX when unreachable.
 * frontier_sizes (optional, cap entries) receives |F| per round.  Returns the
 * number of rounds executed (rounds with a non-empty frontier).
 */
int32_t or_sssp(int64_t n, const int32_t *rp, const int32_t *ci, const int32_t *wt, int32_t src,
                int32_t *dist, int64_t *frontier_sizes, int32_t cap) {
  for (int64_t v = 0; v < n; ++v) dist[v] = INT32_MAX;
  if (src < 0 || src >= n) return 0;
  int32_t *front = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int32_t *front_d = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  uint8_t *in_next = (uint8_t *)calloc((size_t)n, 1);
  int32_t *next = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  dist[src] = 0;
  int64_t nf = 1;
  front[0] = src;
  int32_t rounds = 0;
  while (nf > 0) {
    if (frontier_sizes && rounds < cap) frontier_sizes[rounds] = nf;
    for (int64_t i = 0; i < nf; ++i) front_d[i] = dist[front[i]];  /* start-of-round values */
    int64_t nn = 0;
    for (int64_t i = 0; i < nf; ++i) {
      int32_t u = front[i];
      for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
        int32_t v = ci[e];
        int64_t nd = (int64_t)front_d[i] + wt[e];
        if (nd < dist[v]) {
          dist[v] = (int32_t)nd;
          if (!in_next[v]) { in_next[v] = 1; next[nn++] = v; }
        }
      }
    }
    for (int64_t i = 0; i < nn; ++i) in_next[next[i]] = 0;
    memcpy(front, next, sizeof(int32_t) * (size_t)nn);
    nf = nn;
    ++rounds;
  }
  free(front); free(front_d); free(in_next); free(next);
  return rounds;
}

/* ------------------------------------------------------------------ CC --- */

/*
 * Synchronous min-label propagation (the label-propagation CC of Sec. 7):
 * label_0[v] = v, all vertices active; in each round every active u offers its
 * start-of-round label to its out-neighbours, which keep the minimum; vertices
 * whose label dropped are active in the next round.  Stops when no label
 * changes.  Returns the number of rounds executed.
 */
int32_t or_cc(int64_t n, const int32_t *rp, const int32_t *ci, int32_t *label, int64_t *frontier_sizes,
              int32_t cap) {
  int32_t *front = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int32_t *front_l = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int32_t *next = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  uint8_t *in_next = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
  for (int64_t v = 0; v < n; ++v) { label[v] = (int32_t)v; front[v] = (int32_t)v; }
  int64_t nf = n;
  int32_t rounds = 0;
  while (nf > 0) {
    if (frontier_sizes && rounds < cap) frontier_sizes[rounds] = nf;
    for (int64_t i = 0; i < nf; ++i) front_l[i] = label[front[i]];
    int64_t nn = 0;
    for (int64_t i = 0; i < nf; ++i) {
      int32_t u = front[i];
      for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
        int32_t v = ci[e];
        if (front_l[i] < label[v]) {
          label[v] = front_l[i];
          if (!in_next[v]) { in_next[v] = 1; next[nn++] = v; }
        }
      }
    }
    for (int64_t i = 0; i < nn; ++i) in_next[next[i]] = 0;
    memcpy(front, next, sizeof(int32_t) * (size_t)nn);
    nf = nn;
    ++rounds;
  }
  free(front); free(front_l); free(next); free(in_next);
  return rounds;
}

/* ------------------------------------------------------------------ BC --- */

/*
 * Single-source betweenness dependencies, the per-source term of Betweenness
 * Centrality (Sec. 7 runs BC from single starting points, synchronously, as
 * two edgeset applies: a forward path-counting BFS and a backward dependency
 * accumulation).  The paper prints no formula; this is Brandes' algorithm
 * (2001) as published:
 *   forward: BFS from src over out-arcs; sigma[w] = number of shortest
 *     src-w paths = sum of sigma[v] over the predecessors v of w (arcs (v,w)
 *     with d(v) = d(w) - 1); sigma[src] = 1;
 *   backward: every w in order of non-increasing distance (reverse BFS
 *     order) passes to each predecessor v the share
 *     delta[v] += sigma[v] / sigma[w] * (1 + delta[w]).
 * Predecessors are read from the in-arcs (in_rp, in_ci; the CSR twice for a
 * symmetric graph).  delta[src] = 0; unreached vertices have sigma = delta = 0.
 * Returns the number of BFS levels (0 if src is invalid).
 */
int32_t or_bc(int64_t n, const int32_t *rp, const int32_t *ci, const int32_t *in_rp, const int32_t *in_ci,
              int32_t src, double *delta, double *sigma) {
  for (int64_t v = 0; v < n; ++v) { delta[v] = 0.0; sigma[v] = 0.0; }
  if (src < 0 || src >= n) return 0;
  int32_t *d = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  for (int64_t v = 0; v < n; ++v) d[v] = -1;
  int64_t head = 0, tail = 0;
  order[tail++] = src;
  d[src] = 0;
  sigma[src] = 1.0;
  while (head < tail) {
    int32_t v = order[head++];
    for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
      int32_t w = ci[e];
      if (d[w] < 0) {
        d[w] = d[v] + 1;
        order[tail++] = w;
      }
      if (d[w] == d[v] + 1) sigma[w] += sigma[v];
    }
  }
  for (int64_t i = tail - 1; i >= 0; --i) {
    int32_t w = order[i];
    for (int64_t e = in_rp[w]; e < in_rp[w + 1]; ++e) {
      int32_t v = in_ci[e];
      if (d[v] >= 0 && d[v] == d[w] - 1) delta[v] += sigma[v] / sigma[w] * (1.0 + delta[w]);
    }
  }
  delta[src] = 0.0;
  int32_t levels = d[order[tail - 1]] + 1;
  free(d);
  free(order);
  return levels;
}

/* ------------------------------------------------------------ PageRank --- */

/*
 * PageRank power iteration (the PR of Sec. 7, 20 iterations; the paper prints
 * no formula, so the standard one consistent with the base score (1-d)/V of
 * the PageRankDelta code in Sec. 3 is used):
 *   PR_0[v] = 1/V,  PR_{k+1}[v] = (1-d)/V + d * sum_{u in in(v)} PR_k[u] / outdeg(u).
 * Vertices without out-arcs contribute nothing.  After the last iteration the
 * ranks are divided by their sum.  out_deg[u] = number of out-arcs of u.
 */
void or_pagerank(int64_t n, const int32_t *in_rp, const int32_t *in_ci, const int32_t *out_deg, double d,
                 int32_t iters, int32_t normalize, double *rank) {
  double *cur = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (int64_t v = 0; v < n; ++v) cur[v] = 1.0 / (double)n;
  for (int32_t k = 0; k < iters; ++k) {
    for (int64_t v = 0; v < n; ++v) {
      double s = 0.0;
      for (int64_t e = in_rp[v]; e < in_rp[v + 1]; ++e) s += cur[in_ci[e]] / (double)out_deg[in_ci[e]];
      rank[v] = (1.0 - d) / (double)n + d * s;
    }
    memcpy(cur, rank, sizeof(double) * (size_t)n);
  }
  if (iters == 0) memcpy(rank, cur, sizeof(double) * (size_t)n);
  if (normalize) {
    double total = 0.0;
    for (int64_t v = 0; v < n; ++v) total += rank[v];
    for (int64_t v = 0; v < n; ++v) rank[v] /= total;
  }
  free(cur);
}

/*
 * PageRankDelta, Fig. 1 / the GraphIt program of Fig. 3, for max_iter rounds:
 *   Rank = 0, DeltaSum = 0, Delta = 1/V, Frontier = all vertices.
 *   Each round: every frontier src adds Delta[src]/OutDegree[src] to
 *   DeltaSum[dst] of each out-neighbour dst; then every vertex v:
 *     round 1:  Delta = a*DeltaSum + (1-a)/V;  Rank += Delta;  Delta -= 1/V
 *     later:    Delta = a*DeltaSum;            Rank += Delta
 *     DeltaSum = 0;  v joins the next frontier iff |Delta| > eps*Rank.
 * In round 1, Rank is updated before 1/V is subtracted (the order of the
 * Fig. 3 code); with eps = 0 this makes Rank after round k equal PR_k.
 * frontier_sizes (optional) receives |Frontier| at the start of each round.
 * delta_hist / rank_hist (optional, max_iter*n doubles each) receive Delta and
 * Rank of every vertex at the end of each round (row round-1), i.e. the two
 * values whose comparison |Delta| > eps*Rank decides the next frontier.
 */
void or_prdelta(int64_t n, const int32_t *rp, const int32_t *ci, double a, double eps, int32_t max_iter,
                double *rank, int64_t *frontier_sizes, double *delta_hist, double *rank_hist) {
  double *delta = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double *dsum = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  uint8_t *front = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
  for (int64_t v = 0; v < n; ++v) { rank[v] = 0.0; delta[v] = 1.0 / (double)n; front[v] = 1; }
  for (int32_t round = 1; round <= max_iter; ++round) {
    int64_t nf = 0;
    for (int64_t u = 0; u < n; ++u) {
      if (!front[u]) continue;
      ++nf;
      int64_t deg = rp[u + 1] - rp[u];
      for (int64_t e = rp[u]; e < rp[u + 1]; ++e) dsum[ci[e]] += delta[u] / (double)deg;
    }
    if (frontier_sizes) frontier_sizes[round - 1] = nf;
    for (int64_t v = 0; v < n; ++v) {
      if (round == 1) {
        delta[v] = a * dsum[v] + (1.0 - a) / (double)n;
        rank[v] += delta[v];
        delta[v] -= 1.0 / (double)n;
      } else {
        delta[v] = a * dsum[v];
        rank[v] += delta[v];
      }
      dsum[v] = 0.0;
      front[v] = fabs(delta[v]) > eps * rank[v];
    }
    if (delta_hist) memcpy(delta_hist + (size_t)(round - 1) * (size_t)n, delta, sizeof(double) * (size_t)n);
    if (rank_hist) memcpy(rank_hist + (size_t)(round - 1) * (size_t)n, rank, sizeof(double) * (size_t)n);
  }
  free(delta); free(dsum); free(front);
}

/* -------------------------------------------- frontier statistics ------ */

/*
 * Quantities the direction heuristics read (Sec. 2, hybrid traversal): for a
 * frontier mask F and a visited mask: out[0] = |F|, out[1] = m_f = sum of
 * out-degrees over F, out[2] = n_u = unvisited vertices, out[3] = m_u = sum of
 * out-degrees over unvisited vertices.  visited may be NULL (then n_u = m_u = 0).
 */
void or_frontier_stats(int64_t n, const int32_t *rp, const uint8_t *front, const uint8_t *visited,
                       int64_t *out) {
  int64_t nf = 0, mf = 0, nu = 0, mu = 0;
  for (int64_t v = 0; v < n; ++v) {
    int64_t deg = rp[v + 1] - rp[v];
    if (front[v]) { ++nf; mf += deg; }
    if (visited && !visited[v]) { ++nu; mu += deg; }
  }
  out[0] = nf; out[1] = mf; out[2] = nu; out[3] = mu;
}

/*
 * Beamer's direction-optimising rule (Beamer et al. 2012, which the paper
 * adopts through Ligra for its hybrid schedules): while pushing, switch to pull
 * when m_f > m_u / alpha; while pulling, switch back to push when |F| < V / beta.
 * Returns 1 for pull, 0 for push.
 */
int32_t or_beamer(int64_t n, int64_t nf, int64_t mf, int64_t mu, int32_t was_pull, double alpha, double beta) {
  if (!was_pull) return (double)mf > (double)mu / alpha ? 1 : 0;
  return (double)nf < (double)n / beta ? 0 : 1;
}

/* Ligra's rule (the one used in the Ligra PageRankDelta listing): pull iff |F| + m_f > m / 20. */
int32_t or_ligra_dense(int64_t m, int64_t nf, int64_t mf) { return (nf + mf) > m / 20 ? 1 : 0; }

/* --------------------------------------------------------------- MLP --- */
/*
 * The learned schedule selector: 16 -> 64 -> 64 -> 3 perceptron with ReLU on
 * the two hidden layers and a linear output (predicted log-time of each
 * schedule).  Parameters are packed as W1[64][16], b1[64], W2[64][64], b2[64],
 * W3[3][64], b3[3] (row-major, out x in).  This is not from the paper.
 */
#define OR_D_IN 16
#define OR_H 64
#define OR_D_OUT 3
#define OR_NPARAM (OR_H * OR_D_IN + OR_H + OR_H * OR_H + OR_H + OR_D_OUT * OR_H + OR_D_OUT)

int32_t or_mlp_num_params(void) { return OR_NPARAM; }

static void or_mlp_one(const double *p, const double *x, double *h1, double *h2, double *y) {
  const double *W1 = p, *b1 = W1 + OR_H * OR_D_IN, *W2 = b1 + OR_H, *b2 = W2 + OR_H * OR_H,
               *W3 = b2 + OR_H, *b3 = W3 + OR_D_OUT * OR_H;
  for (int j = 0; j < OR_H; ++j) {
    double s = b1[j];
    for (int i = 0; i < OR_D_IN; ++i) s += W1[j * OR_D_IN + i] * x[i];
    h1[j] = s > 0 ? s : 0;
  }
  for (int j = 0; j < OR_H; ++j) {
    double s = b2[j];
    for (int i = 0; i < OR_H; ++i) s += W2[j * OR_H + i] * h1[i];
    h2[j] = s > 0 ? s : 0;
  }
  for (int j = 0; j < OR_D_OUT; ++j) {
    double s = b3[j];
    for (int i = 0; i < OR_H; ++i) s += W3[j * OR_H + i] * h2[i];
    y[j] = s;
  }
}

void or_mlp_forward(const double *params, const double *X, int64_t B, double *Y) {
  double h1[OR_H], h2[OR_H];
  for (int64_t b = 0; b < B; ++b) or_mlp_one(params, X + b * OR_D_IN, h1, h2, Y + b * OR_D_OUT);
}

/*
 * Masked mean-squared error L = sum_{b,j} M[b,j] (Y[b,j] - T[b,j])^2 / sum M and its
 * gradient with respect to every parameter (backpropagation written out layer
 * by layer).  Returns L; grad has OR_NPARAM entries.
 */
double or_mlp_loss_grad(const double *params, const double *X, const double *T, const double *M, int64_t B,
                        double *grad) {
  const double *W2 = params + OR_H * OR_D_IN + OR_H, *W3 = W2 + OR_H * OR_H + OR_H;
  double *gW1 = grad, *gb1 = gW1 + OR_H * OR_D_IN, *gW2 = gb1 + OR_H, *gb2 = gW2 + OR_H * OR_H,
         *gW3 = gb2 + OR_H, *gb3 = gW3 + OR_D_OUT * OR_H;
  memset(grad, 0, sizeof(double) * OR_NPARAM);
  double msum = 0.0;
  for (int64_t b = 0; b < B * OR_D_OUT; ++b) msum += M[b];
  if (msum <= 0) return 0.0;
  double loss = 0.0;
  double h1[OR_H], h2[OR_H], y[OR_D_OUT], dy[OR_D_OUT], dh2[OR_H], dh1[OR_H];
  for (int64_t b = 0; b < B; ++b) {
    const double *x = X + b * OR_D_IN;
    or_mlp_one(params, x, h1, h2, y);
    for (int j = 0; j < OR_D_OUT; ++j) {
      double r = y[j] - T[b * OR_D_OUT + j], mk = M[b * OR_D_OUT + j];
      loss += mk * r * r;
      dy[j] = 2.0 * mk * r / msum;
    }
    for (int j = 0; j < OR_D_OUT; ++j) {
      gb3[j] += dy[j];
      for (int i = 0; i < OR_H; ++i) gW3[j * OR_H + i] += dy[j] * h2[i];
    }
    for (int i = 0; i < OR_H; ++i) {
      double s = 0.0;
      for (int j = 0; j < OR_D_OUT; ++j) s += W3[j * OR_H + i] * dy[j];
      dh2[i] = h2[i] > 0 ? s : 0.0;
    }
    for (int j = 0; j < OR_H; ++j) {
      gb2[j] += dh2[j];
      for (int i = 0; i < OR_H; ++i) gW2[j * OR_H + i] += dh2[j] * h1[i];
    }
    for (int i = 0; i < OR_H; ++i) {
      double s = 0.0;
      for (int j = 0; j < OR_H; ++j) s += W2[j * OR_H + i] * dh2[j];
      dh1[i] = h1[i] > 0 ? s : 0.0;
    }
    for (int j = 0; j < OR_H; ++j) {
      gb1[j] += dh1[j];
      for (int i = 0; i < OR_D_IN; ++i) gW1[j * OR_D_IN + i] += dh1[j] * x[i];
    }
  }
  return loss / msum;
}

/*
 * One Adam step (Kingma & Ba 2015) at step number t >= 1:
 *   m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
 *   p -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).
 */
void or_adam_step(int64_t np, double *p, const double *g, double *m, double *v, int32_t t, double lr, double b1,
                  double b2, double eps) {
  double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
  for (int64_t i = 0; i < np; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * g[i];
    v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
    p[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
  }
}

/*
 * Selector features of one traversal level (not from the paper).  Inputs are
 * the graph size (n, m, max out-degree), the frontier statistics of
 * or_frontier_stats, the level index, whether the previous level pulled and the
 * previous frontier size.  x receives 16 values:
 *   0 lg|F|  1 lg m_f  2 lg n_u  3 lg m_u  4 lg V  5 lg E  6 |F|/V  7 m_f/E
 *   8 n_u/V  9 m_u/E  10 lg(m_f/|F|)  11 lg maxdeg  12 lg(E/V)  13 lg level
 *   14 was_pull  15 lg|F_prev|        where lg(z) = log2(1 + z).
 */
void or_features(int64_t n, int64_t m, int64_t maxdeg, int64_t nf, int64_t mf, int64_t nu, int64_t mu,
                 int32_t level, int32_t was_pull, int64_t nf_prev, double *x) {
  double V = (double)(n > 0 ? n : 1), E = (double)(m > 0 ? m : 1);
  x[0] = log2(1.0 + (double)nf);
  x[1] = log2(1.0 + (double)mf);
  x[2] = log2(1.0 + (double)nu);
  x[3] = log2(1.0 + (double)mu);
  x[4] = log2(1.0 + (double)n);
  x[5] = log2(1.0 + (double)m);
  x[6] = (double)nf / V;
  x[7] = (double)mf / E;
  x[8] = (double)nu / V;
  x[9] = (double)mu / E;
  x[10] = log2(1.0 + (double)mf / (double)(nf > 0 ? nf : 1));
  x[11] = log2(1.0 + (double)maxdeg);
  x[12] = log2(1.0 + (double)m / V);
  x[13] = log2(1.0 + (double)level);
  x[14] = was_pull ? 1.0 : 0.0;
  x[15] = log2(1.0 + (double)nf_prev);
}
