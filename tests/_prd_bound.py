"""Which PageRankDelta differences a threshold flip can explain (test helper).

PageRankDelta (Fig. 1) keeps v active for the next round iff
|Delta(v)| > eps * Rank(v).  The GPU computes Delta and Rank in FP32 and the
oracle in FP64, so a vertex whose margin |Delta| - eps*Rank is within rounding
of zero may take the other branch.  Such a flip changes whether Delta(v) is
propagated, which moves the ranks of the vertices downstream by at most the
propagated mass.  This module bounds that effect from the oracle's per-round
history, round by round:

  S_r(v)  magnitude scale of the round-r sum that forms Delta_r(v)
          (d * sum over in-arcs of |Delta_{r-1}(u)|/deg(u); round 1 adds the
          base terms), so tau * S_r bounds the new FP32 rounding of Delta_r(v);
  D_r(v)  bound on the rounding error of Delta_r(v), old errors carried
          along the arcs: D_r = d * sum over in-arcs (u, v) of
          D_{r-1}(u)/deg(u) + tau * (S_r + |Delta_r|).  Late rounds form
          Delta by heavy cancellation, so D_r can exceed |Delta_r| itself;
  A_r(v)  bound on |Delta_gpu - Delta_oracle| caused by earlier flips:
          A_r = d * sum over in-arcs (u, v) of (A_{r-1}(u) + N_{r-1}(u) *
          (|Delta_{r-1}(u)| + D_{r-1}(u) + A_{r-1}(u))) / deg(u), N = the
          flip-possible set;
  R_r(v)  bound on the rank deviation caused by flips: R_r = R_{r-1} + A_r;
  N_r     vertices whose margin is within D_r + A_r + eps*(E_r + R_r) of zero
          (E_r = sum of D and tau*Rank over rounds <= r: the rounding of
          Rank), i.e. whose decision the GPU may legitimately take the other
          way.

tau = 1e-5 bounds the relative rounding of one FP32 Delta or Rank: at most
~64 roundings of 2^-24 each (32 serial adds per thread, a reduction tree of
depth <= 12, the vertex update), 64 * 6e-8 < 1e-5.  A GPU result is explained
when every vertex is within tol * Rank + R_final(v) of the oracle and every
round's frontier size is within |N_{r-1}| of the oracle's.
"""
from __future__ import annotations

import numpy as np

import oracle

TAU = 1e-5


class FlipBound:
    def __init__(self, hg, eps, iters, damping=0.85, tau=TAU):
        self.rank, self.fs, dh, rh = oracle.prdelta(hg, damping, eps, iters, history=True)
        n = hg.n
        rp = np.asarray(hg.row_ptr, np.int64)
        col = np.asarray(hg.col, np.int64)
        deg = np.diff(rp).astype(np.float64)
        inv = np.where(deg > 0, 1.0 / np.maximum(deg, 1.0), 0.0)
        src = np.repeat(np.arange(n), np.diff(rp))

        def spread(x):  # d * sum over arcs (u, w) of x[u] / deg(u), per destination w
            return damping * np.bincount(col, weights=(x * inv)[src], minlength=n)

        A = np.zeros(n)
        R = np.zeros(n)
        E = np.zeros(n)
        D = np.zeros(n)
        near_prev = np.zeros(n, bool)
        self.near_counts = []
        for r in range(iters):
            if r == 0:
                S = spread(np.full(n, 1.0 / n)) + (1.0 - damping) / n + 1.0 / n
            else:
                A = spread(A + near_prev * (np.abs(dh[r - 1]) + D + A))
                S = spread(np.abs(dh[r - 1]))
            D = (spread(D) if r > 0 else 0.0) + tau * (S + np.abs(dh[r]))
            R = R + A
            E = E + D + tau * rh[r]
            margin = np.abs(dh[r]) - eps * rh[r]
            near_prev = np.abs(margin) <= D + A + eps * (E + R)
            self.near_counts.append(int(near_prev.sum()))
        self.rank_dev = R
        self.n = n

    def violations(self, got_rank, got_frontier, tol):
        """Vertices and rounds the flips cannot explain (empty lists = explained)."""
        got = np.asarray(got_rank, np.float64)
        bad_v = np.flatnonzero(np.abs(got - self.rank) > tol * np.abs(self.rank) + self.rank_dev)
        bad_r = []
        for r in range(1, min(len(got_frontier), len(self.fs))):
            if abs(int(got_frontier[r]) - int(self.fs[r])) > self.near_counts[r - 1]:
                bad_r.append(r)
        if len(got_frontier) and int(got_frontier[0]) != int(self.fs[0]):
            bad_r.insert(0, 0)
        return bad_v.tolist(), bad_r


def prdelta_fp32(hg, damping, eps, iters):
    """Fig. 1 in FP32 arithmetic with numpy (a CPU stand-in for an FP32
    implementation, used only to exercise FlipBound): (rank, frontier sizes)."""
    n = hg.n
    f = np.float32
    rp = np.asarray(hg.row_ptr, np.int64)
    col = np.asarray(hg.col, np.int64)
    deg = np.diff(rp)
    inv = np.where(deg > 0, (f(1) / np.maximum(deg, 1).astype(f)), f(0)).astype(f)
    src = np.repeat(np.arange(n), deg)
    rank = np.zeros(n, f)
    delta = np.full(n, f(1) / f(n), f)
    front = np.ones(n, bool)
    fs = []
    base, inv_n = f((1 - damping) / n), f(1) / f(n)
    a = f(damping)
    for r in range(iters):
        fs.append(int(front.sum()))
        contrib = np.where(front, delta * inv, f(0)).astype(f)
        dsum = np.zeros(n, f)
        np.add.at(dsum, col, contrib[src])
        if r == 0:
            delta = (a * dsum + base).astype(f)
            rank = (rank + delta).astype(f)
            delta = (delta - inv_n).astype(f)
        else:
            delta = (a * dsum).astype(f)
            rank = (rank + delta).astype(f)
        front = np.abs(delta) > f(eps) * rank
    return rank, np.array(fs, np.int64)
