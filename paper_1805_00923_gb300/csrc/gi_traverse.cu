// edgeset apply (Table 2 operators under the Table 3 direction choices).
#include "gi_traverse.cuh"

namespace gi {

static bool is_pull(int32_t dir) { return dir == GI_DIR_DENSE_PULL; }

int apply_dispatch(gi_graph *g, gi_vset *from, gi_vset *to, int32_t dir, const gi_schedule &sc, int32_t kernel_id,
                   const void *args, gi_vset *out, uint32_t flags, cudaStream_t s) {
  // Only BFS modifies each destination at most once, so only there may
  // deduplication be skipped without the output outgrowing the vertex count.
  const bool dedup = !(flags & GI_NO_DEDUP) || kernel_id != GI_K_BFS;
  if (out) GI_TRY(vset_clear(out, s));
  OutSet o = out_of(out, dedup);
  const uint32_t *to_bm = nullptr;
  if (to) {
    GI_TRY(vset_ensure_bitmap(to, s));
    to_bm = to->bitmap;
  }
  if (dir == GI_DIR_SPARSE_PULL) {
    // only the destinations of `to` pull (gi_edgeset_apply passes a non-NULL to)
    GI_TRY(vset_ensure_queue(to, s));
    FSet F;
    if (from) {
      if (sc.dense_rep == GI_REP_BOOL) {
        GI_TRY(vset_ensure_bool(from, s));
        F = FSet(static_cast<const uint8_t *>(from->boolmap));
      } else {
        GI_TRY(vset_ensure_bitmap(from, s));
        F = FSet(static_cast<const uint32_t *>(from->bitmap));
      }
    }
    switch (kernel_id) {
      case GI_K_BFS: {
        const gi_bfs_args *a = static_cast<const gi_bfs_args *>(args);
        OpBFSPull op{a->depth, a->parent, a->level};
        GI_TRY(launch_pull_sparse(g, op, g->in, to->queue, to->count, 0, F, o, sc, s, kClassBfsPull));
        break;
      }
      case GI_K_SSSP: {
        const gi_sssp_args *a = static_cast<const gi_sssp_args *>(args);
        if (!g->symmetric && g->in.wt == nullptr) {
          gi::set_error("pull SSSP needs in-edge weights (gi_load_csc with weights)");
          return GI_ERR_UNSUPPORTED;
        }
        OpMinInt op{a->dist, a->snap, g->in.wt};
        GI_TRY(launch_pull_sparse(g, op, g->in, to->queue, to->count, 0, F, o, sc, s, kClassMinPull));
        break;
      }
      case GI_K_CC: {
        const gi_cc_args *a = static_cast<const gi_cc_args *>(args);
        OpMinInt op{a->label, a->snap, nullptr};
        GI_TRY(launch_pull_sparse(g, op, g->in, to->queue, to->count, 0, F, o, sc, s, kClassMinPull));
        break;
      }
      case GI_K_SUM: {
        const gi_sum_args *a = static_cast<const gi_sum_args *>(args);
        OpSum op{a->contrib, a->acc};
        GI_TRY(launch_pull_sparse(g, op, g->in, to->queue, to->count, 0, F, o, sc, s));
        break;
      }
      case GI_K_PROBE: {
        const gi_probe_args *a = static_cast<const gi_probe_args *>(args);
        OpProbe op{a->count, a->srcsum};
        GI_TRY(launch_pull_sparse(g, op, g->in, to->queue, to->count, 0, F, o, sc, s));
        break;
      }
      default:
        gi::set_error("unknown kernel_id %d", kernel_id);
        return GI_ERR_INVALID_ARG;
    }
  } else if (is_pull(dir)) {
    if (!g->has_csc) {
      gi::set_error("pull traversal needs the in-edges: load a symmetric graph or call gi_load_csc");
      return GI_ERR_UNSUPPORTED;
    }
    FSet F;
    if (from) {
      if (sc.dense_rep == GI_REP_BOOL) {
        GI_TRY(vset_ensure_bool(from, s));
        F = FSet(static_cast<const uint8_t *>(from->boolmap));
      } else {
        GI_TRY(vset_ensure_bitmap(from, s));
        F = FSet(static_cast<const uint32_t *>(from->bitmap));
      }
    }
    const bool vp = sc.balance == GI_BAL_VERTEX;
    switch (kernel_id) {
      case GI_K_BFS: {
        const gi_bfs_args *a = static_cast<const gi_bfs_args *>(args);
        int32_t tw = sc.balance == GI_BAL_VERTEX ? INT32_MAX : (sc.t_warp > 0 ? sc.t_warp : 32);
        // rows long enough to be deferred exist only above this degree; and
        // once 1/64 of the arcs leave the frontier, a row's first kBfsScanCap
        // arcs all miss it with probability about e^-16, so the deferred pass
        // (one more launch) is left out
        const bool long_rows = (g->symmetric ? (int64_t)g->max_deg : g->m) > kBfsScanCap + kBfsDeferChunk + 4;
        const int64_t mf = from == g->hint_vset ? g->hint_mf : -1;
        const bool sparse_front = mf < 0 || mf * 64 < g->m;
        void *defer = nullptr;
        const int32_t dcap = bfs_defer_cap(g->m);
        if (tw != INT32_MAX && long_rows && sparse_front) {
          GI_TRY(bfs_defer_get(g, s));
          defer = g->bfs_defer;
        }
        const int tok = timing_begin(kClassBfsPull, s);
        k_pull_bfs<<<grid_for(g, g->n, 256), 256, 0, s>>>(g->in.ptr, g->in.idx, g->n, F, to_bm, a->depth, a->parent,
                                                          a->level, tw, o.bm, o.q, o.qc, nullptr, defer, dcap,
                                                          to_bm == nullptr ? g->bfs_unv_query : BfsUnv{});
        if (defer)
          k_pull_bfs_deferred<<<g->num_sms * 8, 256, 0, s>>>(g->in.ptr, g->in.idx, F, defer, dcap, a->depth,
                                                              a->parent, a->level, o.bm, o.q, o.qc);
        timing_end(tok, s);
        GI_LAUNCH_CHECK();
        break;
      }
      case GI_K_SSSP: {
        const gi_sssp_args *a = static_cast<const gi_sssp_args *>(args);
        if (!g->symmetric && g->in.wt == nullptr) {
          gi::set_error("pull SSSP needs in-edge weights (gi_load_csc with weights)");
          return GI_ERR_UNSUPPORTED;
        }
        OpMinInt op{a->dist, a->snap, g->in.wt};
        GI_TRY(launch_pull_tiled(g, op, g->in, g->in_tiles, F, to_bm, o, s, kClassMinPull, vp));
        break;
      }
      case GI_K_CC: {
        const gi_cc_args *a = static_cast<const gi_cc_args *>(args);
        OpMinInt op{a->label, a->snap, nullptr};
        GI_TRY(launch_pull_tiled(g, op, g->in, g->in_tiles, F, to_bm, o, s, kClassMinPull, vp));
        break;
      }
      case GI_K_SUM: {
        const gi_sum_args *a = static_cast<const gi_sum_args *>(args);
        OpSum op{a->contrib, a->acc};
        GI_TRY(launch_pull_tiled(g, op, g->in, g->in_tiles, F, to_bm, o, s, kClassOtherPull, vp));
        break;
      }
      case GI_K_PROBE: {
        const gi_probe_args *a = static_cast<const gi_probe_args *>(args);
        OpProbe op{a->count, a->srcsum};
        GI_TRY(launch_pull_tiled(g, op, g->in, g->in_tiles, F, to_bm, o, s, kClassOtherPull, vp));
        break;
      }
      default:
        gi::set_error("unknown kernel_id %d", kernel_id);
        return GI_ERR_INVALID_ARG;
    }
  } else {
    int mode = kSrcAll;
    if (from) {
      if (dir == GI_DIR_SPARSE_PUSH) {
        GI_TRY(vset_ensure_queue(from, s));
        mode = kSrcQueue;
      } else if (sc.dense_rep == GI_REP_BOOL) {
        GI_TRY(vset_ensure_bool(from, s));
        mode = kSrcBitmap;
      } else {
        GI_TRY(vset_ensure_bitmap(from, s));
        mode = kSrcBitmap;
      }
    }
    switch (kernel_id) {
      case GI_K_BFS: {
        const gi_bfs_args *a = static_cast<const gi_bfs_args *>(args);
        OpBFS op{a->depth, a->parent, a->level};
        GI_TRY(launch_push(g, op, mode, from, to_bm, o, sc, s));
        break;
      }
      case GI_K_SSSP: {
        const gi_sssp_args *a = static_cast<const gi_sssp_args *>(args);
        OpMinInt op{a->dist, a->snap, g->out.wt};
        GI_TRY(launch_push(g, op, mode, from, to_bm, o, sc, s));
        break;
      }
      case GI_K_CC: {
        const gi_cc_args *a = static_cast<const gi_cc_args *>(args);
        OpMinInt op{a->label, a->snap, nullptr};
        GI_TRY(launch_push(g, op, mode, from, to_bm, o, sc, s));
        break;
      }
      case GI_K_SUM: {
        const gi_sum_args *a = static_cast<const gi_sum_args *>(args);
        OpSum op{a->contrib, a->acc};
        GI_TRY(launch_push(g, op, mode, from, to_bm, o, sc, s));
        break;
      }
      case GI_K_PROBE: {
        const gi_probe_args *a = static_cast<const gi_probe_args *>(args);
        OpProbe op{a->count, a->srcsum};
        GI_TRY(launch_push(g, op, mode, from, to_bm, o, sc, s));
        break;
      }
      default:
        gi::set_error("unknown kernel_id %d", kernel_id);
        return GI_ERR_INVALID_ARG;
    }
  }
  if (out) out->reps = GI_REP_SPARSE | GI_REP_BITMAP;
  return GI_OK;
}

int check_schedule(const gi_schedule *sc) {
  GI_ARG(sc != nullptr, "schedule is NULL");
  GI_ARG(sc->direction >= GI_DIR_SPARSE_PUSH && sc->direction <= GI_DIR_SPARSE_PULL, "unknown direction");
  GI_ARG(sc->balance == GI_BAL_VERTEX || sc->balance == GI_BAL_EDGE_AWARE || sc->balance == GI_BAL_EDGE_PARALLEL,
         "unknown balance mode");
  GI_ARG(sc->num_segments >= 1 && sc->num_segments <= 1024, "num_segments must be in [1, 1024]");
  GI_ARG(sc->rule == GI_RULE_BEAMER || sc->rule == GI_RULE_LIGRA, "unknown rule");
  GI_ARG(sc->dense_rep == GI_REP_BITMAP || sc->dense_rep == GI_REP_BOOL, "dense_rep must be GI_REP_BITMAP or BOOL");
  GI_ARG(sc->tile_edges == 0 || (sc->tile_edges >= 256 && sc->tile_edges <= 8192 &&
                                 (sc->tile_edges & (sc->tile_edges - 1)) == 0),
         "tile_edges must be a power of two in [256, 8192]");
  GI_ARG(sc->hot_cache >= 0 && sc->hot_cache <= 2, "hot_cache must be 0, 1 or 2");
  GI_ARG(sc->seg_strategy == GI_SEG_FVC || sc->seg_strategy == GI_SEG_EVC, "seg_strategy must be FVC or EVC");
  GI_ARG(sc->persistent >= 0 && sc->persistent <= 2, "persistent must be 0, 1 or 2");
  GI_ARG(sc->delta >= 0, "delta must be >= 0");
  GI_ARG(sc->block == 128 || sc->block == 256 || sc->block == 512, "block must be 128, 256 or 512");
  GI_ARG(sc->dst_list == 0 || sc->dst_list == 1, "dst_list must be 0 or 1");
  return GI_OK;
}

DecideParams decide_params(const gi_schedule &sc, int32_t level, bool track_unvisited) {
  DecideParams p{};
  p.level = level;
  p.rule = sc.rule;
  p.alpha = sc.alpha > 0 ? sc.alpha : 14.0f;
  p.beta = sc.beta > 0 ? sc.beta : 24.0f;
  p.track_unvisited = track_unvisited ? 1 : 0;
  p.hybrid_kind = sc.direction == GI_DIR_HYBRID_DPUSH ? GI_DIR_HYBRID_DPUSH : GI_DIR_HYBRID_PULL;
  if (forced_direction(sc.direction) >= 0) {
    p.mode = 0;
    p.forced = forced_direction(sc.direction);
  } else if (sc.direction == GI_DIR_LEARNED) {
    p.mode = 2;
  } else {
    p.mode = 1;
  }
  return p;
}

// keep the in-edge tiles at the schedule's tile size
int ensure_tiles(gi_graph *g, const gi_schedule &sc, cudaStream_t s) {
  int32_t te = sc.tile_edges > 0 ? sc.tile_edges : 2048;
  if (g->has_csc && g->in_tiles.tile_edges != te) GI_TRY(use_tiles(g, te, s));
  return GI_OK;
}

}  // namespace gi

using namespace gi;

extern "C" int gi_edgeset_apply(gi_graph *g, gi_vset *from, gi_vset *to, const gi_schedule *sched, int32_t kernel_id,
                                const void *kernel_args, gi_vset *out_modified, uint32_t flags, void *stream) {
  GI_ARG(g != nullptr, "graph is NULL");
  GI_TRY(check_schedule(sched));
  GI_ARG(kernel_args != nullptr, "kernel_args is NULL");
  GI_ARG(kernel_id >= GI_K_BFS && kernel_id <= GI_K_PROBE, "unknown kernel_id");
  GI_ARG(out_modified == nullptr || (out_modified != from && out_modified != to), "out_modified aliases an input");
  GI_ARG(!from || from->g == g, "from belongs to another graph");
  GI_ARG(!to || to->g == g, "to belongs to another graph");
  GI_ARG(!out_modified || out_modified->g == g, "out_modified belongs to another graph");
  if (kernel_id == GI_K_SSSP) GI_ARG(g->out.wt != nullptr, "GI_K_SSSP needs edge weights");
  cudaStream_t s = (cudaStream_t)stream;
  GI_TRY(ensure_tiles(g, *sched, s));
  int32_t dir = sched->direction;
  if (dir == GI_DIR_SPARSE_PULL) {
    if (!to) dir = GI_DIR_DENSE_PULL;  // every destination: the dense form
    if (!g->has_csc) {
      gi::set_error("pull traversal needs the in-edges: load a symmetric graph or call gi_load_csc");
      return GI_ERR_UNSUPPORTED;
    }
  } else if (dir > GI_DIR_DENSE_PULL) {
    if (!from) {
      dir = GI_DIR_DENSE_PULL;
    } else {
      DecideParams p = decide_params(*sched, 0, false);
      GI_TRY(ctrl_init(g, 0, 0, s));
      GI_TRY(frontier_decide(g, from, p, s));
      GI_TRY(ctrl_fetch(g, s));
      dir = (int32_t)g->ctrl_host[kDecision];
    }
    if (dir == GI_DIR_DENSE_PULL && !g->has_csc) dir = GI_DIR_DENSE_PUSH;
    if (from) {  // |from| was just read back with the statistics
      g->hint_vset = from;
      g->hint_nf = g->ctrl_host[kNf];
      g->hint_mf = g->ctrl_host[kMf];
    }
  }
  const int r = apply_dispatch(g, from, to, dir, *sched, kernel_id, kernel_args, out_modified, flags, s);
  g->hint_vset = nullptr;
  g->hint_nf = -1;
  g->hint_mf = -1;
  return r;
}
