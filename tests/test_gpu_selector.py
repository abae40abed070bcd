"""The learned selector: GPU training kernels vs the FP64 oracle, fused
inference consistency, bit-exact results under the learned schedule, and the
gain over Beamer's rule measured on recorded per-level timings."""
import os

import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
from _graphs import grid, rmat

pytestmark = pytest.mark.gpu


def _data(seed, B=777):
    rng = np.random.default_rng(seed)
    p = (rng.normal(0, 0.3, oracle.mlp_num_params())).astype(np.float32)
    X = rng.normal(size=(B, 16)).astype(np.float32)
    T = rng.normal(size=(B, 3)).astype(np.float32)
    M = (rng.random((B, 3)) < 0.7).astype(np.float32)
    return p, X, T, M


def _cuda(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def test_mlp_forward_matches_oracle(gi):
    from paper_1805_00923_gb300 import selector as sel
    p, X, _, _ = _data(1)
    Y = sel.forward(*_cuda(p, X)).cpu().numpy()
    want = oracle.mlp_forward(p.astype(np.float64), X.astype(np.float64))
    assert np.allclose(Y, want, rtol=1e-4, atol=1e-4)


@pytest.mark.parametrize("seed", [2, 3])
def test_mlp_gradient_matches_oracle(gi, seed):
    from paper_1805_00923_gb300 import selector as sel
    p, X, T, M = _data(seed)
    loss, grad = sel.loss_grad(*_cuda(p, X, T, M))
    want_loss, want = oracle.mlp_loss_grad(p.astype(np.float64), X.astype(np.float64), T.astype(np.float64),
                                           M.astype(np.float64))
    grad = grad.cpu().numpy().astype(np.float64)
    assert abs(float(loss[0]) - want_loss) <= 1e-4 * abs(want_loss)
    scale = np.abs(want).max()
    assert np.all(np.abs(grad - want) <= 1e-3 * np.abs(want) + 1e-5 * scale)
    assert np.linalg.norm(grad - want) <= 1e-4 * np.linalg.norm(want)


def test_adam_matches_oracle(gi):
    from paper_1805_00923_gb300 import selector as sel
    rng = np.random.default_rng(4)
    n = oracle.mlp_num_params()
    p = rng.normal(size=n).astype(np.float32)
    g = rng.normal(size=n).astype(np.float32)
    m = (rng.normal(size=n) * 0.1).astype(np.float32)
    v = (rng.random(n) * 0.1).astype(np.float32)
    pt, gt, mt, vt = _cuda(p, g, m, v)
    sel.adam(pt, gt, mt, vt, 3, lr=0.01)
    p64, m64, v64 = p.astype(np.float64), m.astype(np.float64), v.astype(np.float64)
    oracle.adam_step(p64, g.astype(np.float64), m64, v64, 3, lr=0.01)
    assert np.allclose(pt.cpu().numpy(), p64, rtol=1e-5, atol=1e-6)
    assert np.allclose(mt.cpu().numpy(), m64, rtol=1e-5, atol=1e-7)
    assert np.allclose(vt.cpu().numpy(), v64, rtol=1e-5, atol=1e-8)


def test_training_fits_a_known_function(gi):
    from paper_1805_00923_gb300 import selector as sel
    rng = np.random.default_rng(5)
    X = rng.normal(size=(4096, 16)).astype(np.float32)
    T = np.stack([X[:, 0] + 0.5 * X[:, 1], np.abs(X[:, 2]), X[:, 3] * X[:, 4] * 0.3], 1).astype(np.float32)
    params, mean, inv_std, losses = sel.train(X, T, steps=1500, lr=3e-3)
    assert losses[-1] < 0.1 * losses[0]


def _profile_many(gi, sel, hg, kernel, sources):
    g = gi.Graph.from_host(hg)
    feats, times = [], []
    for s in sources:
        f, t = sel.profile(g, kernel, int(s))
        feats.append(f)
        times.append(t)
    return g, feats, times


def test_profile_levels_match_oracle(gi):
    from paper_1805_00923_gb300 import selector as sel
    hg = rmat(14)
    g = gi.Graph.from_host(hg)
    f, t = sel.profile(g, gi.GI_K_BFS, 0)
    _, _, levels = oracle.bfs(hg, 0)
    assert f.shape[0] == len(levels) and (t > 0).all()
    assert np.allclose(np.exp2(f[:, 0]) - 1, levels, rtol=1e-5)   # feature 0 = log2(1+|F|)


WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1805_00923_gb300",
                       "selector_weights.npz")


@pytest.mark.skipif(not os.path.exists(WEIGHTS), reason="no trained selector weights committed")
def test_learned_schedule_bit_exact_and_fused_inference(gi):
    from paper_1805_00923_gb300 import selector as sel
    params, mean, inv_std = sel.install(WEIGHTS)
    for hg in [rmat(16), grid(64)]:
        g = gi.Graph.from_host(hg)
        for src in [0, int(gg.pick_sources(hg, 1, seed=3)[0])]:
            want_d, want_p, levels = oracle.bfs(hg, src)
            tr = gi.Trace(4096)
            d, p = gi.bfs(g, src, sched=gi.schedule("learned"), trace=tr)
            assert np.array_equal(d.cpu().numpy(), want_d) and np.array_equal(p.cpu().numpy(), want_p)
            t = tr.as_dict()
            # the fused kernel's choice equals the batched forward kernel's argmin
            # on the same features, wherever the margin exceeds float noise, and
            # SparsePush where |F| + m_f < m / 200 (no evaluation there)
            f = t["features"]
            Xn = torch.from_numpy(((f - mean) * inv_std).astype(np.float32)).cuda()
            Y = sel.forward(torch.from_numpy(params).cuda(), Xn).cpu().numpy()
            srt = np.sort(Y, axis=1)
            nfmf = t["frontier"].astype(np.float64) + t["edges"].astype(np.float64)
            gate = nfmf * sel.SELECTOR_GATE < hg.m
            # the replay's gate from the (rounded) features agrees away from the boundary
            far = np.abs(nfmf * sel.SELECTOR_GATE / hg.m - 1.0) > 1e-3
            assert np.array_equal(gate[far], sel.gated(f)[far])
            assert (t["direction"][gate] == 0).all()
            clear = ((srt[:, 1] - srt[:, 0]) > 1e-3) & ~gate
            assert np.array_equal(t["direction"][clear], Y.argmin(1)[clear])


@pytest.mark.skipif(not os.path.exists(WEIGHTS), reason="no trained selector weights committed")
def test_learned_selector_gain_over_beamer(gi):
    """On held-out graphs, the levels the network picks cost less (in the recorded
    per-level timings of all three directions) than the levels Beamer's rule picks."""
    from paper_1805_00923_gb300 import selector as sel
    params, mean, inv_std = sel.load(WEIGHTS)
    tot = {"learned": 0.0, "beamer": 0.0, "best": 0.0}
    for hg, kern in [(gg.rmat_graph(19, seed=77), gi.GI_K_BFS), (gg.grid_graph(384, seed=77), gi.GI_K_BFS),
                     (gg.rmat_graph(17, seed=78, weights=(1, 1000)), gi.GI_K_SSSP)]:
        srcs = gg.pick_sources(hg, 3, seed=9)
        g, feats, times = _profile_many(gi, sel, hg, kern, srcs)
        for s, f, t in zip(srcs, feats, times):
            tr = gi.Trace(16384)
            if kern == gi.GI_K_BFS:
                gi.bfs(g, int(s), want_parent=False, sched=gi.schedule("hybrid_pull"), trace=tr)
            else:
                gi.sssp(g, int(s), sched=gi.schedule("hybrid_pull"), trace=tr)
            beamer = tr.as_dict()["direction"]
            assert len(beamer) == len(t)
            learned = sel.choose(params, mean, inv_std, f)
            idx = np.arange(len(t))
            tot["learned"] += float(t[idx, learned].sum())
            tot["beamer"] += float(t[idx, beamer].sum())
            tot["best"] += float(t.min(axis=1).sum())
    print("recorded level time (ms):", tot)
    assert tot["learned"] <= tot["beamer"]
