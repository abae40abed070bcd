"""Graph fixtures shared by the GPU parity tests (inputs only; no expected values)."""
import functools

import numpy as np

import graphgen as gg


@functools.lru_cache(maxsize=None)
def rmat(scale, weights=False, seed=1, edge_factor=16):
    return gg.rmat_graph(scale, edge_factor=edge_factor, seed=seed, weights=(1, 1000) if weights else None)


@functools.lru_cache(maxsize=None)
def grid(side, weights=False, seed=1, shortcut_frac=0.01):
    return gg.grid_graph(side, shortcut_frac=shortcut_frac, seed=seed, weights=(1, 100) if weights else None)


def _edges(n, pairs, weights=False, seed=3):
    return gg.from_edge_list(n, pairs, weights=(seed, 1, 50) if weights else None)


@functools.lru_cache(maxsize=None)
def adversarial(name, weights=False):
    """Small graphs with the degenerate shapes the method has."""
    if name == "single":
        return _edges(1, [], weights)
    if name == "isolated":            # no arcs at all, V not a multiple of 32
        return _edges(45, [], weights)
    if name == "star":                # hub degree above the block-cooperative threshold
        n = 3000
        return _edges(n, [(0, i) for i in range(1, n)], weights)
    if name == "path":                # diameter n-1
        n = 777
        return _edges(n, [(i, i + 1) for i in range(n - 1)], weights)
    if name == "components":          # several components + isolated vertices, V = 1000
        rng = np.random.default_rng(5)
        pairs = []
        for lo, hi in [(0, 200), (300, 520), (600, 610), (700, 999)]:
            e = rng.integers(lo, hi, (3 * (hi - lo), 2))
            pairs += [tuple(x) for x in e]
        return _edges(1000, pairs, weights)
    if name == "hub_tail":            # a 40k-degree hub at an odd id plus a sparse tail
        n = 41_003
        rng = np.random.default_rng(9)
        pairs = [(7, i) for i in range(n) if i != 7]
        pairs += [tuple(x) for x in rng.integers(0, n, (20_000, 2))]
        return _edges(n, pairs, weights)
    raise KeyError(name)


ADVERSARIAL = ["single", "isolated", "star", "path", "components", "hub_tail"]
