"""Host side of the learned selector that needs no GPU: the gate the library
applies before the network (frontiers with |F| + m_f < m / SELECTOR_GATE are
pushed without an evaluation), decoded from the raw features as the training
and replay scripts see them, and the committed weights' shapes."""
import numpy as np

import oracle
from paper_1805_00923_gb300 import selector as sel


def _frontier_rows(rng, m, n, count, spread):
    rows, want = [], []
    for _ in range(count):
        # |F| + m_f drawn around the gate's threshold m / SELECTOR_GATE
        total = max(0, int(m / sel.SELECTOR_GATE * rng.uniform(1 - spread, 1 + spread)))
        nf = int(rng.integers(0, min(total, n) + 1))
        mf = total - nf
        if mf > m:
            continue
        if abs((nf + mf) * sel.SELECTOR_GATE - m) <= 0.01 * m:
            continue  # float32 features do not resolve counts this close to the threshold
        # the unvisited counts vary on their own, so that no other feature can stand in for m
        nu = int(rng.integers(0, n - nf + 1))
        mu = int(rng.integers(0, m - mf + 1))
        rows.append(oracle.features(n=n, m=m, maxdeg=max(1, m // 8), nf=nf, mf=mf, nu=nu, mu=mu,
                                    level=2, was_pull=0, nf_prev=nf))
        want.append((nf + mf) * sel.SELECTOR_GATE < m)
    return np.asarray(rows), np.asarray(want)


def test_gate_decodes_the_frontier_counts():
    rng = np.random.default_rng(11)
    for m, n in ((4_000, 1_000), (2_000_000, 65_536), (128_310_386, 4_194_304), (520_765_678, 16_777_216)):
        X, want = _frontier_rows(rng, m, n, 200, 0.9)
        assert want.any() and not want.all()
        assert np.array_equal(sel.gated(X), want)
        # the features as the library stores them (float32)
        assert np.array_equal(sel.gated(X.astype(np.float32)), want)


def test_gate_on_empty_and_whole_frontiers():
    m, n = 520_765_678, 16_777_216
    empty = oracle.features(n=n, m=m, maxdeg=1000, nf=0, mf=0, nu=n, mu=m, level=0, was_pull=0, nf_prev=0)
    whole = oracle.features(n=n, m=m, maxdeg=1000, nf=n, mf=m, nu=0, mu=0, level=1, was_pull=1, nf_prev=1)
    assert sel.gated(np.asarray([empty, whole])).tolist() == [True, False]


def test_committed_weights_fit_the_network():
    params, mean, inv_std = sel.load()
    assert params.dtype == np.float32 and params.shape == (oracle.mlp_num_params(),)
    assert mean.shape == (16,) and inv_std.shape == (16,)
    assert np.all(np.isfinite(params)) and np.all(np.isfinite(mean)) and np.all(inv_std > 0)
