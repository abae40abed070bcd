"""CPU checks of the PageRankDelta flip bound used by the GPU parity tests.

The bound (tests/_prd_bound.py) says which differences between an FP32
PageRankDelta and the FP64 oracle a threshold decision taken the other way can
cause.  Here it must (a) explain an independent FP32 evaluation of Fig. 1 on
the CPU, and (b) flag mistakes planted into that evaluation's output: a rank
moved by 1e-3 where no flip can reach, and a frontier size off by more than the
flip-possible count."""
import numpy as np
import pytest

import graphgen as gg
from _prd_bound import FlipBound, prdelta_fp32


@pytest.mark.parametrize("scale,eps", [(12, 1e-2), (12, 1e-3), (13, 1e-7)])
def test_bound_explains_fp32_evaluation(scale, eps):
    hg = gg.rmat_graph(scale, seed=1)
    fb = FlipBound(hg, eps, 10)
    r32, fs32 = prdelta_fp32(hg, 0.85, eps, 10)
    assert fb.violations(r32, fs32, 1e-4) == ([], [])
    # the bound is not vacuous: most vertices keep the plain 1e-4 tolerance
    assert np.mean(fb.rank_dev <= 1e-4 * fb.rank) > 0.6
    assert max(fb.near_counts[:4]) < 0.01 * hg.n


def test_bound_flags_planted_mistakes():
    hg = gg.rmat_graph(12, seed=1)
    fb = FlipBound(hg, 1e-2, 10)
    r32, fs32 = prdelta_fp32(hg, 0.85, 1e-2, 10)
    v = int(np.argmin(fb.rank_dev / fb.rank))          # a vertex no flip reaches
    bad = r32.astype(np.float64).copy()
    bad[v] *= 1 + 1e-3
    assert fb.violations(bad, fs32, 1e-4)[0] == [v]
    r = 1 + int(np.argmin(fb.near_counts[:-1]))
    fbad = fs32.copy()
    fbad[r] += fb.near_counts[r - 1] + 1
    assert fb.violations(r32, fbad, 1e-4)[1] == [r]
    fbad = fs32.copy()
    fbad[0] -= 1                                        # round 1 is always the whole vertex set
    assert fb.violations(r32, fbad, 1e-4)[1] == [0]
