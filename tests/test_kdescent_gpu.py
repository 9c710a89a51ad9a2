"""k-descent (tc_kdescent): the GCP / ECP as k-COL problems for decreasing k.

Every reported colouring is re-verified by the oracle's checker; on a
planted graph with 6 hidden groups (chromatic number 6) the descent stops at
exactly 6, and the equitable variant returns an equitable legal colouring.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_02261_gb300 import inputs
from paper_1909_02261_gb300.tenscol import TC_ECP, TC_KCOL, TensCol, TensColError, params

pytestmark = pytest.mark.gpu


def ctx_for(rp, ci):
    c = TensCol(0)
    c.tc_init_graph(len(rp) - 1, rp, ci)
    return c


def test_kdescent_reaches_the_planted_chromatic_number():
    rp, ci, hidden = inputs.planted_partition(125, 6, 0.5, seed=4)
    u, v = inputs.edge_list(rp, ci)
    with ctx_for(rp, ci) as c:
        k_best, col, iters = c.tc_kdescent(seed=11, D=20, k_start=9, k_min=2, max_iters=4000,
                                           p=params(TC_KCOL))
        assert k_best == 6
        assert col.min() >= 0 and col.max() < 6 and O.check_conflicts(u, v, col) == 0
        assert iters > 0
        # the context holds the population of k = 5, which found no legal colouring
        assert c.k == 5 and c.tc_best()["conflicts"] > 0


def test_kdescent_equitable():
    rp, ci, _ = inputs.planted_partition(120, 6, 0.5, seed=5)  # groups of 20: equitable at k = 6
    u, v = inputs.edge_list(rp, ci)
    with ctx_for(rp, ci) as c:
        # equitable colourings need classes of n / k vertices, each inside one
        # hidden group of 20 at p = 0.5: k = 6 is the only feasible value here
        k_best, col, _ = c.tc_kdescent(seed=3, D=20, k_start=6, k_min=4, max_iters=4000, p=params(TC_ECP))
        assert k_best == 6
        assert O.check_conflicts(u, v, col) == 0 and O.check_equity(col, k_best) == 0


def test_kdescent_arguments():
    rp, ci = inputs.gnp(30, 0.5, seed=1)
    with ctx_for(rp, ci) as c:
        for bad in [(0, 5, 2, 10), (4, 2, 3, 10), (4, 5, 0, 10), (4, 5, 2, 0)]:
            with pytest.raises(TensColError):
                c.tc_kdescent(1, *bad)
    empty = TensCol(0)
    with pytest.raises(TensColError):
        empty.tc_kdescent(1, 4, 5, 2, 10)
    empty.close()
