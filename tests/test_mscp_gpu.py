"""Minimum sum colouring (Section 6: the colour-cost fitness f_mscp in place of
f_eq) on the GPU against the oracle, in every step form:

* one iteration checked element by element (colours, conflicts, colour
  costs, M~, loss, grad_S L and the W step), with the default costs
  z_l = l + 1 and with costs set through tc_set_color_costs, in the one-hot
  form (dense pair walk, and the adjacency-list walk with mu = 0 on a sparse
  graph) and in the FP8 tensor-core and FP32 CUDA-core dense forms;
* the best-so-far individual minimises f_color + f_mscp, re-verified by the
  oracle's counters; bad costs are refused.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_02261_gb300 import inputs
from paper_1909_02261_gb300.tenscol import (TC_FORM_DENSE_FP32, TC_FORM_DENSE_FP8, TC_FORM_ONEHOT, TC_MSCP, TensCol,
                                            TensColError, params)

from helpers import check_iteration, oracle_params

pytestmark = pytest.mark.gpu
FORMS = [TC_FORM_ONEHOT, TC_FORM_DENSE_FP8, TC_FORM_DENSE_FP32]


def make_ctx(rp, ci, D, k, p, W, t, z=None):
    ctx = TensCol(0)
    ctx.tc_init_graph(len(rp) - 1, rp, ci)
    ctx.tc_init_population(1, D, k, p)
    if z is not None:
        ctx.tc_set_color_costs(z)
    ctx.tc_set_state(W, t)
    return ctx


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("costs", ["default", "set"])
@pytest.mark.parametrize("n,p_edge,D,k,mu", [(125, 0.5, 20, 18, 1e-4), (300, 0.1, 9, 6, 0.0), (97, 0.9, 5, 60, 1e-4)])
def test_mscp_one_step(form, costs, n, p_edge, D, k, mu):
    rp, ci = inputs.gnp(n, p_edge, seed=n + k)
    W = inputs.init_weights(D, n, k, 0.02, seed=7)
    z = None if costs == "default" else np.random.default_rng(k).integers(0, 50, k).astype(np.int32)
    p = params(TC_MSCP, stop_on_legal=0, lambda_=1e-3, mu=mu, nu=3e-3, form=form)
    with make_ctx(rp, ci, D, k, p, W, 9, z) as ctx:
        check_iteration(ctx, rp, ci, p, 9, zcost=z)


def test_mscp_best_so_far():
    n, D, k, iters = 150, 16, 8, 60
    rp, ci = inputs.gnp(n, 0.2, seed=4)
    W = inputs.init_weights(D, n, k, 0.01, seed=5)
    z = np.array([1, 1, 2, 3, 5, 8, 13, 21], np.int32)
    p = params(TC_MSCP, stop_on_legal=1)
    first = O.step(rp, ci, W, oracle_params(p, z), 0)
    with make_ctx(rp, ci, D, k, p, W, 0, z) as ctx:
        assert ctx.tc_step(iters) == iters  # costs are positive: f never reaches 0
        best = ctx.tc_best()
    col = best["coloring"]
    u, v = inputs.edge_list(rp, ci)
    assert best["conflicts"] == O.check_conflicts(u, v, col)
    assert best["equity"] == int(O.mscp(col[None], z)[0])
    assert best["conflicts"] + best["equity"] <= first["f_min"]


def test_color_costs_are_checked():
    rp, ci = inputs.gnp(40, 0.3, seed=1)
    with TensCol(0) as ctx:
        ctx.tc_init_graph(40, rp, ci)
        with pytest.raises(TensColError):
            ctx.tc_set_color_costs([1, 2, 3])  # no population yet
        ctx.tc_init_population(1, 3, 5, params(TC_MSCP))
        for bad in ([1, 2, 3], [1, 2, -3, 4, 5]):  # another k, a negative cost
            with pytest.raises(TensColError):
                ctx.tc_set_color_costs(bad)
        with pytest.raises(TensColError):
            ctx.tc_kdescent(1, 3, 5, 3, 10, params(TC_MSCP))


def test_mscp_at_workload_shape():
    """Minimum sum colouring on the benchmark's graph shape (G(1000, 0.5),
    k = 90), default costs, one-hot form, one iteration compared in full."""
    rp, ci = inputs.gnp(1000, 0.5, seed=2)
    W = inputs.init_weights(40, 1000, 90, 0.01, seed=2)
    p = params(TC_MSCP, stop_on_legal=0, lambda_=1e-4, mu=1e-5, nu=1e-5)
    with make_ctx(rp, ci, 40, 90, p, W, 321) as ctx:
        check_iteration(ctx, rp, ci, p, 321)
