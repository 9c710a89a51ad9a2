"""k-partitioning and balanced k-partitioning (Section 6: Algorithm 1 with
every M_d replaced by J - M_d, fitness = cut edges, plus f_eq for the
balanced variant) on the GPU against the oracle, in every step form:

* one iteration checked element by element (colours, conflicts, equity,
  M~, loss, grad_S L and the W step) in the one-hot form (dense pair walk
  and, with mu = 0 on a sparse graph, the adjacency-list walk) and in the
  FP8 tensor-core and FP32 CUDA-core dense forms;
* consecutive iterations, each checked against an oracle step from the
  GPU's own weights;
* the best-so-far individual minimises cut (+ f_eq), re-verified by the
  oracle's counters; a planted balanced partition stops the run at once.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_02261_gb300 import inputs
from paper_1909_02261_gb300.tenscol import (TC_FORM_DENSE_FP32, TC_FORM_DENSE_FP8, TC_FORM_ONEHOT, TC_KPART,
                                            TC_KPART_BAL, TensCol, TensColError, params)

from helpers import check_iteration, oracle_params

pytestmark = pytest.mark.gpu
FORMS = [TC_FORM_ONEHOT, TC_FORM_DENSE_FP8, TC_FORM_DENSE_FP32]


def make_ctx(rp, ci, D, k, p, W, t):
    ctx = TensCol(0)
    ctx.tc_init_graph(len(rp) - 1, rp, ci)
    ctx.tc_init_population(1, D, k, p)
    ctx.tc_set_state(W, t)
    return ctx


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("problem", [TC_KPART, TC_KPART_BAL])
@pytest.mark.parametrize("n,p_edge,D,k,mu", [
    (125, 0.5, 20, 4, 1e-4), (97, 0.3, 7, 33, 1e-4), (300, 0.1, 9, 6, 0.0), (257, 0.9, 3, 12, 1e-4)])
def test_partition_one_step(form, problem, n, p_edge, D, k, mu):
    rp, ci = inputs.gnp(n, p_edge, seed=n + k)
    W = inputs.init_weights(D, n, k, 0.02, seed=5)
    p = params(problem, stop_on_legal=0, lambda_=1e-3, mu=mu, nu=1e-3 if problem == TC_KPART_BAL else 0.0,
               form=form)
    with make_ctx(rp, ci, D, k, p, W, 7) as ctx:
        check_iteration(ctx, rp, ci, p, 7)


@pytest.mark.parametrize("form", [TC_FORM_ONEHOT, TC_FORM_DENSE_FP8])
def test_partition_consecutive_iterations(form):
    n, D, k = 160, 12, 5
    rp, ci = inputs.gnp(n, 0.4, seed=3)
    W = inputs.init_weights(D, n, k, 0.01, seed=4)
    p = params(TC_KPART_BAL, stop_on_legal=0, lambda_=1e-3, mu=1e-4, nu=1e-3, nb_iter=3, rho=2.0, form=form)
    with make_ctx(rp, ci, D, k, p, W, 1) as ctx:
        for t in range(1, 8):  # crosses two smoothing steps
            check_iteration(ctx, rp, ci, p, t, want_G=(t % 3 == 1))


@pytest.mark.parametrize("problem", [TC_KPART, TC_KPART_BAL])
def test_best_so_far_minimises_cut(problem):
    n, D, k, iters = 200, 16, 4, 60
    rp, ci = inputs.gnp(n, 0.3, seed=8)
    W = inputs.init_weights(D, n, k, 0.01, seed=9)
    p = params(problem, stop_on_legal=0, form=TC_FORM_ONEHOT)
    n_edges = len(ci) // 2
    po = oracle_params(p)
    first = O.step(rp, ci, W, po, 0)
    with make_ctx(rp, ci, D, k, p, W, 0) as ctx:
        assert ctx.tc_step(iters) == iters
        best = ctx.tc_best()
    col = best["coloring"]
    cut = int(O.cut(rp, ci, col[None])[0])
    assert cut == n_edges - best["conflicts"]
    assert best["equity"] == O.check_equity(col, k)
    f_best = cut + (best["equity"] if problem == TC_KPART_BAL else 0)
    assert f_best <= first["f_min"]  # never worse than the first population's best
    assert 0 <= best["iteration"] < iters


def test_planted_balanced_partition_stops_at_once():
    """Four disjoint cliques of 25, k = 4: the hidden partition cuts nothing
    and is exactly balanced, so the balanced problem's f is 0 and the run
    stops before its first update."""
    groups, size = 4, 25
    edges = [(g * size + a, g * size + b) for g in range(groups) for a in range(size) for b in range(a + 1, size)]
    n = groups * size
    rp, ci = inputs.from_edges(n, edges)
    hidden = np.repeat(np.arange(groups), size).astype(np.int32)
    rng = np.random.default_rng(0)
    cols = np.stack([rng.integers(0, groups, n).astype(np.int32), hidden, hidden])
    W = inputs.one_hot_weights(cols, groups)
    p = params(TC_KPART_BAL, stop_on_legal=1)
    with make_ctx(rp, ci, 3, groups, p, W, 0) as ctx:
        assert ctx.tc_step(10) == 0
        best = ctx.tc_best()
        assert best["individual"] == 1 and best["iteration"] == 0
        assert best["conflicts"] == len(edges) and best["equity"] == 0  # every edge inside a group
        assert np.array_equal(best["coloring"], hidden)


def test_partition_rejected_where_undefined():
    rp, ci = inputs.gnp(50, 0.3, seed=1)
    with TensCol(0) as ctx:
        ctx.tc_init_graph(50, rp, ci)
        with pytest.raises(TensColError):
            ctx.tc_kdescent(1, 4, 6, 3, 10, params(TC_KPART))


def test_partition_at_workload_shape():
    """Balanced k-partitioning on the benchmark's graph shape (G(1000, 0.5),
    k = 90) in the one-hot form, one iteration compared in full."""
    rp, ci = inputs.gnp(1000, 0.5, seed=2)
    W = inputs.init_weights(40, 1000, 90, 0.01, seed=2)
    p = params(TC_KPART_BAL, stop_on_legal=0, lambda_=1e-4, mu=1e-5, nu=1e-4)
    with make_ctx(rp, ci, 40, 90, p, W, 321) as ctx:
        check_iteration(ctx, rp, ci, p, 321)
