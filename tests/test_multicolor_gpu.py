"""Multicolouring (Section 6: vertex i takes its c_i largest-weight colours)
on the GPU against the oracle, in the two dense forms (FP8 tensor cores and
FP32 CUDA cores), whose GEMMs compute A.S and S S^T of the multi-hot S:

* one iteration element by element: the colour sets of Step 1, the shared-
  colour conflicts per vertex and per individual, M~ (diagonal D c_i), the
  loss terms, grad_S L and the W step, then the next colour sets;
* consecutive iterations, each checked against an oracle step from the
  GPU's own weights;
* the best-so-far multicolouring re-verified edge by edge; unit demands give
  back the one-colour step; invalid demands and forms are refused.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_02261_gb300 import inputs
from paper_1909_02261_gb300.tenscol import (TC_ECP, TC_FORM_DENSE_FP32, TC_FORM_DENSE_FP8, TC_FORM_ONEHOT, TC_KCOL,
                                            TensCol, TensColError, params)

from helpers import W_RTOL, check_iteration, g_rel_error, oracle_params, w_step_rel_error

pytestmark = pytest.mark.gpu
FORMS = [TC_FORM_DENSE_FP8, TC_FORM_DENSE_FP32]


def make_ctx(rp, ci, D, k, p, W, t, demand):
    ctx = TensCol(0)
    ctx.tc_init_graph(len(rp) - 1, rp, ci)
    ctx.tc_init_population(1, D, k, p)
    ctx.tc_set_demands(demand)
    ctx.tc_set_state(W, t)
    return ctx


def sets_of(S):
    """Oracle S (D x n x k 0/1) as -1 padded increasing colour lists."""
    D, n, k = S.shape
    cmax = int(S.sum(axis=2).max())
    out = -np.ones((D, n, cmax), np.int32)
    for d in range(D):
        for i in range(n):
            js = np.nonzero(S[d, i])[0]
            out[d, i, :len(js)] = js
    return out


def check_multi_iteration(ctx, rp, ci, p, t, demand, want_G=True):
    W0, t0 = ctx.tc_get_state()
    assert t0 == t
    po = oracle_params(p)
    ev = ctx.tc_evaluate(want_G=want_G)
    ref = O.step_multi(rp, ci, W0, demand, po, t)
    S = ref["S"]
    got = ctx.tc_get_multicolors()
    assert np.array_equal(got, sets_of(S)[:, :, :got.shape[2]])
    A = inputs.dense(rp, ci).astype(np.float64)
    gam = np.einsum("dij,dij->di", S, np.einsum("im,dmj->dij", A, S)).astype(np.int64)
    assert np.array_equal(ev["gamma_own"], gam)
    assert np.array_equal(ev["f_color"], ref["f_color"])
    assert np.array_equal(ev["Mt"], ref["Mt"])
    L, kap, var, fsum = [float(x) for x in ev["loss"]]
    assert fsum == float(ref["f_color"].sum())
    assert kap == pytest.approx(ref["kappa"], rel=1e-5)
    assert var == pytest.approx(ref["varpi"], rel=1e-5, abs=1e-30)
    scale = abs(ref["f_color"].sum()) + po.lambda_ * t * abs(ref["kappa"]) + po.mu * t * abs(ref["varpi"])
    assert abs(L - ref["loss"]) <= 1e-5 * max(scale, 1.0)
    if want_G:
        assert g_rel_error(ev["G"], ref["G"]) <= W_RTOL
    assert ctx.tc_step(1) == 1
    W1, t1 = ctx.tc_get_state()
    assert t1 == t + 1
    assert w_step_rel_error(W1, ref, po, t) <= W_RTOL
    # Step 1 of the next iteration on the stepped weights
    assert np.array_equal(ctx.tc_get_multicolors(), sets_of(O.assign_multi(W1, demand))[:, :, :got.shape[2]])


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("n,p_edge,D,k,cmax", [(120, 0.3, 9, 16, 3), (300, 0.1, 5, 24, 4), (65, 0.6, 12, 40, 8)])
def test_multicolor_one_step(form, n, p_edge, D, k, cmax):
    rp, ci = inputs.gnp(n, p_edge, seed=n + k)
    W = inputs.init_weights(D, n, k, 0.02, seed=3)
    demand = np.random.default_rng(n).integers(1, cmax + 1, n).astype(np.int32)
    p = params(TC_KCOL, stop_on_legal=0, lambda_=1e-3, mu=1e-4, form=form)
    with make_ctx(rp, ci, D, k, p, W, 5, demand) as ctx:
        check_multi_iteration(ctx, rp, ci, p, 5, demand)


def test_multicolor_consecutive_iterations():
    n, D, k = 150, 10, 20
    rp, ci = inputs.gnp(n, 0.25, seed=11)
    W = inputs.init_weights(D, n, k, 0.01, seed=12)
    demand = np.random.default_rng(1).integers(1, 4, n).astype(np.int32)
    p = params(TC_KCOL, stop_on_legal=0, lambda_=1e-3, mu=1e-4, nb_iter=3, rho=2.0, form=TC_FORM_DENSE_FP8)
    with make_ctx(rp, ci, D, k, p, W, 1, demand) as ctx:
        for t in range(1, 7):
            check_multi_iteration(ctx, rp, ci, p, t, demand, want_G=(t % 3 == 1))


def test_unit_demands_are_the_one_colour_step():
    n, D, k = 100, 8, 12
    rp, ci = inputs.gnp(n, 0.4, seed=2)
    W = inputs.init_weights(D, n, k, 0.02, seed=2)
    p = params(TC_KCOL, stop_on_legal=0, lambda_=1e-3, mu=1e-4, form=TC_FORM_DENSE_FP8)
    with make_ctx(rp, ci, D, k, p, W, 3, np.full(n, 2, np.int32)) as ctx:
        ctx.tc_set_demands(np.ones(n, np.int32))  # back to one colour per vertex
        check_iteration(ctx, rp, ci, p, 3)
        with pytest.raises(TensColError):
            ctx.tc_best_multi()


def test_multicolor_best_so_far():
    n, D, k, iters = 120, 16, 12, 50
    rp, ci = inputs.gnp(n, 0.15, seed=5)
    W = inputs.init_weights(D, n, k, 0.01, seed=6)
    demand = np.random.default_rng(7).integers(1, 4, n).astype(np.int32)
    p = params(TC_KCOL, stop_on_legal=1, form=TC_FORM_DENSE_FP8)
    first = O.step_multi(rp, ci, W, demand, oracle_params(p), 0)
    with make_ctx(rp, ci, D, k, p, W, 0, demand) as ctx:
        ctx.tc_step(iters)
        best = ctx.tc_best_multi()
    sets = best["colors"]
    for i in range(n):
        mine = sets[i][sets[i] >= 0]
        assert len(mine) == demand[i] == len(set(mine.tolist())) and mine.max() < k
    u, v = inputs.edge_list(rp, ci)
    shared = sum(len(set(sets[a][sets[a] >= 0]) & set(sets[b][sets[b] >= 0])) for a, b in zip(u, v))
    assert best["conflicts"] == shared
    assert best["conflicts"] <= first["f_min"]


def test_multicolor_refusals():
    n, D, k = 40, 3, 6
    rp, ci = inputs.gnp(n, 0.3, seed=1)
    W = inputs.init_weights(D, n, k, 0.02, seed=1)
    with TensCol(0) as ctx:
        ctx.tc_init_graph(n, rp, ci)
        ctx.tc_init_population(1, D, k, params(TC_KCOL, form=TC_FORM_ONEHOT))
        with pytest.raises(TensColError):
            ctx.tc_set_demands(np.full(n, 2, np.int32))  # the one-hot form has one colour per vertex
        ctx.tc_init_population(1, D, k, params(TC_KCOL, form=TC_FORM_DENSE_FP8))
        for bad in (np.zeros(n, np.int32), np.full(n, 7, np.int32), np.full(n - 1, 2, np.int32)):
            with pytest.raises(TensColError):
                ctx.tc_set_demands(bad)
        ctx.tc_set_demands(np.full(n, 2, np.int32))
        for q in (params(TC_KCOL, form=TC_FORM_ONEHOT), params(TC_ECP, form=TC_FORM_DENSE_FP8)):
            with pytest.raises(TensColError):
                ctx.tc_set_params(q)
        ctx.tc_set_state(W, 0)
        ctx.tc_step(2)  # still runs as a multicolouring
        assert ctx.tc_get_multicolors().shape == (D, n, 2)


def test_multicolor_at_workload_shape():
    """Multicolouring on the benchmark's graph shape (G(1000, 0.5), k = 90)
    with demands 1..3, FP8 tensor-core form, one iteration compared in full."""
    n, D, k = 1000, 24, 90
    rp, ci = inputs.gnp(n, 0.5, seed=2)
    W = inputs.init_weights(D, n, k, 0.01, seed=2)
    demand = np.random.default_rng(2).integers(1, 4, n).astype(np.int32)
    p = params(TC_KCOL, stop_on_legal=0, lambda_=1e-4, mu=1e-5, form=TC_FORM_DENSE_FP8)
    with make_ctx(rp, ci, D, k, p, W, 321, demand) as ctx:
        check_multi_iteration(ctx, rp, ci, p, 321, demand)
