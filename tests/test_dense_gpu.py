"""Parity of the dense forms of the step against the oracle: the tensor-core
form (A.S and S S^T as FP8 tcgen05 GEMMs) and the FP32 CUDA-core form (the
same GEMMs with FP32 FFMA).  Their M~ and gamma come straight from the GEMM
outputs, so exact equality with the oracle checks the GEMMs element by
element."""
import numpy as np
import pytest

from paper_1909_02261_gb300 import inputs
from paper_1909_02261_gb300.tenscol import (TC_ECP, TC_FORM_DENSE_FP32, TC_FORM_DENSE_FP8,
                                            TC_FORM_ONEHOT, TC_KCOL, TensCol, TensColError, params)

from helpers import check_iteration

pytestmark = pytest.mark.gpu
FORMS = [TC_FORM_DENSE_FP8, TC_FORM_DENSE_FP32]


def make_ctx(rp, ci, D, k, p, W, t):
    ctx = TensCol(0)
    ctx.tc_init_graph(len(rp) - 1, rp, ci)
    ctx.tc_init_population(1, D, k, p)
    ctx.tc_set_state(W, t)
    return ctx


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("n,p_edge,D,k", [
    (125, 0.5, 20, 18), (97, 0.3, 7, 33), (1, 0.0, 1, 1), (300, 0.5, 9, 40), (257, 0.9, 3, 300),
    (40, 1.0, 2, 40)])
def test_dense_form_one_step(form, n, p_edge, D, k):
    rp, ci = inputs.gnp(n, p_edge, seed=n + k)
    W = inputs.init_weights(D, n, k, 0.02, seed=5)
    p = params(TC_KCOL, stop_on_legal=0, lambda_=1e-3, mu=1e-4, form=form)
    with make_ctx(rp, ci, D, k, p, W, 7) as ctx:
        check_iteration(ctx, rp, ci, p, 7)


@pytest.mark.parametrize("form", FORMS)
def test_dense_form_ecp(form):
    rp, ci = inputs.gnp(150, 0.1, seed=3)
    W = inputs.init_weights(12, 150, 10, 0.01, seed=3)
    p = params(TC_ECP, stop_on_legal=0, nu=1e-2, form=form)
    with make_ctx(rp, ci, 12, 10, p, W, 5) as ctx:
        check_iteration(ctx, rp, ci, p, 5)


@pytest.mark.parametrize("form", FORMS)
def test_dense_form_trajectory(form):
    rp, ci = inputs.gnp(125, 0.5, seed=1)
    W = inputs.init_weights(20, 125, 18, 0.01, seed=1)
    p = params(TC_KCOL, stop_on_legal=0, form=form)
    with make_ctx(rp, ci, 20, 18, p, W, 0) as ctx:
        for t in range(8):
            check_iteration(ctx, rp, ci, p, t, want_G=(t % 4 == 0))


def test_full_size_tensor_core_form():
    rp, ci = inputs.gnp(1000, 0.5, seed=2)
    W = inputs.init_weights(200, 1000, 90, 0.01, seed=2)
    p = params(TC_KCOL, stop_on_legal=0, form=TC_FORM_DENSE_FP8)
    with make_ctx(rp, ci, 200, 90, p, W, 1234) as ctx:
        check_iteration(ctx, rp, ci, p, 1234, want_G=True)


def test_forms_agree_over_many_steps():
    """Integer outputs identical across forms over a run; weights within the
    FP32 rounding of different summation orders."""
    rp, ci = inputs.gnp(200, 0.5, seed=9)
    W = inputs.init_weights(16, 200, 24, 0.01, seed=9)
    outs = {}
    for form in (TC_FORM_ONEHOT, TC_FORM_DENSE_FP8, TC_FORM_DENSE_FP32):
        p = params(TC_KCOL, stop_on_legal=0, form=form)
        with make_ctx(rp, ci, 16, 24, p, W, 0) as ctx:
            ctx.tc_step(1)
            ev = ctx.tc_evaluate(want_G=False)
            outs[form] = (ev, ctx.tc_get_state()[0])
    e0, w0 = outs[TC_FORM_ONEHOT]
    for form in FORMS:
        e, w = outs[form]
        for key in ("colors", "gamma_own", "f_color", "f_eq", "Mt"):
            assert np.array_equal(e[key], e0[key]), key
        assert np.allclose(w, w0, rtol=1e-5, atol=1e-9)


def test_switch_form_on_live_population():
    rp, ci = inputs.gnp(90, 0.5, seed=4)
    W = inputs.init_weights(6, 90, 12, 0.01, seed=4)
    p = params(TC_KCOL, stop_on_legal=0)
    with make_ctx(rp, ci, 6, 12, p, W, 3) as ctx:
        ctx.tc_step(2)
        for form in (TC_FORM_DENSE_FP8, TC_FORM_DENSE_FP32, TC_FORM_ONEHOT):
            p.form = form
            ctx.tc_set_params(p)
            _, t = ctx.tc_get_state()
            check_iteration(ctx, rp, ci, p, t)


# (Gamma unit rows, column tile, cluster), (M~ unit rows, column tile,
# cluster), M~ K splits[, one launch for both]; 256-row units run on a CTA
# pair (cta_group::2)
PLANS = [
    ((128, 256, 1), (128, 256, 1), 1), ((128, 256, 2), (128, 256, 2), 3), ((128, 256, 4), (128, 256, 1), 4),
    ((128, 128, 1), (128, 128, 1), 1), ((128, 128, 2), (128, 128, 1), 4), ((128, 128, 4), (128, 256, 2), 2),
    ((256, 256, 2), (256, 256, 2), 3), ((256, 128, 2), (256, 128, 2), 4), ((256, 256, 2), (128, 256, 2), 1),
    ((128, 256, 1), (256, 256, 2), 2), ((128, 256, 1), (128, 256, 1), 3, True),
    ((128, 256, 2), (128, 256, 2), 2, True), ((128, 128, 1), (128, 128, 1), 4, True),
    ((256, 256, 2), (256, 256, 2), 3, True), ((256, 128, 2), (256, 128, 2), 2, True)]


def plan_of(got):
    return ((got["gamma_tile_m"], got["gamma_tile_n"], got["gamma_cluster"]),
            (got["mtilde_tile_m"], got["mtilde_tile_n"], got["mtilde_cluster"]), got["mtilde_splits"],
            got["fused"])


def full(plan):
    return plan if len(plan) == 4 else (*plan, False)


@pytest.mark.parametrize("plan", PLANS)
def test_every_tensor_core_plan_is_exact(plan):
    """Each tile / cluster / split-K variant the autotuner may pick, pinned,
    on a graph spanning several row tiles (n_pad = 768: 6 of 128, 3 of 256)
    and column tiles, against the oracle element by element."""
    n, D, k = 700, 11, 37
    rp, ci = inputs.gnp(n, 0.5, seed=21)
    W = inputs.init_weights(D, n, k, 0.02, seed=22)
    p = params(TC_KCOL, stop_on_legal=0, lambda_=1e-3, mu=1e-4, form=TC_FORM_DENSE_FP8)
    with make_ctx(rp, ci, D, k, p, W, 7) as ctx:
        if plan[0][2] == 4:  # clusters of 4 need the 128-row tiles to come in fours
            with pytest.raises(TensColError):
                ctx.tc_dense_set_plan(*plan)
            return
        ctx.tc_dense_set_plan(*plan)
        assert plan_of(ctx.tc_dense_plan()) == full(plan)
        check_iteration(ctx, rp, ci, p, 7)


@pytest.mark.parametrize("plan", [((128, 256, 4), (128, 256, 2), 5), ((128, 128, 4), (128, 128, 1), 9),
                                  ((256, 256, 2), (256, 256, 2), 10), ((256, 128, 2), (256, 256, 2), 7),
                                  ((128, 256, 2), (128, 256, 2), 7, True), ((128, 256, 1), (128, 256, 1), 10, True),
                                  ((256, 256, 2), (256, 256, 2), 8, True)])
def test_workload_sized_plans_are_exact(plan):
    n, D, k = 1000, 30, 41  # n_pad = 1024: 8 row tiles of 128; D k = 1230: 10 K blocks
    rp, ci = inputs.gnp(n, 0.5, seed=23)
    W = inputs.init_weights(D, n, k, 0.02, seed=24)
    p = params(TC_KCOL, stop_on_legal=0, lambda_=1e-3, mu=1e-4, form=TC_FORM_DENSE_FP8)
    with make_ctx(rp, ci, D, k, p, W, 7) as ctx:
        ctx.tc_dense_set_plan(*plan)
        check_iteration(ctx, rp, ci, p, 7)


def test_autotuner_times_candidates_and_rejects_bad_plans():
    rp, ci = inputs.gnp(300, 0.5, seed=25)
    W = inputs.init_weights(5, 300, 20, 0.02, seed=26)
    with make_ctx(rp, ci, 5, 20, params(TC_KCOL, form=TC_FORM_DENSE_FP8), W, 0) as ctx:
        got = ctx.tc_dense_plan()
        assert got["candidates"] >= 4 and got["gamma_us"] > 0 and got["mtilde_us"] > 0
        for bad in [((128, 64, 1), (128, 256, 1), 1), ((128, 256, 3), (128, 256, 1), 1),
                    ((128, 128, 1), (128, 128, 2), 1), ((128, 256, 1), (128, 256, 1), 0),
                    ((256, 256, 1), (128, 256, 1), 1), ((128, 256, 1), (256, 256, 4), 1),
                    ((512, 256, 2), (128, 256, 1), 1), ((128, 256, 1), (128, 128, 1), 1, True),
                    ((256, 256, 2), (128, 256, 2), 1, True), ((128, 256, 4), (128, 256, 4), 1, True)]:
            with pytest.raises(TensColError):
                ctx.tc_dense_set_plan(*bad)
        assert ctx.tc_dense_plan() == got  # unchanged by the refused plans
    with make_ctx(rp, ci, 5, 20, params(TC_KCOL, form=TC_FORM_ONEHOT), W, 0) as ctx:
        with pytest.raises(TensColError):
            ctx.tc_dense_plan()


@pytest.mark.parametrize("form", FORMS)
def test_full_size_workload_one_step(form):
    """The benchmark workload G(1000, 0.5), k = 90, D = 200 in the dense forms,
    on the plan the autotuner picks (as the benchmark runs it), compared in
    full on one iteration: every Gamma-derived conflict count and every M~
    entry exactly, grad_S L and the W step within the step tolerance."""
    rp, ci = inputs.gnp(1000, 0.5, seed=2)
    W = inputs.init_weights(200, 1000, 90, 0.01, seed=2)
    p = params(TC_KCOL, stop_on_legal=0, form=form)
    with make_ctx(rp, ci, 200, 90, p, W, 777) as ctx:
        check_iteration(ctx, rp, ci, p, 777, want_G=True)
