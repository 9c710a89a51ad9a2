"""Parity of the dense forms of the step against the oracle: the tensor-core
form (A.S and S S^T as FP8 tcgen05 GEMMs) and the FP32 CUDA-core form (the
same GEMMs with FP32 FFMA).  Their M~ and gamma come straight from the GEMM
outputs, so exact equality with the oracle checks the GEMMs element by
element."""
import numpy as np
import pytest

from paper_1909_02261_gb300 import inputs
from paper_1909_02261_gb300.tenscol import (TC_ECP, TC_FORM_DENSE_FP32, TC_FORM_DENSE_FP8,
                                            TC_FORM_ONEHOT, TC_KCOL, TensCol, params)

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
