"""The iteration trace (tc_set_trace / tc_get_trace): the per-iteration
population minimum, its individual, f_color, additive term and the loss
terms of eq. 5-7 that the paper follows over a run (Section 4.3), recorded on
the device.  Every record equals what tc_evaluate reports for the same
iteration of a second context stepped one iteration at a time (the same
kernels, so bit for bit); the ring keeps the newest records; graph replay
records the same values."""
import numpy as np
import pytest

from paper_1909_02261_gb300 import inputs
from paper_1909_02261_gb300.tenscol import TC_ECP, TC_KCOL, TensCol, TensColError, params

pytestmark = pytest.mark.gpu


def make_ctx(rp, ci, D, k, p, W, t):
    ctx = TensCol(0)
    ctx.tc_init_graph(len(rp) - 1, rp, ci)
    ctx.tc_init_population(1, D, k, p)
    ctx.tc_set_state(W, t)
    return ctx


def expected(ctx, problem):
    ev = ctx.tc_evaluate(want_G=False, want_M=False)
    f = ev["f_color"].astype(np.int64) + (ev["f_eq"] if problem == TC_ECP else 0)
    d = int(np.argmin(f))
    return dict(f_min=int(f[d]), individual=d, f_color=int(ev["f_color"][d]), f_add=int(ev["f_eq"][d]),
                loss=float(ev["loss"][0]), kappa=float(ev["loss"][1]), varpi=float(ev["loss"][2]))


@pytest.mark.parametrize("problem,every,cap,iters", [(TC_KCOL, 1, 64, 12), (TC_ECP, 3, 64, 13), (TC_KCOL, 1, 4, 12)])
def test_trace_matches_evaluate(problem, every, cap, iters):
    n, D, k, t0 = 150, 12, 9, 5
    rp, ci = inputs.gnp(n, 0.4, seed=3)
    W = inputs.init_weights(D, n, k, 0.01, seed=4)
    p = params(problem, stop_on_legal=0, lambda_=1e-3, mu=0.0 if problem == TC_ECP else 1e-4, nu=1e-3)
    with make_ctx(rp, ci, D, k, p, W, t0) as a, make_ctx(rp, ci, D, k, p, W, t0) as b:
        a.tc_set_trace(cap, every)
        assert a.tc_step(iters) == iters
        want = []
        for t in range(t0, t0 + iters):
            if t % every == 0:
                want.append(dict(t=t, **expected(b, problem)))
            assert b.tc_step(1) == 1
        got = a.tc_get_trace()
        assert got == want[-cap:]  # the ring keeps the newest records, oldest first
        a.tc_set_trace(0)
        assert a.tc_get_trace() == []


def test_trace_through_graph_replay():
    n, D, k = 120, 8, 7
    rp, ci = inputs.gnp(n, 0.5, seed=5)
    W = inputs.init_weights(D, n, k, 0.01, seed=6)
    p = params(TC_KCOL, stop_on_legal=0)
    with make_ctx(rp, ci, D, k, p, W, 0) as a, make_ctx(rp, ci, D, k, p, W, 0) as b:
        a.tc_set_trace(32)
        b.tc_set_trace(32)
        a.tc_set_graph_chunk(4)
        a.tc_step(10)  # two graph replays and two direct launches
        b.tc_step(10)
        ta, tb = a.tc_get_trace(), b.tc_get_trace()
        assert len(ta) == 10 and ta == tb


def test_trace_arguments():
    rp, ci = inputs.gnp(40, 0.3, seed=1)
    with TensCol(0) as ctx:
        ctx.tc_init_graph(40, rp, ci)
        with pytest.raises(TensColError):
            ctx.tc_set_trace(8)  # no population yet
        ctx.tc_init_population(1, 3, 5, params(TC_KCOL))
        for cap, every in ((-1, 1), (8, 0)):
            with pytest.raises(TensColError):
                ctx.tc_set_trace(cap, every)
        assert ctx.tc_get_trace() == []
