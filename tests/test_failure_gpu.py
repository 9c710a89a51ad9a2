"""Failure handling on the GPU, made on the host or through the library's
own bounded waits and index checks (nothing here faults, traps or hangs a
GPU): a device wait whose arrival is withheld runs out after the context's
wait limit and tc_step reports TC_ERR_TIMEOUT; injected copy and launch
failures return TC_ERR_INJECTED; the index checks of libtenscol_bounds.so
catch a vertex index planted past n (it would land inside the shared-memory
panel, so even an unchecked read stays in bounds) and report
TC_ERR_DEVICE_BOUNDS.  After each failure the context is re-initialised and
one iteration is checked against the oracle."""
import numpy as np
import pytest

from helpers import check_iteration
from paper_1909_02261_gb300 import inputs
from paper_1909_02261_gb300.tenscol import TC_KCOL, TensCol, TensColError, params

pytestmark = pytest.mark.gpu

N, D, K = 60, 6, 8


def fresh(ctx, rp, ci, p, W, t=4):
    ctx.tc_init_population(1, D, K, p)
    ctx.tc_set_state(W, t)


def graph():
    rp, ci = inputs.gnp(N, 0.5, seed=71)
    W = inputs.init_weights(D, N, K, 0.01, seed=72)
    return rp, ci, W, params(TC_KCOL, stop_on_legal=0)


def test_withheld_device_wait_runs_out_and_the_context_recovers(monkeypatch):
    rp, ci, W, p = graph()
    with TensCol(0) as ctx:
        ctx.tc_init_graph(N, rp, ci)
        fresh(ctx, rp, ci, p, W)
        ctx.tc_set_wait_limit(20_000)  # 20 us
        monkeypatch.setenv("TC_FAULT", "wait")
        with pytest.raises(TensColError) as e:
            ctx.tc_step(1)
        assert e.value.code == -6  # TC_ERR_TIMEOUT
        monkeypatch.delenv("TC_FAULT")
        ctx.tc_set_wait_limit(0)
        fresh(ctx, rp, ci, p, W)
        check_iteration(ctx, rp, ci, p, 4)


def test_wait_limit_is_validated():
    with TensCol(0) as ctx:
        with pytest.raises(TensColError) as e:
            ctx.tc_set_wait_limit(-1)
        assert e.value.code == -1


def test_injected_copy_and_launch_failures(monkeypatch):
    rp, ci, W, p = graph()
    with TensCol(0) as ctx:
        ctx.tc_init_graph(N, rp, ci)
        fresh(ctx, rp, ci, p, W)
        W0, t0 = ctx.tc_get_state()
        monkeypatch.setenv("TC_FAULT", "copy")
        for call in (lambda: ctx.tc_get_state(), lambda: ctx.tc_set_state(W, 9)):
            with pytest.raises(TensColError) as e:
                call()
            assert e.value.code == -10  # TC_ERR_INJECTED
        monkeypatch.setenv("TC_FAULT", "launch")
        for call in (lambda: ctx.tc_step(1), lambda: ctx.tc_step_async(1)):
            with pytest.raises(TensColError) as e:
                call()
            assert e.value.code == -10
        monkeypatch.delenv("TC_FAULT")
        W1, t1 = ctx.tc_get_state()  # nothing changed: the failed calls stopped before any work
        assert t1 == t0 and np.array_equal(W1, W0)
        check_iteration(ctx, rp, ci, p, t0)


def test_device_index_checks_catch_a_planted_index(monkeypatch):
    rp, ci, W, p = graph()
    with TensCol(0, bounds=True) as ctx:
        ctx.tc_init_graph(N, rp, ci)
        fresh(ctx, rp, ci, p, W)
        check_iteration(ctx, rp, ci, p, 4)  # the checked build computes the same step
        monkeypatch.setenv("TC_FAULT", "index")
        with pytest.raises(TensColError) as e:
            ctx.tc_step(1)
        assert e.value.code == -7  # TC_ERR_DEVICE_BOUNDS
        monkeypatch.delenv("TC_FAULT")
        fresh(ctx, rp, ci, p, W)
        check_iteration(ctx, rp, ci, p, 4)
