"""Batches of uneven instances stepped by one CUDA-graph launch (tc_batch_*).

* A batch advances every member exactly as separate tc_step calls would:
  weights, iteration counters and best-so-far bit for bit, across graph
  replays and the directly launched remainder.
* One batched step of every instance of the batched workload (G(4000, 0.5)
  k = 290 D = 100 plus eight instances of n = 250 ... 2000, all in the FP8
  tensor-core form) matches the oracle's step: exact colours, conflicts and
  equity, W within the 1e-5 step tolerance.
* Members keep their own stop flags: a solved instance stops, the others go
  on.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_02261_gb300 import inputs
from paper_1909_02261_gb300.tenscol import (TC_ECP, TC_FORM_DENSE_FP8, TC_FORM_ONEHOT, TC_KCOL, TensCol,
                                            TensColBatch, TensColError, params)

from helpers import W_RTOL, oracle_params, w_step_rel_error

pytestmark = pytest.mark.gpu


def make(rp, ci, D, k, p, W, t, seed=1):
    c = TensCol(0)
    c.tc_init_graph(len(rp) - 1, rp, ci)
    c.tc_init_population(seed, D, k, p)
    c.tc_set_state(W, t)
    return c


SMALL = [  # n, p_edge, D, k, problem, form
    (60, 0.5, 7, 9, TC_KCOL, TC_FORM_ONEHOT),
    (130, 0.1, 12, 5, TC_ECP, TC_FORM_ONEHOT),
    (250, 0.9, 5, 70, TC_KCOL, TC_FORM_DENSE_FP8),
    (97, 0.3, 9, 33, TC_KCOL, TC_FORM_ONEHOT),
]


def small_instances():
    out = []
    for q, (n, pe, D, k, problem, form) in enumerate(SMALL):
        rp, ci = inputs.gnp(n, pe, seed=40 + q)
        W = inputs.init_weights(D, n, k, 0.05, seed=50 + q)
        p = params(problem, stop_on_legal=0, lambda_=1e-3, mu=0.0 if problem == TC_ECP else 1e-3, nu=1e-3,
                   form=form)
        out.append((rp, ci, D, k, p, W))
    return out


@pytest.mark.parametrize("n_iters,chunk", [(7, 3), (5, 0), (4, 4)])
def test_batch_equals_separate_steps(n_iters, chunk):
    insts = small_instances()
    alone = [make(rp, ci, D, k, p, W, 3) for rp, ci, D, k, p, W in insts]
    members = [make(rp, ci, D, k, p, W, 3) for rp, ci, D, k, p, W in insts]
    with TensColBatch(0) as b:
        for m in members:
            b.add(m)
        assert b.size() == len(insts)
        b.step(n_iters, chunk)
    for a, m in zip(alone, members):
        assert a.tc_step(n_iters) == n_iters
        Wa, ta = a.tc_get_state()
        Wm, tm = m.tc_get_state()
        assert ta == tm == 3 + n_iters
        assert np.array_equal(Wa, Wm)
        ba, bm = a.tc_best(), m.tc_best()
        assert np.array_equal(ba.pop("coloring"), bm.pop("coloring")) and ba == bm
    for c in alone + members:
        c.close()


def test_batch_replays_graph_and_recaptures_after_changes():
    insts = small_instances()[:2]
    members = [make(rp, ci, D, k, p, W, 0) for rp, ci, D, k, p, W in insts]
    alone = [make(rp, ci, D, k, p, W, 0) for rp, ci, D, k, p, W in insts]
    with TensColBatch(0) as b:
        for m in members:
            b.add(m)
        b.step(4, 2)
        b.step(4, 2)  # the same graph, replayed
        p2 = params(TC_KCOL, stop_on_legal=0, lambda_=5e-3, mu=2e-3)
        members[0].tc_set_params(p2)  # stale graph: captured again
        alone[0].tc_step(8)
        alone[0].tc_set_params(p2)
        alone[1].tc_step(8)
        b.step(3, 2)
    alone[0].tc_step(3)
    alone[1].tc_step(3)
    for a, m in zip(alone, members):
        assert np.array_equal(a.tc_get_state()[0], m.tc_get_state()[0])
    for c in alone + members:
        c.close()


def test_batch_members_stop_independently():
    rp, ci, hidden = inputs.planted_partition(200, 8, 0.5, seed=4)
    Wp = inputs.one_hot_weights(np.tile(hidden, (4, 1)), 8)  # every individual legal
    solved = make(rp, ci, 4, 8, params(TC_KCOL, stop_on_legal=1), Wp, 0)
    rp2, ci2 = inputs.gnp(150, 0.5, seed=9)
    W2 = inputs.init_weights(6, 150, 4, 0.05, seed=9)  # k = 4 is far too few: never legal
    busy = make(rp2, ci2, 6, 4, params(TC_KCOL, stop_on_legal=1), W2, 0)
    with TensColBatch(0) as b:
        b.add(solved)
        b.add(busy)
        b.step(6, 4)
    assert solved.tc_get_state()[1] == 0  # stopped before its first update
    best = solved.tc_best()
    assert best["conflicts"] == 0 and best["iteration"] == 0
    assert O.check_conflicts(*inputs.edge_list(rp, ci), best["coloring"]) == 0
    assert busy.tc_get_state()[1] == 6
    solved.close()
    busy.close()


def test_batch_rejects_bad_members():
    with TensColBatch(0) as b:
        empty = TensCol(0)
        with pytest.raises(TensColError):
            b.add(empty)  # no population
        empty.close()
        rp, ci = inputs.gnp(40, 0.5, seed=1)
        c = make(rp, ci, 2, 4, params(TC_KCOL), inputs.init_weights(2, 40, 4, 0.05, seed=1), 0)
        b.add(c)
        with pytest.raises(TensColError):
            b.add(c)  # already a member
        c.close()  # leaves the batch
        assert b.size() == 0
        b.step(2, 1)  # an empty batch is a no-op


def test_batched_workload_one_step_against_oracle():
    """The batched workload, every instance in the FP8 tensor-core form, one
    graph launch; each instance checked in full against the oracle."""
    specs = inputs.batched_instances()
    t = 17
    ctxs = []
    for w in specs:
        rp, ci = inputs.gnp(w["n"], w["p"], seed=w["graph_seed"])
        W = inputs.init_weights(w["D"], w["n"], w["k"], 0.01, seed=w["w_seed"])
        p = params(TC_KCOL, stop_on_legal=0, form=TC_FORM_DENSE_FP8)
        ctxs.append((make(rp, ci, w["D"], w["k"], p, W, t), rp, ci, W, p))
    with TensColBatch(0) as b:
        for c, *_ in ctxs:
            b.add(c)
        evs = [c.tc_evaluate(want_G=False, want_M=False) for c, *_ in ctxs]
        b.step(1, 1)
    for (c, rp, ci, W, p), ev in zip(ctxs, evs):
        po = oracle_params(p)
        ref = O.step(rp, ci, W, po, t, stop_on_legal=False)
        assert np.array_equal(ev["colors"], ref["colors"])
        assert np.array_equal(ev["f_color"], ref["f_color"])
        assert np.array_equal(ev["f_eq"], ref["f_eq"])
        W1, t1 = c.tc_get_state()
        assert t1 == t + 1
        assert w_step_rel_error(W1, ref, po, t) <= W_RTOL
        c.close()
