"""Pins of the oracle's multicolouring (Section 6: vertex i takes the c_i
colours of largest weight; everything else of Algorithm 1 on the multi-hot S)
against closed forms, brute force, library routines and finite differences:

* Step 1 against a stable numpy sort (lowest index first among equal
  weights) on random and hand-built tied rows;
* legal multicolourings counted over the exhaustive population of colour
  sets: C(k, c1) C(k - c1, c2) for one edge, k (k - 1) C(k - 2, 2) for a
  triangle with demands (1, 1, 2);
* f_color equals an edge-by-edge count of shared colours;
* with every demand 1 the step is the k-COL step;
* grad_S L (eq. 13 on multi-hot S) equals central differences of eq. 7.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_02261_gb300 import inputs


def topc_numpy(W, demand):
    D, n, k = W.shape
    S = np.zeros_like(W)
    for d in range(D):
        for i in range(n):
            order = np.argsort(-W[d, i], kind="stable")  # larger first, lower index first on ties
            S[d, i, order[:demand[i]]] = 1.0
    return S


def test_assign_multi_is_stable_top_c():
    rng = np.random.default_rng(0)
    W = rng.normal(size=(4, 9, 7))
    W[0, 0] = [1, 3, 3, 0, 3, -1, 2]  # ties among the largest
    demand = rng.integers(1, 8, 9)
    demand[0] = 2
    S = O.assign_multi(W, demand)
    assert np.array_equal(S, topc_numpy(W, demand))
    assert np.array_equal(np.nonzero(S[0, 0])[0], [1, 2])
    assert np.array_equal(S.sum(axis=2), np.broadcast_to(demand, (4, 9)))


def sets_population(k, demands):
    """Every assignment of colour sets (one individual each), as one-hot W."""
    per_vertex = [list(itertools.combinations(range(k), c)) for c in demands]
    rows = []
    for choice in itertools.product(*per_vertex):
        w = np.zeros((len(demands), k))
        for i, cs in enumerate(choice):
            w[i, list(cs)] = 1.0
        rows.append(w)
    return np.array(rows)


@pytest.mark.parametrize("k,c1,c2", [(4, 1, 2), (5, 2, 2), (6, 3, 2)])
def test_single_edge_legal_count(k, c1, c2):
    rp, ci = inputs.from_edges(2, [(0, 1)])
    W = sets_population(k, [c1, c2])
    out = O.step_multi(rp, ci, W, [c1, c2], O.make_params(), t=0)
    assert int((out["f_color"] == 0).sum()) == math.comb(k, c1) * math.comb(k - c1, c2)
    # f_color is the number of shared colours of the edge
    inter = (W[:, 0, :] * W[:, 1, :]).sum(axis=1)
    assert np.array_equal(out["f_color"], inter.astype(np.int64))


def test_triangle_legal_count():
    k = 4
    rp, ci = inputs.from_edges(3, [(0, 1), (1, 2), (0, 2)])
    W = sets_population(k, [1, 1, 2])
    out = O.step_multi(rp, ci, W, [1, 1, 2], O.make_params(), t=0)
    assert int((out["f_color"] == 0).sum()) == k * (k - 1) * math.comb(k - 2, 2)


def test_conflicts_are_shared_colours_per_edge():
    D, n, k = 5, 30, 8
    rp, ci = inputs.gnp(n, 0.3, seed=3)
    W = inputs.init_weights(D, n, k, 0.1, seed=4)
    demand = np.random.default_rng(5).integers(1, 4, n)
    out = O.step_multi(rp, ci, W, demand, O.make_params(), t=2)
    u, v = inputs.edge_list(rp, ci)
    S = out["S"]
    recount = [(S[d, u] * S[d, v]).sum() for d in range(D)]
    assert np.array_equal(out["f_color"], np.array(recount, np.int64))
    # M~ of eq. 4: shared colours summed over individuals, m~_ii = D c_i
    assert np.array_equal(np.diag(out["Mt"]), D * demand)


def test_unit_demands_give_the_kcol_step():
    D, n, k, t = 4, 25, 6, 11
    rp, ci = inputs.gnp(n, 0.4, seed=6)
    W = inputs.init_weights(D, n, k, 0.01, seed=7)
    p = O.make_params(lambda_=1e-3, mu=1e-4)
    a = O.step_multi(rp, ci, W, np.ones(n, np.int32), p, t)
    b = O.step(rp, ci, W, p, t)
    assert np.array_equal(a["f_color"], b["f_color"]) and np.array_equal(a["Mt"], b["Mt"])
    assert np.allclose(a["G"], b["G"], rtol=1e-12, atol=1e-12)
    assert np.allclose(a["W"], b["W"], rtol=1e-12, atol=0)
    assert a["loss"] == pytest.approx(b["loss"], rel=1e-12)


def loss_of_S(A, S, t, p):
    M = np.einsum("dij,dmj->dim", S, S)
    Mt = M.sum(0)
    return 0.5 * (A[None] * M).sum() + p.lambda_ * t * (A * Mt ** p.alpha).sum() - \
        p.mu * t * ((1.0 - A) * Mt ** p.beta).sum()


def test_multi_gradient_is_central_difference():
    """Integer exponents keep eq. 7 a polynomial in S, so every entry of
    grad_S L at the multi-hot S is checked."""
    D, n, k, t = 3, 8, 5, 6
    rp, ci = inputs.gnp(n, 0.5, seed=8)
    A = inputs.dense(rp, ci).astype(np.float64)
    W = inputs.init_weights(D, n, k, 0.1, seed=9)
    demand = np.array([1, 2, 3, 1, 2, 1, 2, 3])
    p = O.make_params(alpha=2.0, beta=2.0, lambda_=2e-2, mu=1e-2)
    out = O.step_multi(rp, ci, W, demand, p, t)
    S0 = out["S"]
    h = 1e-5
    for d in range(D):
        for i in range(n):
            for j in range(k):
                Sp, Sm = S0.copy(), S0.copy()
                Sp[d, i, j] += h
                Sm[d, i, j] -= h
                fd = (loss_of_S(A, Sp, t, p) - loss_of_S(A, Sm, t, p)) / (2 * h)
                assert out["G"][d, i, j] == pytest.approx(fd, rel=1e-6, abs=1e-6), (d, i, j)


def test_bad_demands_are_rejected():
    W = np.zeros((1, 3, 4))
    for bad in ([0, 1, 1], [1, 5, 1]):
        with pytest.raises(ValueError):
            O.assign_multi(W, bad)
