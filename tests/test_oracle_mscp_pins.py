"""Pins of the oracle's minimum sum colouring (Section 6: Algorithm 1 with the
additive fitness f_mscp(S_d) = sum_i sum_l s_{d,i,l} z_l in place of f_eq)
against closed forms, brute force and finite differences:

* over the exhaustive population of all k^n colourings every vertex takes
  every colour k^(n-1) times, so the costs sum to n k^(n-1) sum_l z_l;
* brute force on C_6 with z = (1, 2, 3): the fitness f_color + f_mscp is
  smallest (9) exactly at the two legal 2-colourings with colours 1 and 2;
* the gradient's additive term is the derivative of nu t f_mscp, checked by
  central differences on a continuous S;
* with all costs zero the step is the k-COL step.
"""
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_02261_gb300 import inputs

MSCP = 4


def all_colorings(n, k):
    return np.array(list(itertools.product(range(k), repeat=n)), dtype=np.int32)


@pytest.mark.parametrize("n,k,z", [(4, 3, None), (5, 2, [7, 0]), (3, 4, [1, 5, 2, 9])])
def test_cost_sum_over_all_colorings(n, k, z):
    cols = all_colorings(n, k)
    f = O.mscp(cols, z)
    zs = list(range(1, k + 1)) if z is None else z
    assert int(f.sum()) == n * k ** (n - 1) * sum(zs)
    for d in range(0, len(cols), max(1, len(cols) // 17)):  # per individual, by the definition
        assert f[d] == sum(zs[c] for c in cols[d])


def test_cycle_minimum_sum_brute_force():
    n, k = 6, 3
    rp, ci = inputs.from_edges(n, [(i, (i + 1) % n) for i in range(n)])
    cols = all_colorings(n, k)
    W = inputs.one_hot_weights(cols, k).astype(np.float64)
    out = O.step(rp, ci, W, O.make_params(problem=MSCP, nu=1e-4), t=0)
    f = out["f_color"] + out["f_mscp"]
    assert out["f_min"] == 9 == f.min()
    winners = {tuple(c) for c in cols[f == 9]}
    assert winners == {(0, 1, 0, 1, 0, 1), (1, 0, 1, 0, 1, 0)}
    assert np.array_equal(out["f_mscp"], O.mscp(cols))


def test_cost_gradient_is_central_difference():
    """With lambda = mu = 0, eq. 7 is f_color + nu t f_mscp, linear in each
    s_{d,i,l} (a_ii = 0): the central difference is exact up to rounding."""
    D, n, k, t = 3, 10, 4, 13
    rp, ci = inputs.gnp(n, 0.4, seed=5)
    A = inputs.dense(rp, ci).astype(np.float64)
    cols = inputs.random_colors(D, n, k, seed=6)
    z = np.array([3, 0, 8, 1])
    nu = 0.07
    p = O.make_params(problem=MSCP, lambda_=0.0, mu=0.0, nu=nu, zcost=z)
    W = inputs.one_hot_weights(cols, k).astype(np.float64)
    G = O.step(rp, ci, W, p, t)["G"]

    def loss(S):
        M = np.einsum("dij,dmj->dim", S, S)
        return 0.5 * (A[None] * M).sum() + nu * t * (S * z[None, None, :]).sum()

    S0 = inputs.one_hot_weights(cols, k).astype(np.float64)
    h = 1e-4
    for d in range(D):
        for i in range(n):
            for j in range(k):
                Sp, Sm = S0.copy(), S0.copy()
                Sp[d, i, j] += h
                Sm[d, i, j] -= h
                fd = (loss(Sp) - loss(Sm)) / (2 * h)
                assert G[d, i, j] == pytest.approx(fd, rel=1e-9, abs=1e-9)


def test_zero_costs_reduce_to_kcol():
    D, n, k, t = 5, 30, 6, 8
    rp, ci = inputs.gnp(n, 0.3, seed=2)
    W = inputs.init_weights(D, n, k, 0.01, seed=3)
    a = O.step(rp, ci, W, O.make_params(problem=MSCP, nu=1e-3, lambda_=1e-3, mu=1e-4, zcost=[0] * k), t)
    b = O.step(rp, ci, W, O.make_params(problem=0, nu=0.0, lambda_=1e-3, mu=1e-4), t)
    assert np.array_equal(a["W"], b["W"]) and a["loss"] == b["loss"] and a["f_min"] == b["f_min"]
    assert np.all(a["f_mscp"] == 0)


def test_negative_costs_are_rejected():
    rp, ci = inputs.gnp(8, 0.5, seed=1)
    W = inputs.init_weights(1, 8, 3, 0.01, seed=1)
    with pytest.raises(ValueError):
        O.step(rp, ci, W, O.make_params(problem=MSCP, zcost=[1, -2, 3]), 0)
