"""Pins of the oracle's k-partitioning problems (Section 6: Algorithm 1 with
every M_d replaced by J - M_d; fitness = cut edges, plus f_eq for the
balanced variant) against closed forms, brute force and finite differences.

* the number of 2-colourings of the cycle C_n that cut exactly c edges is
  2 binom(n, c) for even c and 0 for odd c (a closed form over the
  exhaustive population of all 2^n colourings);
* cut edges + monochromatic edges = |E| for every individual (two separate
  counting routines of the oracle, and the edge-by-edge checker);
* \\bar M~ + M~ = D J and diag(\\bar M~) = 0;
* eq. 13 for the replaced loss equals central differences of that loss in
  a continuous S;
* brute force: the minimum balanced bisection of two K4 joined by an edge
  cuts one edge, and the oracle's step finds exactly that minimum over the
  exhaustive population.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_02261_gb300 import inputs

KPART, KPART_BAL = 2, 3


def all_colorings(n, k):
    return np.array(list(itertools.product(range(k), repeat=n)), dtype=np.int32)


def one_hot(colors, k):
    return inputs.one_hot_weights(colors, k).astype(np.float64)


def cycle(n):
    return [(i, (i + 1) % n) for i in range(n)]


def two_k4_bridge():
    k4a = [(i, j) for i in range(4) for j in range(i + 1, 4)]
    k4b = [(i + 4, j + 4) for i, j in k4a]
    return 8, k4a + k4b + [(3, 4)]


@pytest.mark.parametrize("n", [4, 5, 7, 8])
def test_cut_counts_on_cycles_are_binomial(n):
    rp, ci = inputs.from_edges(n, cycle(n))
    cols = all_colorings(n, 2)
    cut = O.cut(rp, ci, cols)
    for c in range(n + 1):
        expect = 2 * math.comb(n, c) if c % 2 == 0 else 0
        assert int((cut == c).sum()) == expect, c


@pytest.mark.parametrize("n,p,k", [(12, 0.4, 3), (30, 0.2, 5), (25, 0.8, 4)])
def test_cut_plus_conflicts_is_edge_count(n, p, k):
    rp, ci = inputs.gnp(n, p, seed=n)
    cols = inputs.random_colors(40, n, k, seed=k)
    cut = O.cut(rp, ci, cols)
    _, fc = O.fitness(rp, ci, cols, k)
    n_edges = len(ci) // 2
    assert np.array_equal(cut + fc, np.full(40, n_edges))
    u, v = inputs.edge_list(rp, ci)
    for d in range(0, 40, 7):
        assert cut[d] == n_edges - O.check_conflicts(u, v, cols[d])


def test_mbar_complements_mtilde():
    D, n, k = 9, 23, 5
    cols = inputs.random_colors(D, n, k, seed=3)
    Mb, Mt = O.mbar(cols), O.mtilde(cols)
    assert np.array_equal(Mb + Mt, np.full((n, n), D))
    assert np.all(np.diag(Mb) == 0)
    # sum over ordered pairs: every individual separates n^2 - sum_j |V_j|^2 pairs
    sizes = np.stack([np.bincount(c, minlength=k) for c in cols])
    assert int(Mb.sum()) == int((n * n - (sizes ** 2).sum(axis=1)).sum())


def part_loss_of_S(A, S, t, p, with_diag=True):
    """eq. 7 with every M_d replaced by J - M_d, for a real-valued S
    (D x n x k); the equity term is left out (nu = 0)."""
    D, n, _ = S.shape
    M = np.einsum("dij,dmj->dim", S, S)
    Mbar = 1.0 - M  # J - M_d per individual
    f_cut = 0.5 * (A[None] * Mbar).sum()
    Xt = Mbar.sum(0)
    Abar = 1.0 - A
    if not with_diag:
        np.fill_diagonal(Abar, 0.0)
    # powers only over the pairs each sum runs over (with the diagonal left
    # out, its J - S S^T entry may dip below 0 under a perturbation)
    kappa = (Xt[A > 0] ** p.alpha).sum()
    varpi = (Xt[Abar > 0] ** p.beta).sum()
    return f_cut + p.lambda_ * t * kappa - p.mu * t * varpi


@pytest.mark.parametrize("alpha,beta,diag,integer", [(2.0, 2.0, 1, True), (3.0, 2.0, 0, True),
                                                     (2.5, 1.2, 0, False)])
def test_partition_grad_S_is_derivative_of_loss(alpha, beta, diag, integer):
    D, n, k, t = 3, 9, 4, 7
    rp, ci = inputs.gnp(n, 0.5, seed=13)
    A = inputs.dense(rp, ci).astype(np.float64)
    cols = inputs.random_colors(D, n, k, seed=17)
    p = O.make_params(problem=KPART, alpha=alpha, beta=beta, lambda_=3e-2, mu=2e-2, nu=0.0,
                      bonus_diag=diag)
    G = O.grad_S(rp, ci, cols, O.mbar(cols), None, k, p, t)
    S0 = one_hot(cols, k)
    h = 1e-5
    checked = 0
    for d in range(D):
        for i in range(n):
            for j in range(k):
                # non-integer powers are smooth only where every pair term the
                # entry moves stays positive: off the selected colour, the
                # pairs it touches are separated in individual d (\bar m >= 1)
                if not integer and j == cols[d, i]:
                    continue
                Sp, Sm = S0.copy(), S0.copy()
                Sp[d, i, j] += h
                Sm[d, i, j] -= h
                fd = (part_loss_of_S(A, Sp, t, p, diag) - part_loss_of_S(A, Sm, t, p, diag)) / (2 * h)
                assert G[d, i, j] == pytest.approx(fd, rel=1e-6, abs=1e-6), (d, i, j)
                checked += 1
    assert checked >= D * n * (k - 1)


def test_partition_gradient_without_population_terms_is_minus_gamma():
    rp, ci = inputs.gnp(21, 0.3, seed=0)
    cols = inputs.random_colors(2, 21, 5, seed=1)
    p = O.make_params(problem=KPART, lambda_=0.0, mu=0.0, nu=0.0)
    G = O.grad_S(rp, ci, cols, O.mbar(cols), None, 5, p, t=123)
    assert np.array_equal(G, -O.gamma(rp, ci, cols, 5).astype(float))


def test_step_minimises_cut_and_uses_mbar_terms():
    D, n, k, t = 6, 28, 4, 9
    rp, ci = inputs.gnp(n, 0.4, seed=21)
    W = inputs.init_weights(D, n, k, 0.01, seed=22)
    A = inputs.dense(rp, ci).astype(np.float64)
    for problem in (KPART, KPART_BAL):
        p = O.make_params(problem=problem, lambda_=1e-3, mu=1e-4, nu=1e-3 if problem == KPART_BAL else 0.0)
        out = O.step(rp, ci, W, p, t)
        cols = out["colors"]
        cut = O.cut(rp, ci, cols)
        assert np.array_equal(out["f_cut"], cut)
        assert np.array_equal(out["Mt"], O.mtilde(cols))  # M~ itself is still reported
        f = cut + (out["f_eq"] if problem == KPART_BAL else 0)
        assert out["f_min"] == f.min() and out["d_star"] == int(np.argmin(f))
        kap, var = O.penalty_bonus(rp, ci, O.mbar(cols), p.alpha, p.beta, p.bonus_diag)
        expect = cut.sum() + p.nu * t * out["f_eq"].sum() + p.lambda_ * t * kap - p.mu * t * var
        assert out["loss"] == pytest.approx(expect, rel=1e-12)
        assert p.lambda_ * t * kap == pytest.approx(
            p.lambda_ * t * (A * (D - out["Mt"]) ** p.alpha).sum(), rel=1e-12)
        G = O.grad_S(rp, ci, cols, O.mbar(cols), O.equity(cols, k)[2], k, p, t)
        assert np.array_equal(G, out["G"])


def test_balanced_bisection_brute_force():
    """Two K4 joined by one edge, k = 2: over all 2^8 colourings the balanced
    problem's minimum (cut + f_eq) is 1, reached only by the two planted
    bisections; the unbalanced problem's minimum is 0 (one group)."""
    n, edges = two_k4_bridge()
    rp, ci = inputs.from_edges(n, edges)
    cols = all_colorings(n, 2)
    W = one_hot(cols, 2)
    bal = O.step(rp, ci, W, O.make_params(problem=KPART_BAL, nu=1e-5, mu=0.0), t=0)
    f = bal["f_cut"] + bal["f_eq"]
    assert bal["f_min"] == 1
    winners = {tuple(c) for c in cols[f == 1]}
    assert winners == {(0, 0, 0, 0, 1, 1, 1, 1), (1, 1, 1, 1, 0, 0, 0, 0)}
    plain = O.step(rp, ci, W, O.make_params(problem=KPART), t=0, stop_on_legal=True)
    assert plain["f_min"] == 0 and not plain["updated"]
    assert np.all(cols[plain["d_star"]] == 0)  # lowest d: the all-zero colouring
