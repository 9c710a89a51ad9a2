"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: the
worked kappa example of Section 3.6.1, chromatic polynomials and other
closed forms over the exhaustive population of all k^n colourings,
library routines (numpy argmax / matmul) for the special cases they cover,
central finite differences for the gradients of eq. 12 and eq. 13, and an
edge-by-edge recount for the fitness of eq. 1.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_02261_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def all_colorings(n, k):
    """The exhaustive population: one individual per colouring (D = k^n)."""
    return np.array(list(itertools.product(range(k), repeat=n)), dtype=np.int32)


def one_hot(colors, k):
    return inputs.one_hot_weights(colors, k).astype(np.float64)


# --- small textbook graphs and their chromatic polynomials -------------------
def cycle(n):
    return [(i, (i + 1) % n) for i in range(n)]


def complete(n):
    return [(i, j) for i in range(n) for j in range(i + 1, n)]


def wheel(rim):  # hub = vertex rim, rim vertices 0..rim-1
    return cycle(rim) + [(i, rim) for i in range(rim)]


def path(n):
    return [(i, i + 1) for i in range(n - 1)]


CHROMATIC = [
    # (name, n, edges, P(G, k))
    ("C5", 5, cycle(5), lambda k: (k - 1) ** 5 - (k - 1)),
    ("C6", 6, cycle(6), lambda k: (k - 1) ** 6 + (k - 1)),
    ("K4", 4, complete(4), lambda k: k * (k - 1) * (k - 2) * (k - 3)),
    ("P6", 6, path(6), lambda k: k * (k - 1) ** 5),
    ("W5", 6, wheel(5), lambda k: k * ((k - 2) ** 5 - (k - 2))),
    ("empty5", 5, [], lambda k: k ** 5),
]


@pytest.mark.parametrize("name,n,edges,poly", CHROMATIC, ids=[c[0] for c in CHROMATIC])
@pytest.mark.parametrize("k", [2, 3, 4])
def test_legal_count_is_chromatic_polynomial(name, n, edges, poly, k):
    rp, ci = inputs.from_edges(n, edges) if edges else (np.zeros(n + 1, np.int32),
                                                        np.zeros(0, np.int32))
    cols = all_colorings(n, k)
    gown, f = O.fitness(rp, ci, cols, k)
    assert int((f == 0).sum()) == poly(k)
    # every edge is monochromatic in exactly k^(n-1) of the k^n colourings
    assert int(f.sum()) == len(edges) * k ** (n - 1)
    # the checker recounts edge by edge
    u, v = inputs.edge_list(rp, ci)
    for d in range(0, len(cols), max(1, len(cols) // 37)):
        assert O.check_conflicts(u, v, cols[d]) == f[d]
    assert np.all(gown.sum(axis=1) % 2 == 0)


def test_petersen_chromatic_number_is_3():
    outer = cycle(5)
    spokes = [(i, i + 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    rp, ci = inputs.from_edges(10, outer + spokes + inner)
    for k, legal in [(2, False), (3, True)]:
        _, f = O.fitness(rp, ci, all_colorings(10, k), k)
        assert bool((f == 0).any()) == legal


@pytest.mark.parametrize("n,k", [(5, 2), (5, 3), (6, 3), (4, 4), (7, 3)])
def test_equitable_count_closed_form(n, k):
    """#colourings with f_eq = 0 = ways to split n labelled vertices into k
    labelled groups of sizes c1 = floor(n/k) and c2 = ceil(n/k) (eq. 3)."""
    cols = all_colorings(n, k)
    sizes, feq, _ = O.equity(cols, k)
    c1, r = divmod(n, k)
    if r == 0:
        want = math.factorial(n) // math.factorial(c1) ** k
    else:
        want = math.comb(k, r) * math.factorial(n) // (
            math.factorial(c1 + 1) ** r * math.factorial(c1) ** (k - r))
    assert int((feq == 0).sum()) == want
    assert np.all(sizes.sum(axis=1) == n)
    for d in range(0, len(cols), max(1, len(cols) // 31)):
        assert O.check_equity(cols[d], k) == feq[d]


@pytest.mark.parametrize("n,k", [(9, 4), (10, 5), (12, 5), (7, 7), (8, 3)])
def test_equity_gradient_is_central_difference(n, k):
    """eq. 14 is the central difference (step 1/2) of the continuous-count
    form of eq. 3, x -> sum_l min(|x_l - c1|, |x_l - c2|)."""
    c1, c2 = n // k, -(-n // k)
    cols = inputs.random_colors(64, n, k, seed=7)
    sizes, _, E = O.equity(cols, k)

    def feq(x):
        return np.minimum(np.abs(x - c1), np.abs(x - c2))

    h = 0.5
    fd = (feq(sizes + h) - feq(sizes - h)) / (2 * h)
    assert np.array_equal(fd, E.astype(np.float64))


def test_kappa_worked_example():
    ex = json.load(open(os.path.join(GOLDEN, "kappa_worked_example.json")))
    rp, ci = inputs.from_edges(ex["n"], ex["edges"])
    for case in ex["cases"]:
        cols = np.array(case["colors"], np.int32)
        _, f = O.fitness(rp, ci, cols, ex["k"])
        assert f.tolist() == case["conflicts"]
        M = O.mtilde(cols)
        kappa, _ = O.penalty_bonus(rp, ci, M, ex["alpha"], 1.2)
        assert kappa == case["kappa"]


@pytest.mark.parametrize("name,n,edges", [(c[0], c[1], c[2]) for c in CHROMATIC[:5]])
def test_mtilde_kappa_varpi_exhaustive_population(name, n, edges):
    """Over all k^n colourings, any two distinct vertices share a colour in
    k^(n-1) individuals and every vertex with itself in k^n = D."""
    k = 3
    rp, ci = inputs.from_edges(n, edges)
    cols = all_colorings(n, k)
    D = len(cols)
    M = O.mtilde(cols)
    want = np.full((n, n), k ** (n - 1))
    np.fill_diagonal(want, D)
    assert np.array_equal(M, want)
    a, b = 2.5, 1.2
    kap, var = O.penalty_bonus(rp, ci, M, a, b, bonus_diag=1)
    E2 = 2 * len(edges)
    assert kap == pytest.approx(E2 * float(k ** (n - 1)) ** a, rel=1e-13)
    assert var == pytest.approx((n * n - n - E2) * float(k ** (n - 1)) ** b + n * float(D) ** b,
                                rel=1e-13)
    _, var0 = O.penalty_bonus(rp, ci, M, a, b, bonus_diag=0)
    assert var0 == pytest.approx((n * n - n - E2) * float(k ** (n - 1)) ** b, rel=1e-13)


def test_library_special_cases():
    """argmax (first maximum), A.S and S S^T against numpy on random input."""
    rng = np.random.default_rng(11)
    D, n, k = 6, 40, 7
    # integers in a small range force many ties
    W = rng.integers(-2, 3, size=(D, n, k)).astype(np.float64)
    c = O.assign(W)
    assert np.array_equal(c, np.argmax(W, axis=2))
    rp, ci = inputs.gnp(n, 0.3, seed=5)
    A = inputs.dense(rp, ci).astype(np.int64)
    S = np.zeros((D, n, k), np.int64)
    S[np.arange(D)[:, None], np.arange(n)[None, :], c] = 1
    G = O.gamma(rp, ci, c, k)
    assert np.array_equal(G, np.einsum("im,dmj->dij", A, S))
    Scat = S.transpose(1, 0, 2).reshape(n, D * k)
    assert np.array_equal(O.mtilde(c), Scat @ Scat.T)
    gown, f = O.fitness(rp, ci, c, k)
    assert np.array_equal(gown, np.take_along_axis(G, c[:, :, None], 2)[:, :, 0])
    assert np.array_equal(2 * f, np.einsum("im,dim->d", A, np.einsum("dij,dmj->dim", S, S)))
    # row sums of the gamma matrix are the degrees
    assert np.array_equal(G.sum(axis=2), np.broadcast_to(np.diff(rp), (D, n)))


def test_argmax_ties_hand_built():
    W = np.array([[[1, 3, 3, 0], [5, 5, 5, 5], [-1, -2, -1, -3], [0, 0, 0, 1e-300]]], float)
    assert O.assign(W).tolist() == [[1, 0, 0, 3]]


def test_planted_partition_hidden_coloring_is_legal_and_equitable():
    rp, ci, hidden = inputs.planted_partition(500, 20, 0.5, seed=3)
    assert O.validate_graph(rp, ci) == 0
    cols = np.stack([hidden, (hidden + 3) % 20])  # a colour permutation too
    W = one_hot(cols, 20)
    out = O.step(rp, ci, W, O.make_params(problem=1, nu=1e-5, mu=0.0), t=10)
    assert out["f_color"].tolist() == [0, 0]
    assert out["f_eq"].tolist() == [0, 0]
    assert out["f_min"] == 0


def test_validate_graph_rejects_bad_lists():
    rp, ci = inputs.from_edges(4, [(0, 1), (1, 2)])
    assert O.validate_graph(rp, ci) == 0
    assert O.validate_graph(np.array([0, 1, 1, 1, 1]), np.array([1])) != 0  # asymmetric
    assert O.validate_graph(np.array([0, 1, 1]), np.array([0])) != 0  # self loop


# --- gradients ---------------------------------------------------------------
def loss_of_S(A, S, t, p, with_diag=True):
    """eq. 7 for a real-valued S (D x n x k), GCP terms (nu = 0)."""
    M = np.einsum("dij,dmj->dim", S, S)
    f_color = 0.5 * (A[None] * M).sum()
    Mt = M.sum(0)
    Abar = 1.0 - A
    if not with_diag:
        np.fill_diagonal(Abar, 0.0)
    kappa = (A * Mt ** p.alpha).sum()
    varpi = (Abar * Mt ** p.beta).sum()
    return f_color + p.lambda_ * t * kappa - p.mu * t * varpi


@pytest.mark.parametrize("alpha,beta,diag", [(2.0, 2.0, 1), (3.0, 2.0, 0), (2.5, 1.2, 1)])
def test_grad_S_is_derivative_of_loss(alpha, beta, diag):
    """eq. 13 against central differences of eq. 7 (continuous S)."""
    D, n, k, t = 3, 9, 4, 7
    rp, ci = inputs.gnp(n, 0.5, seed=13)
    A = inputs.dense(rp, ci).astype(np.float64)
    cols = inputs.random_colors(D, n, k, seed=17)
    p = O.make_params(alpha=alpha, beta=beta, lambda_=3e-2, mu=2e-2, nu=0.0, bonus_diag=diag)
    M = O.mtilde(cols)
    G = O.grad_S(rp, ci, cols, M, None, k, p, t)
    S0 = one_hot(cols, k)
    h = 1e-5
    integer = float(alpha).is_integer() and float(beta).is_integer()
    for d in range(D):
        for i in range(n):
            for j in range(k):
                # non-integer powers are smooth only where every pair term
                # stays positive: the selected colour (m~ >= 1 there)
                if not integer and j != cols[d, i]:
                    continue
                Sp, Sm = S0.copy(), S0.copy()
                Sp[d, i, j] += h
                Sm[d, i, j] -= h
                fd = (loss_of_S(A, Sp, t, p, diag) - loss_of_S(A, Sm, t, p, diag)) / (2 * h)
                assert G[d, i, j] == pytest.approx(fd, rel=1e-6, abs=1e-6), (d, i, j)


def test_grad_S_toy_property():
    """D = 1, lambda = mu = 0: the gradient at the selected colour is the
    number of conflicting neighbours (Section 4.1), and equals gamma."""
    rp, ci = inputs.gnp(21, 0.3, seed=0)
    cols = inputs.random_colors(1, 21, 5, seed=1)
    p = O.make_params(lambda_=0.0, mu=0.0, nu=0.0)
    G = O.grad_S(rp, ci, cols, O.mtilde(cols), None, 5, p, t=123)
    gown, _ = O.fitness(rp, ci, cols, 5)
    assert np.array_equal(G[0, np.arange(21), cols[0]], gown[0].astype(float))
    assert np.array_equal(G, O.gamma(rp, ci, cols, 5).astype(float))


def test_straight_through_gradient_is_softmax_derivative():
    """eq. 12: gW = d/dW <softmax(W), G> with G held fixed (central FD)."""
    rng = np.random.default_rng(3)
    D, n, k = 2, 5, 6
    W = rng.normal(0, 0.7, (D, n, k))
    G = rng.normal(0, 2.0, (D, n, k))
    p = O.make_params(eta=0.0, nb_iter=1000)
    Wn, gW = O.update(W, G, p, t=0)
    assert np.array_equal(Wn, W)  # eta = 0 and no smoothing: unchanged

    def f(w, g):
        e = np.exp(w - w.max())
        return (e / e.sum()) @ g

    h = 1e-6
    for d in range(D):
        for i in range(n):
            for j in range(k):
                wp, wm = W[d, i].copy(), W[d, i].copy()
                wp[j] += h
                wm[j] -= h
                fd = (f(wp, G[d, i]) - f(wm, G[d, i])) / (2 * h)
                assert gW[d, i, j] == pytest.approx(fd, rel=1e-6, abs=1e-8)
    # gradient rows sum to zero (softmax is shift invariant)
    assert np.allclose(gW.sum(axis=2), 0.0, atol=1e-14)


def test_update_descends_and_smooths_on_schedule():
    rng = np.random.default_rng(5)
    W = rng.normal(0, 0.01, (2, 3, 4))
    G = rng.normal(0, 1.0, (2, 3, 4))
    p = O.make_params(eta=0.0, rho=4.0, nb_iter=5)
    for t in range(12):
        Wn, _ = O.update(W, G, p, t)
        want = W / 4.0 if (t + 1) % 5 == 0 else W
        assert np.array_equal(Wn, want)
    p = O.make_params(eta=1e-3, rho=1.0)
    Wn, gW = O.update(W, G, p, t=0)
    assert np.allclose(Wn, W - 1e-3 * gW, rtol=0, atol=1e-18)

    def lin(w):  # <softmax(w), G> decreases along the step
        e = np.exp(w - w.max(axis=2, keepdims=True))
        return ((e / e.sum(axis=2, keepdims=True)) * G).sum()

    assert lin(Wn) < lin(W)


def test_step_loss_matches_eq7_on_one_hot():
    D, n, k, t = 5, 30, 4, 9
    rp, ci = inputs.gnp(n, 0.4, seed=21)
    A = inputs.dense(rp, ci).astype(np.float64)
    W = inputs.init_weights(D, n, k, 0.01, seed=22)
    p = O.make_params(lambda_=1e-3, mu=1e-4)
    out = O.step(rp, ci, W, p, t)
    S = one_hot(out["colors"], k)
    assert out["loss"] == pytest.approx(loss_of_S(A, S, t, p), rel=1e-12)
    G = O.grad_S(rp, ci, out["colors"], out["Mt"], None, k, p, t)
    assert np.array_equal(G, out["G"])


def test_run_stops_on_legal_population_and_keeps_best():
    rp, ci, hidden = inputs.planted_partition(60, 4, 0.6, seed=9)
    cols = np.stack([inputs.random_colors(1, 60, 4, seed=2)[0], hidden])
    W = one_hot(cols, 4)
    p = O.make_params()
    r = O.run(rp, ci, W, p, t0=0, max_iter=50, stop_on_legal=True)
    assert r["iters"] == 0 and r["best_f"] == 0 and r["best_t"] == 0
    assert np.array_equal(r["best_colors"], hidden)
    assert np.array_equal(r["W"], W)


def test_run_solves_planted_graph():
    """A statistical property of the whole loop: starting from N(0, 0.01)
    weights it finds a legal colouring of an easy planted 6-colourable graph."""
    rp, ci, _ = inputs.planted_partition(125, 6, 0.5, seed=4)
    W = inputs.init_weights(20, 125, 6, 0.01, seed=4)
    p = O.make_params(rho=100.0)
    r = O.run(rp, ci, W, p, t0=0, max_iter=500, stop_on_legal=True)
    assert r["best_f"] == 0
    u, v = inputs.edge_list(rp, ci)
    assert O.check_conflicts(u, v, r["best_colors"]) == 0


def test_grad_S_equity_term_is_central_difference():
    """With lambda = mu = 0, eq. 7 is f_color + nu t f_eq.  f_color is linear
    in any single s_{d,i,j} (a_ii = 0) and f_eq's central difference with
    step 1/2 at integer counts is eq. 14, so the step-1/2 central difference
    of the loss must equal eq. 13 exactly."""
    D, n, k, t = 4, 11, 3, 6
    rp, ci = inputs.gnp(n, 0.5, seed=31)
    A = inputs.dense(rp, ci).astype(np.float64)
    cols = inputs.random_colors(D, n, k, seed=32)
    nu = 0.25
    p = O.make_params(problem=1, lambda_=0.0, mu=0.0, nu=nu)
    _, _, E = O.equity(cols, k)
    G = O.grad_S(rp, ci, cols, O.mtilde(cols), E, k, p, t)
    c1, c2 = n // k, -(-n // k)

    def L(S):
        f_color = 0.5 * (A[None] * np.einsum("dij,dmj->dim", S, S)).sum()
        x = S.sum(axis=1)
        f_eq = np.minimum(np.abs(x - c1), np.abs(x - c2)).sum()
        return f_color + nu * t * f_eq

    S0 = one_hot(cols, k)
    h = 0.5
    for d in range(D):
        for i in range(n):
            for j in range(k):
                Sp, Sm = S0.copy(), S0.copy()
                Sp[d, i, j] += h
                Sm[d, i, j] -= h
                assert G[d, i, j] == pytest.approx((L(Sp) - L(Sm)) / (2 * h), abs=1e-12)


def test_step_fitness_includes_equity_only_for_ecp():
    rp, ci = inputs.gnp(30, 0.3, seed=41)
    W = inputs.init_weights(6, 30, 4, 0.01, seed=42)
    g = O.step(rp, ci, W, O.make_params(problem=0), t=3)
    e = O.step(rp, ci, W, O.make_params(problem=1, nu=1e-5, mu=0.0), t=3)
    assert g["f_min"] == g["f_color"].min()
    assert e["f_min"] == (e["f_color"] + e["f_eq"]).min()
    assert e["d_star"] == int(np.argmin(e["f_color"] + e["f_eq"]))


@pytest.mark.parametrize("alpha,beta,diag", [(2.5, 1.2, 1), (1.5, 2.0, 0)])
def test_relaxed_gradient_is_central_difference(alpha, beta, diag):
    """The relaxed loss (eq. 7 on S = softmax(W / tau)) and its analytic
    gradient (eq. 13 through the softmax Jacobian): central differences,
    h = 1e-3, FP64, on every weight of a small population."""
    D, n, k, t, tau = 3, 12, 4, 9, 0.5
    rp, ci = inputs.gnp(n, 0.5, seed=51)
    W = np.random.default_rng(52).normal(0, 0.3, (D, n, k))
    p = O.make_params(alpha=alpha, beta=beta, lambda_=2e-2, mu=1e-2, bonus_diag=diag)
    L0, g, M = O.relaxed(rp, ci, W, p, t, tau)
    # M~ of the relaxation is the library product of the softmax rows
    S = np.exp(W / tau - (W / tau).max(axis=2, keepdims=True))
    S /= S.sum(axis=2, keepdims=True)
    assert np.allclose(M, np.einsum("dij,dmj->im", S, S), rtol=1e-13, atol=1e-13)
    h = 1e-3
    for d in range(D):
        for i in range(n):
            for j in range(k):
                Wp, Wm = W.copy(), W.copy()
                Wp[d, i, j] += h
                Wm[d, i, j] -= h
                fd = (O.relaxed(rp, ci, Wp, p, t, tau, False)[0] -
                      O.relaxed(rp, ci, Wm, p, t, tau, False)[0]) / (2 * h)
                assert g[d, i, j] == pytest.approx(fd, rel=1e-5, abs=1e-7), (d, i, j)


def test_relaxed_loss_at_sharp_softmax_is_one_hot_loss():
    """As tau -> 0 the relaxation reaches the one-hot loss of the same W."""
    D, n, k, t = 4, 20, 5, 3
    rp, ci = inputs.gnp(n, 0.4, seed=61)
    W = np.random.default_rng(62).normal(0, 1.0, (D, n, k))
    p = O.make_params(lambda_=1e-2, mu=1e-3)
    L_relax, _, _ = O.relaxed(rp, ci, W, p, t, 1e-4, want_grad=False)
    L_hard = O.step(rp, ci, W, p, t, want_G=False)["loss"]
    assert L_relax == pytest.approx(L_hard, rel=1e-9)
