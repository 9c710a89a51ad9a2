"""GPU parity of the TensCol step (through the C ABI) against the CPU oracle.

Colours, per-vertex conflicts, fitness, equity and M~ must be bit-exact; the
gradient rows and the one-step W update must agree to 1e-5 relative to
their scale; kappa / varpi / loss to 1e-5.  The oracle always reads the
GPU's own FP32 weights, so both sides take every argmax on the same values.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_02261_gb300 import inputs
from paper_1909_02261_gb300.tenscol import TC_ECP, TC_KCOL, TensCol, TensColError, params

from helpers import W_RTOL, check_iteration, oracle_params

pytestmark = pytest.mark.gpu


def make_ctx(rp, ci, D, k, p, W=None, t=0, seed=1):
    n = len(rp) - 1
    ctx = TensCol(0)
    ctx.tc_init_graph(n, rp, ci)
    ctx.tc_init_population(seed, D, k, p)
    if W is not None:
        ctx.tc_set_state(W, t)
    return ctx


@pytest.mark.parametrize("t", [0, 4, 37])
def test_one_step_gnp125_k18_D20(t):
    rp, ci = inputs.gnp(125, 0.5, seed=1)
    W = inputs.init_weights(20, 125, 18, 0.01, seed=1)
    p = params(TC_KCOL, stop_on_legal=0, lambda_=1e-3, mu=1e-4)
    with make_ctx(rp, ci, 20, 18, p, W, t) as ctx:
        check_iteration(ctx, rp, ci, p, t)


def test_trajectory_with_reinjection_gnp125():
    """20 consecutive GPU iterations, each checked against an oracle step
    taken from the GPU's own weights (smoothing every 5 iterations)."""
    rp, ci = inputs.gnp(125, 0.5, seed=1)
    W = inputs.init_weights(20, 125, 18, 0.01, seed=1)
    p = params(TC_KCOL, stop_on_legal=0)
    worst = 0.0
    with make_ctx(rp, ci, 20, 18, p, W, 0) as ctx:
        for t in range(20):
            _, err = check_iteration(ctx, rp, ci, p, t, want_G=(t % 5 == 0))
            worst = max(worst, err)
    assert worst <= W_RTOL


@pytest.mark.parametrize("n,p_edge,D,k", [
    (1, 0.0, 1, 1), (2, 1.0, 3, 2), (33, 0.5, 3, 5), (97, 0.3, 7, 33), (70, 0.5, 5, 97),
    (64, 0.0, 4, 3), (40, 1.0, 2, 40), (161, 0.2, 9, 64), (250, 0.5, 31, 130),
    (60, 0.5, 6, 300), (129, 0.7, 5, 256), (200, 0.5, 3, 11)])
def test_ragged_and_degenerate_shapes(n, p_edge, D, k):
    rp, ci = inputs.gnp(n, p_edge, seed=n + D + k)
    W = inputs.init_weights(D, n, k, 0.05, seed=3)
    p = params(TC_KCOL, stop_on_legal=0, lambda_=1e-3, mu=1e-3)
    with make_ctx(rp, ci, D, k, p, W, 9) as ctx:
        check_iteration(ctx, rp, ci, p, 9)


@pytest.mark.parametrize("sizes,t", [
    ([75, 75, 75, 75], 3),                       # every class long: whole-warp walks only
    ([212] + [4] * 22, 4),                       # one class of 212 beside short ones (smoothing step)
    ([32, 31, 33, 28, 36, 64, 1, 2, 3, 30], 3),  # lengths around the 32-entry threshold
    ([200, 40, 40, 40, 40, 40] + [7] * 12, 9),   # long classes split unevenly between the two warps
])
def test_long_classes_in_the_class_walk(sizes, t):
    """Designed colour classes: the class walk hands classes of 32 entries or
    more to the four lane groups of one warp and the rest four side by side;
    both must give the oracle's gradient rows and W step."""
    n, k, D = sum(sizes), len(sizes), 6
    rp, ci = inputs.gnp(n, 0.5, seed=n + k)
    rng = np.random.default_rng(k)
    W = rng.normal(0.0, 0.01, (D, n, k)).astype(np.float32)
    for d in range(D):  # individual d: the classes' sizes in a permuted order of colours
        cols = np.repeat(rng.permutation(k), np.array(sizes)[np.arange(k)])[rng.permutation(n)]
        W[d, np.arange(n), cols] += 1.0
    p = params(TC_KCOL, stop_on_legal=0, lambda_=1e-3, mu=1e-3)
    with make_ctx(rp, ci, D, k, p, W, t) as ctx:
        ev = ctx.tc_evaluate(want_G=False, want_M=False)
        for d in range(D):
            assert sorted(np.bincount(ev["colors"][d], minlength=k).tolist()) == sorted(sizes)
        check_iteration(ctx, rp, ci, p, t)


def test_ties_take_lowest_colour():
    rp, ci = inputs.gnp(50, 0.4, seed=2)
    rng = np.random.default_rng(0)
    W = rng.integers(-1, 2, size=(6, 50, 7)).astype(np.float32)  # many exact ties
    p = params(TC_KCOL, stop_on_legal=0)
    with make_ctx(rp, ci, 6, 7, p, W, 3) as ctx:
        ev = ctx.tc_evaluate(want_G=False)
        assert np.array_equal(ev["colors"], np.argmax(W, axis=2))
        check_iteration(ctx, rp, ci, p, 3)


@pytest.mark.parametrize("bonus_diag", [0, 1])
def test_bonus_diagonal_reading(bonus_diag):
    rp, ci = inputs.gnp(80, 0.5, seed=5)
    W = inputs.init_weights(8, 80, 6, 0.01, seed=5)
    p = params(TC_KCOL, stop_on_legal=0, mu=1e-3, bonus_diag=bonus_diag)
    with make_ctx(rp, ci, 8, 6, p, W, 11) as ctx:
        check_iteration(ctx, rp, ci, p, 11)


@pytest.mark.parametrize("n,k", [(100, 7), (100, 10), (120, 25)])
def test_ecp_step(n, k):
    rp, ci = inputs.gnp(n, 0.1, seed=k)
    W = inputs.init_weights(16, n, k, 0.01, seed=k)
    p = params(TC_ECP, stop_on_legal=0, nu=1e-2)
    with make_ctx(rp, ci, 16, k, p, W, 13) as ctx:
        check_iteration(ctx, rp, ci, p, 13)


@pytest.mark.parametrize("n,p_edge,problem", [
    (1700, 0.3, TC_KCOL),   # B columns of a tile in shared memory, class lists read from global memory
    (2000, 0.3, TC_KCOL),   # B read from global memory (the panel no longer fits), class lists staged
    (2000, 0.01, TC_ECP),   # mu = 0 on a sparse graph: the adjacency walk on shared-memory tiles
])
def test_large_n_gradient_paths(n, p_edge, problem):
    """k_gsum's variants past the shared-memory sizes of the benchmark."""
    rp, ci = inputs.gnp(n, p_edge, seed=n + 7)
    D, k = 3, 20
    W = inputs.init_weights(D, n, k, 0.05, seed=5)
    p = params(problem, stop_on_legal=0, lambda_=1e-3, mu=1e-3 if problem == TC_KCOL else 0.0, nu=1e-3)
    with make_ctx(rp, ci, D, k, p, W, 9) as ctx:
        check_iteration(ctx, rp, ci, p, 9)


def test_full_size_gnp1000_k90_D200_one_step():
    """The benchmark workload itself, compared in full on one iteration."""
    rp, ci = inputs.gnp(1000, 0.5, seed=2)
    W = inputs.init_weights(200, 1000, 90, 0.01, seed=2)
    p = params(TC_KCOL, stop_on_legal=0)
    with make_ctx(rp, ci, 200, 90, p, W, 1234) as ctx:
        check_iteration(ctx, rp, ci, p, 1234, want_G=True)


def test_planted_partition_is_solved_and_reported():
    rp, ci, hidden = inputs.planted_partition(500, 20, 0.5, seed=3)
    W = inputs.one_hot_weights(np.stack([hidden] * 4), 20)
    W += inputs.init_weights(4, 500, 20, 1e-3, seed=3)
    W[1] = inputs.init_weights(1, 500, 20, 0.01, seed=4)[0]
    p = params(TC_KCOL, stop_on_legal=1)
    with make_ctx(rp, ci, 4, 20, p, W, 0) as ctx:
        assert ctx.tc_step(100) == 0  # legal at the first evaluation: no update
        b = ctx.tc_best()
        assert b["conflicts"] == 0 and b["individual"] == 0 and b["iteration"] == 0
        u, v = inputs.edge_list(rp, ci)
        assert O.check_conflicts(u, v, b["coloring"]) == 0
        assert np.array_equal(b["coloring"], hidden)


def test_run_to_legal_and_checker():
    """Whole-loop property: the GPU finds a legal colouring of an easy
    planted graph from random weights; the checker re-verifies it."""
    rp, ci, _ = inputs.planted_partition(125, 6, 0.5, seed=4)
    p = params(TC_KCOL, stop_on_legal=1)
    with make_ctx(rp, ci, 20, 6, p, None, 0, seed=7) as ctx:
        done = ctx.tc_step(2000)
        b = ctx.tc_best()
        assert b["conflicts"] == 0 and done < 2000
        u, v = inputs.edge_list(rp, ci)
        assert O.check_conflicts(u, v, b["coloring"]) == 0
        _, t = ctx.tc_get_state()
        assert t == done and b["iteration"] == done


def test_best_so_far_matches_oracle_run():
    """Best-so-far bookkeeping over a short run (per-step oracle restart)."""
    rp, ci = inputs.gnp(60, 0.5, seed=8)
    W = inputs.init_weights(10, 60, 9, 0.01, seed=8)
    p = params(TC_KCOL, stop_on_legal=0)
    best = None
    with make_ctx(rp, ci, 10, 9, p, W, 0) as ctx:
        for t in range(12):
            Wt, _ = ctx.tc_get_state()
            ref = O.step(rp, ci, Wt, oracle_params(p), t)
            if best is None or ref["f_min"] < best[0]:
                best = (ref["f_min"], ref["d_star"], t, ref["colors"][ref["d_star"]].copy())
            ctx.tc_step(1)
        b = ctx.tc_best()
    assert (b["conflicts"], b["individual"], b["iteration"]) == best[:3]
    assert np.array_equal(b["coloring"], best[3])


def test_graph_replay_is_bitwise_identical():
    rp, ci = inputs.gnp(125, 0.5, seed=1)
    W = inputs.init_weights(20, 125, 18, 0.01, seed=1)
    p = params(TC_KCOL, stop_on_legal=0)
    outs = []
    for chunk in (0, 8):
        with make_ctx(rp, ci, 20, 18, p, W, 0) as ctx:
            ctx.tc_set_graph_chunk(chunk)
            assert ctx.tc_step(37) == 37
            outs.append(ctx.tc_get_state()[0])
    assert np.array_equal(outs[0], outs[1])


def test_population_init_distribution_and_determinism():
    rp, ci = inputs.gnp(200, 0.5, seed=1)
    p = params(TC_KCOL, sigma0=0.01)
    with make_ctx(rp, ci, 50, 40, p, seed=123) as a, make_ctx(rp, ci, 50, 40, p, seed=123) as b, \
            make_ctx(rp, ci, 50, 40, p, seed=124) as c:
        Wa, Wb, Wc = a.tc_get_state()[0], b.tc_get_state()[0], c.tc_get_state()[0]
    assert np.array_equal(Wa, Wb) and not np.array_equal(Wa, Wc)
    x = Wa.astype(np.float64).ravel() / 0.01
    assert abs(x.mean()) < 0.01 and abs(x.std() - 1.0) < 0.01
    # Gaussian tail mass beyond 2 sigma: 4.55 %
    assert abs((np.abs(x) > 2).mean() - 0.0455) < 0.003


def test_errors_leave_context_usable(monkeypatch):
    rp, ci = inputs.gnp(30, 0.5, seed=1)
    p = params(TC_KCOL)
    with TensCol(0) as ctx:
        with pytest.raises(TensColError) as e:
            ctx.tc_step(1)
        assert e.value.code == -8  # no population yet
        bad_rp = np.array([0, 1, 1], np.int32)
        with pytest.raises(TensColError) as e:
            ctx.tc_init_graph(2, bad_rp, np.array([1], np.int32))  # asymmetric
        assert e.value.code == -2
        with pytest.raises(TensColError) as e:
            ctx.tc_init_graph(2, np.array([0, 1, 2], np.int32), np.array([0, 1], np.int32))
        assert e.value.code == -3
        ctx.tc_init_graph(30, rp, ci)
        monkeypatch.setenv("TC_FAULT", "alloc")
        with pytest.raises(TensColError) as e:
            ctx.tc_init_population(1, 4, 5, p)
        assert e.value.code == -10
        monkeypatch.delenv("TC_FAULT")
        ctx.tc_init_population(1, 4, 5, p)
        with pytest.raises(TensColError):
            ctx.tc_init_population(1, 4, 5, params(TC_KCOL, rho=0.5))
        assert ctx.tc_step(3) >= 0


def test_dense_and_csr_inputs_agree():
    rp, ci = inputs.gnp(90, 0.5, seed=6)
    A = inputs.dense(rp, ci)
    W = inputs.init_weights(5, 90, 8, 0.01, seed=6)
    p = params(TC_KCOL, stop_on_legal=0)
    with TensCol(0) as a, TensCol(0) as b:
        a.tc_init_graph(90, rp, ci)
        b.tc_init_graph(90, dense=A)
        for c in (a, b):
            c.tc_init_population(1, 5, 8, p)
            c.tc_set_state(W, 2)
            c.tc_step(3)
        assert np.array_equal(a.tc_get_state()[0], b.tc_get_state()[0])


@pytest.mark.parametrize("name", ["ecp_gnp1000p01_k25_D128", "ecp_gnp1000p09_k230_D128"])
def test_full_size_ecp_workloads(name):
    """The ECP workloads: G(1000, 0.1), k = 25 (mu = 0, so the gradient walks
    the adjacency lists) and G(1000, 0.9), k = 230 (alpha = 1.5; k > 128
    update path), D = 128, nu = 1e-5, compared in full on one iteration."""
    w = inputs.WORKLOADS[name]
    rp, ci, _ = inputs.workload_graph(name)
    W = inputs.init_weights(w["D"], w["n"], w["k"], 0.01, seed=w["w_seed"])
    p = params(TC_ECP, stop_on_legal=0, alpha=w.get("alpha", 2.5))
    with make_ctx(rp, ci, w["D"], w["k"], p, W, 321) as ctx:
        check_iteration(ctx, rp, ci, p, 321, want_G=True)
