"""The data paths that depend on the shape: the bit planes of the colours
behind the pair compares (k <= 128), and the adjacency walk on shared-memory
tiles (mu = 0 on a sparse graph) with its fallback to global memory when the
largest degree makes the tiles too big.  Each case is checked against the
oracle: M~ and the colours exactly, grad_S L and the W step to tolerance."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_02261_gb300 import inputs
from paper_1909_02261_gb300.tenscol import TC_ECP, TC_KCOL, TensCol, params

from helpers import check_iteration

pytestmark = pytest.mark.gpu


def make_ctx(rp, ci, D, k, p, W, t):
    ctx = TensCol(0)
    ctx.tc_init_graph(len(rp) - 1, rp, ci)
    ctx.tc_init_population(1, D, k, p)
    if W is not None:
        ctx.tc_set_state(W, t)
    return ctx


@pytest.mark.parametrize("n,D,k", [(300, 45, 30), (257, 33, 128), (200, 20, 129)])
def test_pair_counts_follow_the_colours_over_a_run(n, D, k):
    """The bit planes are kept by XOR on every colour change; after a run of
    steps M~ must still be the count of the current colours (k = 129 takes
    the packed byte compares instead)."""
    rp, ci = inputs.gnp(n, 0.5, seed=n)
    W = inputs.init_weights(D, n, k, 0.01, seed=D)
    # a large step so that many colours change every iteration
    p = params(TC_KCOL, stop_on_legal=0, eta=0.05, lambda_=1e-3, mu=1e-3)
    with make_ctx(rp, ci, D, k, p, W, 0) as ctx:
        moved = 0
        prev = ctx.tc_evaluate(want_G=False, want_M=False)["colors"]
        for _ in range(6):
            assert ctx.tc_step(4) == 4
            ev = ctx.tc_evaluate(want_G=False)
            W1, _ = ctx.tc_get_state()
            colors = O.assign(W1)
            assert np.array_equal(ev["colors"], colors)
            assert np.array_equal(ev["Mt"], O.mtilde(colors))
            moved += int((colors != prev).sum())
            prev = colors
        assert moved > 0  # the run exercised the incremental updates
        # a fresh state rebuilds the planes from the assignment
        ctx.tc_set_state(inputs.init_weights(D, n, k, 0.01, seed=D + 1), 3)
        W2, _ = ctx.tc_get_state()
        assert np.array_equal(ctx.tc_evaluate(want_G=False)["Mt"], O.mtilde(O.assign(W2)))


def star_plus_random(n, p_edge, seed):
    """A hub joined to every other vertex, on top of G(n, p): one vertex of
    degree n - 1."""
    rp, ci = inputs.gnp(n, p_edge, seed=seed)
    adj = [set(ci[rp[i]:rp[i + 1]].tolist()) for i in range(n)]
    for v in range(1, n):
        adj[0].add(v)
        adj[v].add(0)
    rows = [np.array(sorted(a), np.int32) for a in adj]
    rp2 = np.zeros(n + 1, np.int32)
    rp2[1:] = np.cumsum([len(r) for r in rows])
    return rp2, np.concatenate(rows).astype(np.int32)


@pytest.mark.parametrize("case", ["odd_rows", "isolated", "hub_fallback", "hub_staged"])
def test_adjacency_walk_shapes(case):
    if case == "odd_rows":  # odd n and D: colour rows of odd individuals start mid-word
        n, D, k = 301, 5, 11
        rp, ci = inputs.gnp(n, 0.05, seed=11)
    elif case == "isolated":  # vertices with no neighbours, a ragged last tile
        n, D, k = 333, 8, 9
        rp, ci = inputs.gnp(n, 0.01, seed=12)
        assert (np.diff(rp) == 0).any()
    elif case == "hub_fallback":  # degree n - 1: the staged tiles would not fit (global path)
        n, D, k = 1400, 4, 12
        rp, ci = star_plus_random(n, 0.02, seed=13)
    else:  # a hub of moderate degree: staged, tiles as tall as the hub's degree
        n, D, k = 600, 6, 10
        rp, ci = star_plus_random(n, 0.02, seed=14)
    W = inputs.init_weights(D, n, k, 0.01, seed=n)
    p = params(TC_ECP, stop_on_legal=0, nu=1e-3)
    with make_ctx(rp, ci, D, k, p, W, 17) as ctx:
        check_iteration(ctx, rp, ci, p, 17)


@pytest.mark.parametrize("n,D,k", [(125, 20, 18), (1000, 7, 90), (97, 3, 33), (40, 2, 375), (33, 5, 1)])
def test_state_round_trip_through_page_locked_buffers(n, D, k):
    """tc_set_state / tc_get_state read and write page-locked host buffers
    directly (one block per 32-row tile), pageable ones through a copy and
    the element-wise conversion (also k = 375, whose tile does not fit the
    block's shared memory): both must give back the weights bit for bit,
    ragged last tiles included, and the same colours."""
    torch = pytest.importorskip("torch")
    rp, ci = inputs.gnp(n, 0.5, seed=n + k)
    W = inputs.init_weights(D, n, k, 0.05, seed=D + k)
    p = params(TC_KCOL, stop_on_legal=0)
    Wp = torch.empty((D, n, k), dtype=torch.float32, pin_memory=True).numpy()
    Wp[...] = W
    with make_ctx(rp, ci, D, k, p, W, 3) as a, make_ctx(rp, ci, D, k, p, None, 0) as b:
        b.tc_set_state(Wp, 3)
        out = torch.empty((D, n, k), dtype=torch.float32, pin_memory=True).numpy()
        out[...] = np.nan
        b.tc_get_state(out)
        assert np.array_equal(out, W)
        back, t = a.tc_get_state()
        assert t == 3 and np.array_equal(back, W)
        assert np.array_equal(a.tc_evaluate(want_G=False, want_M=False)["colors"],
                              b.tc_evaluate(want_G=False, want_M=False)["colors"])
        # one step from either state gives the same weights
        assert a.tc_step(1) == 1 and b.tc_step(1) == 1
        b.tc_get_state(out)
        assert np.array_equal(out, a.tc_get_state()[0])
