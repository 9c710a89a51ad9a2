"""The hand-written backward of the loss (eq. 7) on the GPU.

* Straight-through path (eq. 12-13 at the one-hot S): the backward equals the
  update the fused step applies, bit for bit (W_next = W - eta gW with one
  rounding per operation), and the oracle's closed-form FP64 gradient to the
  1e-5 step scale; torch autograd through ``OneHotLoss`` returns it.
* Relaxed path (eq. 7 on S = softmax(W / tau)): the GPU gradient equals the
  oracle's analytic FP64 gradient on the planted-partition workload (n = 500,
  20 hidden groups, k = 20, D = 64, tau = 0.5), and central finite
  differences (h = 1e-3, FP64, on the oracle's loss) on sampled entries.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1909_02261_gb300 import inputs
from paper_1909_02261_gb300.autograd import OneHotLoss, RelaxedLoss
from paper_1909_02261_gb300.tenscol import TC_FORM_DENSE_FP8, TC_KCOL, TensCol, params

from helpers import W_RTOL, oracle_params

pytestmark = pytest.mark.gpu


def ctx_for(rp, ci, D, k, p):
    c = TensCol(0)
    c.tc_init_graph(len(rp) - 1, rp, ci)
    c.tc_init_population(1, D, k, p)
    return c


@pytest.mark.parametrize("n,D,k,form", [(125, 20, 18, 0), (300, 9, 130, 0), (100, 6, 240, 0), (125, 20, 18, TC_FORM_DENSE_FP8)])
def test_straight_through_backward_is_the_step(n, D, k, form):
    rp, ci = inputs.gnp(n, 0.5, seed=3)
    W = inputs.init_weights(D, n, k, 0.02, seed=4)
    p = params(TC_KCOL, stop_on_legal=0, lambda_=1e-3, mu=1e-4, form=form)
    t = 6  # (t + 1) % nb_iter != 0: no smoothing this iteration
    with ctx_for(rp, ci, D, k, p) as c:
        c.tc_set_state(W, t)
        gW = torch.empty((D, n, k), dtype=torch.float32, device="cuda")
        loss = torch.empty(3, dtype=torch.float32, device="cuda")
        c.tc_st_grad_dev(gW.data_ptr(), loss.data_ptr())
        torch.cuda.synchronize()
        gW = gW.cpu().numpy()
        c.tc_step(1)
        W1, _ = c.tc_get_state()
    eta = np.float32(p.eta)
    assert np.array_equal(W1, (W - eta * gW).astype(np.float32))
    ref = O.step(rp, ci, W, oracle_params(p), t)
    scale = np.maximum(np.abs(ref["gW"]).max(axis=2, keepdims=True), 1e-30)
    assert float((np.abs(gW - ref["gW"]) / scale).max()) <= W_RTOL
    assert float(loss[0].cpu()) == pytest.approx(ref["loss"], rel=1e-5)


def test_autograd_one_hot_loss():
    n, D, k = 125, 20, 18
    rp, ci = inputs.gnp(n, 0.5, seed=1)
    W0 = inputs.init_weights(D, n, k, 0.01, seed=1)
    p = params(TC_KCOL, stop_on_legal=0)
    with ctx_for(rp, ci, D, k, p) as c:
        c.tc_set_state(None, 11)
        W = torch.tensor(W0, device="cuda", requires_grad=True)
        L = OneHotLoss.apply(W, c)
        (3.0 * L).backward()
        ref = O.step(rp, ci, W0, oracle_params(p), 11)
    assert float(L) == pytest.approx(ref["loss"], rel=1e-5)
    g = W.grad.cpu().numpy() / 3.0
    scale = np.maximum(np.abs(ref["gW"]).max(axis=2, keepdims=True), 1e-30)
    assert float((np.abs(g - ref["gW"]) / scale).max()) <= W_RTOL


def test_relaxed_gradient_planted_workload():
    rp, ci, _ = inputs.planted_partition(500, 20, 0.5, seed=3)
    D, n, k, tau, t = 64, 500, 20, 0.5, 50
    W0 = inputs.init_weights(D, n, k, 0.3, seed=3)
    p = params(TC_KCOL, stop_on_legal=0, lambda_=1e-5, mu=1e-6)
    with ctx_for(rp, ci, D, k, p) as c:
        W = torch.tensor(W0, device="cuda", requires_grad=True)
        L = RelaxedLoss.apply(W, c, tau, t)
        L.backward()
    Lr, gr, _ = O.relaxed(rp, ci, W0, oracle_params(p), t, tau)
    assert float(L) == pytest.approx(Lr, rel=1e-5)
    g = W.grad.cpu().numpy().astype(np.float64)
    scale = np.abs(gr).max(axis=2, keepdims=True)
    assert float((np.abs(g - gr) / scale).max()) <= 1e-4


def test_relaxed_gradient_central_differences():
    """GPU backward vs central differences of the FP64 relaxed loss."""
    rp, ci = inputs.gnp(40, 0.5, seed=8)
    D, n, k, tau, t = 6, 40, 7, 0.5, 30
    W0 = inputs.init_weights(D, n, k, 0.5, seed=9).astype(np.float64)
    p = params(TC_KCOL, stop_on_legal=0, lambda_=1e-3, mu=1e-4)
    with ctx_for(rp, ci, D, k, p) as c:
        W = torch.tensor(W0, dtype=torch.float32, device="cuda", requires_grad=True)
        RelaxedLoss.apply(W, c, tau, t).backward()
    g = W.grad.cpu().numpy().astype(np.float64)
    po = oracle_params(p)
    W32 = W0.astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(10)
    idx = [tuple(int(x) for x in (rng.integers(D), rng.integers(n), rng.integers(k))) for _ in range(64)]
    h = 1e-3
    gscale = np.abs(g).max()
    for (d, i, j) in idx:
        Wp, Wm = W32.copy(), W32.copy()
        Wp[d, i, j] += h
        Wm[d, i, j] -= h
        fd = (O.relaxed(rp, ci, Wp, po, t, tau, False)[0] - O.relaxed(rp, ci, Wm, po, t, tau, False)[0]) / (2 * h)
        assert abs(g[d, i, j] - fd) <= 1e-4 * gscale, (d, i, j, g[d, i, j], fd)
