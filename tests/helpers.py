"""Shared test helpers: oracle parameters matching the library's FP32
parameters, and the tolerances of the parity bar."""
import numpy as np

from oracle import oracle as O

# The W step must agree with the FP64 oracle to 1e-5 relative to the step's
# own scale: max(|W_ref|, eta * max_j |grad_W L[d, i, j]|) (divided by rho
# when the iteration smooths).  Colours, conflicts, equity and M~ are exact.
W_RTOL = 1e-5


def f32(x):
    return float(np.float32(x))


def oracle_params(p, zcost=None):
    """Oracle parameter block holding exactly the FP32 values the library uses
    (zcost: the colour costs of the minimum sum colouring, None = l + 1)."""
    return O.make_params(problem=int(p.problem), sigma0=f32(p.sigma0), eta=f32(p.eta),
                         alpha=f32(p.alpha), lambda_=f32(p.lambda_), beta=f32(p.beta),
                         mu=f32(p.mu), nu=f32(p.nu), rho=f32(p.rho), nb_iter=int(p.nb_iter),
                         bonus_diag=int(p.bonus_diag), zcost=zcost)


def additive(ref, po):
    """The oracle's additive fitness term: f_mscp (minimum sum colouring) or f_eq."""
    return ref["f_mscp"] if po.problem == 4 else ref["f_eq"]


def w_step_rel_error(W_gpu, ref, po, t):
    """Max over elements of |W_gpu - W_ref| / scale (see W_RTOL)."""
    div = po.rho if (t + 1) % po.nb_iter == 0 else 1.0
    gmax = np.abs(ref["gW"]).max(axis=2, keepdims=True)
    scale = np.maximum(np.abs(ref["W"]), po.eta * gmax / div)
    scale = np.maximum(scale, np.finfo(np.float32).tiny)
    return float((np.abs(W_gpu.astype(np.float64) - ref["W"]) / scale).max())


def g_rel_error(G_gpu, G_ref):
    """grad_S L rows: error relative to max(1, row max |G_ref|)."""
    scale = np.maximum(1.0, np.abs(G_ref).max(axis=2, keepdims=True))
    return float((np.abs(G_gpu.astype(np.float64) - G_ref) / scale).max())


def loss_close(gpu_loss, ref, po, t, rtol=1e-5):
    """loss[0..3] = L, kappa, varpi, sum f_color against the oracle (the
    fitness term of L is the cut edges for the partitioning problems)."""
    L, kap, var, fsum = [float(x) for x in gpu_loss]
    assert fsum == float(ref["f_color"].sum())
    assert kap == _approx(ref["kappa"], rtol)
    assert var == _approx(ref["varpi"], rtol)
    fit = ref["f_cut"] if po.problem in (2, 3) else ref["f_color"]
    scale = abs(fit.sum()) + po.nu * t * abs(additive(ref, po).sum()) + \
        po.lambda_ * t * abs(ref["kappa"]) + po.mu * t * abs(ref["varpi"])
    assert abs(L - ref["loss"]) <= rtol * max(scale, 1.0), (L, ref["loss"])


def _approx(x, rtol):
    import pytest
    return pytest.approx(x, rel=rtol, abs=1e-30)


def check_iteration(ctx, rp, ci, p, t, want_G=True, zcost=None):
    """Evaluate + one step on the GPU vs one oracle step from the GPU's own
    weights: exact colours / conflicts / equity (or colour costs) / M~, G and
    W within W_RTOL."""
    W0, t0 = ctx.tc_get_state()
    assert t0 == t
    po = oracle_params(p, zcost)
    ev = ctx.tc_evaluate(want_G=want_G)
    ref = O.step(rp, ci, W0, po, t, stop_on_legal=False)
    assert np.array_equal(ev["colors"], ref["colors"])
    assert np.array_equal(ev["gamma_own"], ref["gamma_own"])
    assert np.array_equal(ev["f_color"], ref["f_color"])
    assert np.array_equal(ev["f_eq"], additive(ref, po))
    assert np.array_equal(ev["Mt"], ref["Mt"])
    loss_close(ev["loss"], ref, po, t)
    if want_G:
        assert g_rel_error(ev["G"], ref["G"]) <= W_RTOL
    assert ctx.tc_step(1) == 1
    W1, t1 = ctx.tc_get_state()
    assert t1 == t + 1
    err = w_step_rel_error(W1, ref, po, t)
    assert err <= W_RTOL, err
    # the next assignment (argmax epilogue of the update) equals Step 1 on W1
    ev1 = ctx.tc_evaluate(want_G=False, want_M=False)
    assert np.array_equal(ev1["colors"], O.assign(W1))
    return ref, err
