"""The allocation-free entry point tc_pair_terms_noalloc serves callers that
cannot allocate device memory (a process sharing a GPU whose memory another
framework's pool manages, a loop that must not call cudaMalloc / cudaFree
because they can synchronise the device, an embedding with a fixed memory
budget).  Its kappa and varpi must equal the FP64 oracle's and the
context-based evaluation's on two calls in a row: the scratch array keeps
the previous call's contents between calls, so a call that forgot to clear
it would show on the second one.  This file is collected last so that a run
stopping at the first failure has already run every other test."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1909_02261_gb300 import inputs
from paper_1909_02261_gb300.tenscol import TC_KCOL, TensCol, TensColError, params, tc_pair_terms_noalloc

pytestmark = pytest.mark.gpu


def call_noalloc(n, D, colors, adj, p, bonus_diag, out):
    out.fill_(float("nan"))
    tc_pair_terms_noalloc(n, D, colors.data_ptr(), adj.data_ptr(), float(p.alpha), float(p.beta), bonus_diag,
                          out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().tolist()


@pytest.mark.parametrize("n,D,k,p_edge,bonus_diag", [(125, 20, 18, 0.5, 1), (301, 37, 9, 0.3, 0),
                                                     (1000, 200, 90, 0.5, 1)])
def test_noalloc_pair_terms_match_oracle_and_context_path(n, D, k, p_edge, bonus_diag):
    rp, ci = inputs.gnp(n, p_edge, seed=n)
    W = inputs.init_weights(D, n, k, 0.01, seed=D)
    p = params(TC_KCOL, stop_on_legal=0, bonus_diag=bonus_diag)
    # expected values from the oracle alone: its own Step 1 and eq. 4-6
    colors_ref = O.assign(W)
    Mt = O.mtilde(colors_ref)
    kap_ref, var_ref = O.penalty_bonus(rp, ci, Mt, float(np.float32(p.alpha)), float(np.float32(p.beta)),
                                       bonus_diag)
    with TensCol(0) as ctx:
        ctx.tc_init_graph(n, rp, ci)
        ctx.tc_init_population(1, D, k, p)
        ctx.tc_set_state(W, 5)
        ev = ctx.tc_evaluate(want_G=False, want_M=False)
    colors = torch.tensor(colors_ref.astype(np.int32), device="cuda").to(torch.int16)
    adj = torch.tensor(inputs.dense(rp, ci), device="cuda")
    out = torch.empty(2, dtype=torch.float32, device="cuda")
    for call in range(2):
        kappa, varpi = call_noalloc(n, D, colors, adj, p, bonus_diag, out)
        assert kappa == pytest.approx(kap_ref, rel=1e-5), call
        assert varpi == pytest.approx(var_ref, rel=1e-5), call
        assert kappa == pytest.approx(float(ev["loss"][1]), rel=1e-5), call
        assert varpi == pytest.approx(float(ev["loss"][2]), rel=1e-5), call


def test_noalloc_calls_leave_device_memory_unchanged():
    n, D, k = 301, 37, 9
    rp, ci = inputs.gnp(n, 0.3, seed=7)
    colors_ref = O.assign(inputs.init_weights(D, n, k, 0.01, seed=7))
    colors = torch.tensor(colors_ref.astype(np.int32), device="cuda").to(torch.int16)
    adj = torch.tensor(inputs.dense(rp, ci), device="cuda")
    out = torch.empty(2, dtype=torch.float32, device="cuda")
    p = params(TC_KCOL)
    first = call_noalloc(n, D, colors, adj, p, 1, out)  # loads the kernel's module (lazy loading)
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert call_noalloc(n, D, colors, adj, p, 1, out) == first
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_sizes_beyond_its_array():
    x = torch.zeros(8, dtype=torch.int16, device="cuda")
    out = torch.zeros(2, dtype=torch.float32, device="cuda")
    with pytest.raises(TensColError) as e:
        tc_pair_terms_noalloc(8193, 1, x.data_ptr(), x.data_ptr(), 2.5, 1.2, 1, out.data_ptr())
    assert e.value.code == -1
