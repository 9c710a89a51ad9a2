"""The allocation-free entry point, for callers that cannot allocate device
memory (inside a graph capture, under a foreign memory pool, on a fixed
budget): tc_pair_terms_noalloc must give the pair terms (kappa of eq. 5,
varpi of eq. 6) the context-based evaluation gives, on two calls in a row
(its scratch array keeps the previous call's contents between calls)."""
import numpy as np
import pytest
import torch

from paper_1909_02261_gb300 import inputs
from paper_1909_02261_gb300.tenscol import TC_KCOL, TensCol, params, tc_pair_terms_noalloc

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,D,k,p_edge,bonus_diag", [(125, 20, 18, 0.5, 1), (301, 37, 9, 0.3, 0),
                                                     (1000, 200, 90, 0.5, 1)])
def test_noalloc_pair_terms_match_context_path(n, D, k, p_edge, bonus_diag):
    rp, ci = inputs.gnp(n, p_edge, seed=n)
    W = inputs.init_weights(D, n, k, 0.01, seed=D)
    p = params(TC_KCOL, stop_on_legal=0, bonus_diag=bonus_diag)
    with TensCol(0) as ctx:
        ctx.tc_init_graph(n, rp, ci)
        ctx.tc_init_population(1, D, k, p)
        ctx.tc_set_state(W, 5)
        ev = ctx.tc_evaluate(want_G=False, want_M=False)
    colors = torch.tensor(ev["colors"].astype(np.int32), device="cuda").to(torch.int16)
    adj = torch.tensor(inputs.dense(rp, ci), device="cuda")
    out = torch.full((2,), float("nan"), dtype=torch.float32, device="cuda")
    for call in range(2):
        out.fill_(float("nan"))
        tc_pair_terms_noalloc(n, D, colors.data_ptr(), adj.data_ptr(), float(p.alpha), float(p.beta),
                              bonus_diag, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        kappa, varpi = out.cpu().tolist()
        assert kappa == pytest.approx(float(ev["loss"][1]), rel=1e-5), call
        assert varpi == pytest.approx(float(ev["loss"][2]), rel=1e-5), call


def test_noalloc_rejects_sizes_beyond_its_array():
    from paper_1909_02261_gb300.tenscol import TensColError
    x = torch.zeros(8, dtype=torch.int16, device="cuda")
    out = torch.zeros(2, dtype=torch.float32, device="cuda")
    with pytest.raises(TensColError) as e:
        tc_pair_terms_noalloc(8193, 1, x.data_ptr(), x.data_ptr(), 2.5, 1.2, 1, out.data_ptr())
    assert e.value.code == -1
