"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every entry point include/tenscol.h declares, and
fails cleanly (status codes, no crash) where a device would be needed."""
import ctypes as C
import os
import subprocess

import pytest

from paper_1909_02261_gb300 import tenscol as T


def test_library_exports_every_header_symbol():
    L = T.load()
    names = T.header_functions()
    assert len(names) >= 15
    missing = [nm for nm in names if not hasattr(L, nm)]
    assert not missing, missing


@pytest.mark.parametrize("loader", [T.load, T.load_bounds])
def test_exported_symbols_match_nm(loader):
    # the main library and the build with device index checks export the same ABI
    lib = loader()._name
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    for nm in T.header_functions():
        assert nm in exported, nm


def test_params_default_table2():
    g = T.params(T.TC_KCOL)
    e = T.params(T.TC_ECP)
    assert (g.eta, g.nb_iter, g.rho) == (pytest.approx(1e-3), 5, 100.0)
    assert g.alpha == pytest.approx(2.5) and g.beta == pytest.approx(1.2)
    assert g.lambda_ == pytest.approx(1e-5) and g.mu == pytest.approx(1e-6) and g.nu == 0.0
    assert e.mu == 0.0 and e.nu == pytest.approx(1e-5) and e.lambda_ == pytest.approx(1e-5)
    assert g.sigma0 == pytest.approx(0.01) and g.form == T.TC_FORM_ONEHOT
    L = T.load()
    assert L.tc_params_default(None, 0) == -1
    assert L.tc_params_default(C.byref(T.tc_params()), 7) == -1


def test_strerror_names_every_code():
    for code in range(0, -11, -1):
        s = T.tc_strerror(code)
        assert s and s != "unknown status"
    assert T.tc_strerror(-999) == "unknown status"


def test_null_context_is_rejected():
    L = T.load()
    i64 = C.c_int64()
    assert L.tc_step(None, 1, C.byref(i64)) == -1
    assert L.tc_init_graph(None, 3, None, None, None) == -1
    assert L.tc_destroy(None) == 0
    assert L.tc_create(None, 0) == -1


@pytest.mark.skipif(os.path.exists("/dev/nvidia0"), reason="a GPU is present")
def test_create_without_gpu_fails_cleanly():
    L = T.load()
    h = C.c_void_p(1)
    assert L.tc_create(C.byref(h), 0) == -5  # TC_ERR_CUDA
    assert h.value is None
