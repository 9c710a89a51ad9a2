"""ctypes binding of the TensCol CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It compiles ``tenscol_oracle.c`` with
gcc on first use (into ``oracle/_build/``) and wraps each step of the
iteration of Goudet, Duval, Hao (TensCol), Algorithm 1, with numpy arrays.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
and, for the k-partitioning problems of Section 6, by
``tests/test_oracle_partition_pins.py`` (closed forms, brute force, finite
differences, the worked kappa example of Section 3.6.1); none is "parity
unpinned".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tenscol_oracle.c")
_HDR = os.path.join(_HERE, "tenscol_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


class Params(C.Structure):
    _fields_ = [
        ("problem", C.c_int),
        ("sigma0", C.c_double),
        ("eta", C.c_double),
        ("alpha", C.c_double),
        ("lambda_", C.c_double),
        ("beta", C.c_double),
        ("mu", C.c_double),
        ("nu", C.c_double),
        ("rho", C.c_double),
        ("nb_iter", C.c_int),
        ("bonus_diag", C.c_int),
        ("zcost", C.c_void_p),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc -O2, plain C99 + libm)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB)) or force or max(
        os.path.getmtime(_SRC), os.path.getmtime(_HDR)) > os.path.getmtime(_LIB)
    if stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


_i = C.c_int
_ll = C.c_longlong
_p = C.c_void_p


def _declare(L):
    L.orc_validate_graph.argtypes = [_i, _p, _p]
    L.orc_assign.argtypes = [_i, _i, _i, _p, _p]
    L.orc_gamma.argtypes = [_i, _i, _i, _p, _p, _p, _p]
    L.orc_fitness.argtypes = [_i, _i, _i, _p, _p, _p, _p, _p]
    L.orc_equity.argtypes = [_i, _i, _i, _p, _p, _p, _p]
    L.orc_mtilde.argtypes = [_i, _i, _p, _p]
    L.orc_cut.argtypes = [_i, _i, _p, _p, _p, _p]
    L.orc_mscp.argtypes = [_i, _i, _i, _p, _p, _p]
    L.orc_mbar.argtypes = [_i, _i, _p, _p]
    L.orc_assign_multi.argtypes = [_i, _i, _i, _p, _p, _p]
    L.orc_step_multi.argtypes = [_i, _i, _i, _p, _p, _p, C.POINTER(Params), _ll, _i, _p,
                                 _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p]
    L.orc_penalty_bonus.argtypes = [_i, _p, _p, _p, C.c_double, C.c_double, _i, _p, _p]
    L.orc_grad_S.argtypes = [_i, _i, _i, _p, _p, _p, _p, _p, C.POINTER(Params), _ll, _p]
    L.orc_update.argtypes = [_i, _i, _i, C.POINTER(Params), _ll, _p, _p, _p]
    L.orc_step.argtypes = [_i, _i, _i, _p, _p, C.POINTER(Params), _ll, _i, _p,
                           _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p]
    L.orc_run.restype = _ll
    L.orc_run.argtypes = [_i, _i, _i, _p, _p, C.POINTER(Params), C.POINTER(_ll), _ll,
                          _i, _p, _p, C.POINTER(_ll), C.POINTER(_ll)]
    L.orc_relaxed.argtypes = [_i, _i, _i, _p, _p, C.POINTER(Params), _ll, C.c_double, _p, _p, _p,
                              _p]
    L.orc_check_conflicts.restype = _ll
    L.orc_check_conflicts.argtypes = [_ll, _p, _p, _p]
    L.orc_check_equity.restype = _ll
    L.orc_check_equity.argtypes = [_i, _i, _p]


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def make_params(**kw) -> Params:
    """Parameter block; defaults are the GCP column of Table 2 (rho = 100).
    problem: 0 k-COL, 1 ECP, 2 k-partitioning, 3 balanced k-partitioning,
    4 minimum sum colouring; zcost: the colour costs z_l of problem 4 (None:
    z_l = l + 1)."""
    d = dict(problem=0, sigma0=0.01, eta=1e-3, alpha=2.5, lambda_=1e-5,
             beta=1.2, mu=1e-6, nu=0.0, rho=100.0, nb_iter=5, bonus_diag=1)
    if "lambda" in kw:
        kw["lambda_"] = kw.pop("lambda")
    z = kw.pop("zcost", None)
    d.update(kw)
    p = Params(**d)
    if z is not None:
        p._z = _i32(z)  # kept alive with the block
        p.zcost = p._z.ctypes.data
    return p


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def validate_graph(rowptr, colidx) -> int:
    rowptr, colidx = _i32(rowptr), _i32(colidx)
    return lib().orc_validate_graph(len(rowptr) - 1, _ptr(rowptr), _ptr(colidx))


def assign(W):
    W = _f64(W)
    D, n, k = W.shape
    c = np.empty((D, n), np.int32)
    _check(lib().orc_assign(D, n, k, _ptr(W), _ptr(c)), "assign")
    return c


def gamma(rowptr, colidx, colors, k):
    rowptr, colidx, colors = _i32(rowptr), _i32(colidx), _i32(colors)
    D, n = colors.shape
    G = np.empty((D, n, k), np.int32)
    _check(lib().orc_gamma(D, n, k, _ptr(rowptr), _ptr(colidx), _ptr(colors), _ptr(G)), "gamma")
    return G


def fitness(rowptr, colidx, colors, k):
    rowptr, colidx, colors = _i32(rowptr), _i32(colidx), _i32(colors)
    D, n = colors.shape
    g = np.empty((D, n), np.int32)
    f = np.empty((D,), np.int64)
    _check(lib().orc_fitness(D, n, k, _ptr(rowptr), _ptr(colidx), _ptr(colors), _ptr(g), _ptr(f)),
           "fitness")
    return g, f


def equity(colors, k):
    colors = _i32(colors)
    D, n = colors.shape
    sizes = np.empty((D, k), np.int32)
    f = np.empty((D,), np.int64)
    E = np.empty((D, k), np.int32)
    _check(lib().orc_equity(D, n, k, _ptr(colors), _ptr(sizes), _ptr(f), _ptr(E)), "equity")
    return sizes, f, E


def cut(rowptr, colidx, colors):
    """Cut edges per individual (k-partitioning fitness, Section 6)."""
    rowptr, colidx, colors = _i32(rowptr), _i32(colidx), _i32(colors)
    D, n = colors.shape
    f = np.empty((D,), np.int64)
    _check(lib().orc_cut(D, n, _ptr(rowptr), _ptr(colidx), _ptr(colors), _ptr(f)), "cut")
    return f


def mscp(colors, zcost=None):
    """Total colour cost per individual (minimum sum colouring, Section 6)."""
    colors = _i32(colors)
    D, n = colors.shape
    k = int(colors.max()) + 1 if zcost is None else len(zcost)
    z = None if zcost is None else _i32(zcost)
    f = np.empty((D,), np.int64)
    _check(lib().orc_mscp(D, n, k, _ptr(colors), _ptr(z), _ptr(f)), "mscp")
    return f


def mbar(colors):
    """sum_d (J - M_d): pairs in different groups, per individual count."""
    colors = _i32(colors)
    D, n = colors.shape
    M = np.empty((n, n), np.int32)
    _check(lib().orc_mbar(D, n, _ptr(colors), _ptr(M)), "mbar")
    return M


def mtilde(colors):
    colors = _i32(colors)
    D, n = colors.shape
    M = np.empty((n, n), np.int32)
    _check(lib().orc_mtilde(D, n, _ptr(colors), _ptr(M)), "mtilde")
    return M


def penalty_bonus(rowptr, colidx, Mt, alpha, beta, bonus_diag=1):
    rowptr, colidx, Mt = _i32(rowptr), _i32(colidx), _i32(Mt)
    n = len(rowptr) - 1
    ka, va = C.c_double(), C.c_double()
    _check(lib().orc_penalty_bonus(n, _ptr(rowptr), _ptr(colidx), _ptr(Mt), alpha, beta,
                                   bonus_diag, C.byref(ka), C.byref(va)), "penalty_bonus")
    return ka.value, va.value


def grad_S(rowptr, colidx, colors, Mt, E, k, params: Params, t: int):
    rowptr, colidx, colors, Mt = _i32(rowptr), _i32(colidx), _i32(colors), _i32(Mt)
    E = None if E is None else _i32(E)
    D, n = colors.shape
    G = np.empty((D, n, k), np.float64)
    _check(lib().orc_grad_S(D, n, k, _ptr(rowptr), _ptr(colidx), _ptr(colors), _ptr(Mt), _ptr(E),
                            C.byref(params), t, _ptr(G)), "grad_S")
    return G


def update(W, G, params: Params, t: int):
    """Returns (W_new, gW) without touching the input W."""
    W = _f64(W).copy()
    G = _f64(G)
    D, n, k = W.shape
    gW = np.empty_like(W)
    _check(lib().orc_update(D, n, k, C.byref(params), t, _ptr(G), _ptr(W), _ptr(gW)), "update")
    return W, gW


def _check_graph_size(rowptr, n):
    if len(rowptr) - 1 != n:
        raise ValueError(f"graph has {len(rowptr) - 1} vertices, weights have {n}")


def step(rowptr, colidx, W, params: Params, t: int, stop_on_legal: bool = False,
         want_G: bool = True):
    """One iteration of Algorithm 1 on a copy of W (float32 or float64 input).

    Returns a dict with every intermediate of the iteration.
    """
    rowptr, colidx = _i32(rowptr), _i32(colidx)
    W = _f64(W).copy()
    D, n, k = W.shape
    _check_graph_size(rowptr, n)
    out = dict(
        colors=np.empty((D, n), np.int32), gamma_own=np.empty((D, n), np.int32),
        f_color=np.empty((D,), np.int64), f_eq=np.empty((D,), np.int64),
        f_cut=np.empty((D,), np.int64), f_mscp=np.empty((D,), np.int64), Mt=np.empty((n, n), np.int32),
        G=np.empty((D, n, k), np.float64) if want_G else None,
        gW=np.empty((D, n, k), np.float64) if want_G else None)
    loss, kappa, varpi = C.c_double(), C.c_double(), C.c_double()
    fmin, dstar, upd = C.c_longlong(), C.c_int(), C.c_int()
    _check(lib().orc_step(D, n, k, _ptr(rowptr), _ptr(colidx), C.byref(params), t,
                          int(stop_on_legal), _ptr(W),
                          _ptr(out["colors"]), _ptr(out["gamma_own"]), _ptr(out["f_color"]),
                          _ptr(out["f_eq"]), _ptr(out["f_cut"]), _ptr(out["f_mscp"]), _ptr(out["Mt"]), _ptr(out["G"]),
                          _ptr(out["gW"]),
                          C.byref(loss), C.byref(kappa), C.byref(varpi),
                          C.byref(fmin), C.byref(dstar), C.byref(upd)), "step")
    out.update(W=W, loss=loss.value, kappa=kappa.value, varpi=varpi.value,
               f_min=fmin.value, d_star=dstar.value, updated=bool(upd.value))
    return out


def assign_multi(W, demand):
    """Multicolouring Step 1 (Section 6): the dense 0/1 tensor S (D x n x k)."""
    W = _f64(W)
    D, n, k = W.shape
    demand = _i32(demand)
    S = np.empty((D, n, k), np.float64)
    _check(lib().orc_assign_multi(D, n, k, _ptr(W), _ptr(demand), _ptr(S)), "assign_multi")
    return S


def step_multi(rowptr, colidx, W, demand, params: Params, t: int, stop_on_legal: bool = False):
    """One multicolouring iteration on a copy of W; every intermediate."""
    rowptr, colidx = _i32(rowptr), _i32(colidx)
    W = _f64(W).copy()
    D, n, k = W.shape
    _check_graph_size(rowptr, n)
    demand = _i32(demand)
    out = dict(S=np.empty((D, n, k), np.float64), f_color=np.empty((D,), np.int64),
               Mt=np.empty((n, n), np.int32), G=np.empty((D, n, k), np.float64),
               gW=np.empty((D, n, k), np.float64))
    loss, kappa, varpi = C.c_double(), C.c_double(), C.c_double()
    fmin, dstar, upd = C.c_longlong(), C.c_int(), C.c_int()
    _check(lib().orc_step_multi(D, n, k, _ptr(rowptr), _ptr(colidx), _ptr(demand), C.byref(params), t,
                                int(stop_on_legal), _ptr(W), _ptr(out["S"]), _ptr(out["f_color"]),
                                _ptr(out["Mt"]), _ptr(out["G"]), _ptr(out["gW"]), C.byref(loss),
                                C.byref(kappa), C.byref(varpi), C.byref(fmin), C.byref(dstar),
                                C.byref(upd)), "step_multi")
    out.update(W=W, loss=loss.value, kappa=kappa.value, varpi=varpi.value, f_min=fmin.value,
               d_star=dstar.value, updated=bool(upd.value))
    return out


def run(rowptr, colidx, W, params: Params, t0: int, max_iter: int, stop_on_legal=True):
    """Algorithm 1 loop on a copy of W. Returns dict(W, t, iters, best_colors, best_f, best_t)."""
    rowptr, colidx = _i32(rowptr), _i32(colidx)
    W = _f64(W).copy()
    D, n, k = W.shape
    _check_graph_size(rowptr, n)
    t = C.c_longlong(t0)
    best = np.zeros((n,), np.int32)
    bf, bt = C.c_longlong(-1), C.c_longlong(-1)
    done = lib().orc_run(D, n, k, _ptr(rowptr), _ptr(colidx), C.byref(params), C.byref(t),
                         max_iter, int(stop_on_legal), _ptr(W), _ptr(best), C.byref(bf),
                         C.byref(bt))
    if done < 0:
        raise ValueError(f"oracle run failed with code {done}")
    return dict(W=W, t=t.value, iters=done, best_colors=best, best_f=bf.value, best_t=bt.value)


def relaxed(rowptr, colidx, W, params: Params, t: int, tau: float, want_grad: bool = True):
    """Relaxed loss at S = softmax(W / tau) and its exact gradient (FP64)."""
    rowptr, colidx = _i32(rowptr), _i32(colidx)
    W = _f64(W)
    D, n, k = W.shape
    _check_graph_size(rowptr, n)
    loss = C.c_double()
    g = np.empty_like(W) if want_grad else None
    M = np.empty((n, n), np.float64)
    _check(lib().orc_relaxed(D, n, k, _ptr(rowptr), _ptr(colidx), C.byref(params), t, tau,
                             _ptr(W), C.byref(loss), _ptr(g), _ptr(M)), "relaxed")
    return loss.value, g, M


def check_conflicts(edges_u, edges_v, coloring) -> int:
    u, v, c = _i32(edges_u), _i32(edges_v), _i32(coloring)
    r = lib().orc_check_conflicts(len(u), _ptr(u), _ptr(v), _ptr(c))
    if r < 0:
        raise ValueError("bad checker input")
    return int(r)


def check_equity(coloring, k) -> int:
    c = _i32(coloring)
    r = lib().orc_check_equity(len(c), k, _ptr(c))
    if r < 0:
        raise ValueError("bad checker input")
    return int(r)
