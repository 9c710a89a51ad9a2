"""Thin Python binding of libtenscol (include/tenscol.h) through ctypes.

Argument marshalling only: every step of the TensCol iteration runs in the
library's CUDA kernels.  Functions keep the C names (``tc_step`` ...); the
``TensCol`` class wraps one context.  There is no CPU fallback: if the
library cannot be loaded the import-time helpers raise.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

from . import build as _build

TC_OK = 0
TC_KCOL, TC_ECP, TC_KPART, TC_KPART_BAL, TC_MSCP = 0, 1, 2, 3, 4  # problems (tenscol.h)
TC_FORM_ONEHOT, TC_FORM_DENSE_FP8, TC_FORM_DENSE_FP32 = 0, 1, 2
TC_KID_PAIRS, TC_KID_CLASSES, TC_KID_UPDATE, TC_KID_GEMM_M, TC_KID_GEMM_G, TC_KID_GSUM, TC_KID_GEMM_F, \
    TC_KID_FRONT = range(8)
KERNEL_NAMES = {TC_KID_PAIRS: "k_pairs", TC_KID_CLASSES: "k_classes", TC_KID_UPDATE: "k_update",
                TC_KID_GEMM_M: "gemm_mtilde", TC_KID_GEMM_G: "gemm_gamma", TC_KID_GSUM: "k_gsum",
                TC_KID_GEMM_F: "gemm_fused", TC_KID_FRONT: "k_front"}
HEADER = os.path.join(_build.INCLUDE, "tenscol.h")


class tc_params(C.Structure):
    _fields_ = [
        ("problem", C.c_int),
        ("sigma0", C.c_float),
        ("eta", C.c_float),
        ("alpha", C.c_float),
        ("lambda_", C.c_float),
        ("beta", C.c_float),
        ("mu", C.c_float),
        ("nu", C.c_float),
        ("rho", C.c_float),
        ("nb_iter", C.c_int),
        ("stop_on_legal", C.c_int),
        ("bonus_diag", C.c_int),
        ("form", C.c_int),
    ]


class tc_trace_entry(C.Structure):
    _fields_ = [("t", C.c_int64), ("f_min", C.c_int32), ("individual", C.c_int32), ("f_color", C.c_int32),
                ("f_add", C.c_int32), ("loss", C.c_float), ("kappa", C.c_float), ("varpi", C.c_float),
                ("pad", C.c_int32)]


class TensColError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {tc_strerror(code)} ({code})")


_lib = None


def header_functions() -> list[str]:
    """Names of the entry points declared in include/tenscol.h."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tc_[a-z0-9_]+)\s*\(", src)))


_lib_bounds = None


def load_bounds(build_if_missing: bool = True):
    """libtenscol_bounds.so: the same entry points with the device-side index
    checks of the class walk (TC_BOUNDS=1), for failure tests."""
    global _lib_bounds
    if _lib_bounds is None:
        if build_if_missing:
            _build.build()
        _lib_bounds = _declare(C.CDLL(_build.LIB_BOUNDS))
    return _lib_bounds


def load(build_if_missing: bool = True):
    """Load (building if needed) the shared library and declare signatures."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    _lib = _declare(C.CDLL(path))
    return _lib


def _declare(L):
    """Declares the argument and result types of the entry points on L."""
    vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    P = C.POINTER
    sig = {
        "tc_strerror": (C.c_char_p, [C.c_int]),
        "tc_params_default": (C.c_int, [P(tc_params), C.c_int]),
        "tc_create": (C.c_int, [P(vp), C.c_int]),
        "tc_destroy": (C.c_int, [vp]),
        "tc_set_stream": (C.c_int, [vp, vp]),
        "tc_init_graph": (C.c_int, [vp, C.c_int, vp, vp, vp]),
        "tc_init_population": (C.c_int, [vp, C.c_uint64, C.c_int, C.c_int, P(tc_params)]),
        "tc_set_params": (C.c_int, [vp, P(tc_params)]),
        "tc_step": (C.c_int, [vp, i64, P(i64)]),
        "tc_best": (C.c_int, [vp, vp, P(i64), P(i64), P(i32), P(i64)]),
        "tc_get_state": (C.c_int, [vp, vp, P(i64)]),
        "tc_set_state": (C.c_int, [vp, vp, P(i64)]),
        "tc_get_state_dev": (C.c_int, [vp, vp]),
        "tc_set_state_dev": (C.c_int, [vp, vp]),
        "tc_evaluate": (C.c_int, [vp, vp, vp, vp, vp, vp, vp, vp]),
        "tc_launch_count": (C.c_int, [vp, P(i64)]),
        "tc_set_graph_chunk": (C.c_int, [vp, C.c_int]),
        "tc_set_wait_limit": (C.c_int, [vp, i64]),
        "tc_step_async": (C.c_int, [vp, i64]),
        "tc_set_timing": (C.c_int, [vp, C.c_int]),
        "tc_kernel_times": (C.c_int, [vp, vp, vp]),
        "tc_st_grad_dev": (C.c_int, [vp, vp, vp]),
        "tc_relaxed_dev": (C.c_int, [vp, vp, C.c_float, i64, vp, vp]),
        "tc_pair_terms_noalloc": (C.c_int, [C.c_int, C.c_int, vp, vp, C.c_float, C.c_float, C.c_int, vp,
                                            vp]),
        "tc_kdescent": (C.c_int, [vp, C.c_uint64, C.c_int, C.c_int, C.c_int, i64, P(tc_params), P(i32), vp,
                                  P(i64)]),
        "tc_dense_plan": (C.c_int, [vp, vp, vp]),
        "tc_dense_set_plan": (C.c_int, [vp, vp]),
        "tc_set_color_costs": (C.c_int, [vp, vp, C.c_int]),
        "tc_set_demands": (C.c_int, [vp, vp, C.c_int]),
        "tc_set_trace": (C.c_int, [vp, C.c_int, C.c_int]),
        "tc_get_trace": (C.c_int, [vp, vp, C.c_int, P(C.c_int)]),
        "tc_best_multi": (C.c_int, [vp, vp, C.c_int, vp, vp, vp]),
        "tc_get_multicolors": (C.c_int, [vp, vp, C.c_int]),
        "tc_batch_create": (C.c_int, [P(vp), C.c_int]),
        "tc_batch_add": (C.c_int, [vp, vp]),
        "tc_batch_step": (C.c_int, [vp, i64, C.c_int]),
        "tc_batch_size": (C.c_int, [vp, P(C.c_int)]),
        "tc_batch_destroy": (C.c_int, [vp]),
    }
    for name, (res, args) in sig.items():
        if hasattr(L, name):
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
    return L


def tc_strerror(code: int) -> str:
    try:
        return load().tc_strerror(code).decode()
    except OSError:
        return f"status {code}"


def _ck(rc: int, what: str):
    if rc != TC_OK:
        raise TensColError(rc, what)


def _ptr(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


def tc_pair_terms_noalloc(n: int, D: int, colors_ptr: int, adj_ptr: int, alpha: float, beta: float,
                          bonus_diag: int, out_ptr: int, stream_handle: int | None = None):
    """Device pointers in, no allocation: kappa and varpi into out_ptr[0:2]."""
    _ck(load().tc_pair_terms_noalloc(n, D, C.c_void_p(colors_ptr), C.c_void_p(adj_ptr), alpha, beta,
                                     bonus_diag, C.c_void_p(out_ptr), stream_handle),
        "tc_pair_terms_noalloc")


def params(problem: int = TC_KCOL, **kw) -> tc_params:
    """Table 2 defaults for `problem`, overridden by keyword arguments."""
    p = tc_params()
    _ck(load().tc_params_default(C.byref(p), problem), "tc_params_default")
    if "lambda" in kw:
        kw["lambda_"] = kw.pop("lambda")
    for key, val in kw.items():
        if not hasattr(p, key):
            raise KeyError(key)
        setattr(p, key, val)
    return p


class TensCol:
    """One context: a graph and a population on one CUDA device (bounds: on
    the library with device-side index checks)."""

    def __init__(self, device: int = 0, bounds: bool = False):
        self._L = load_bounds() if bounds else load()
        h = C.c_void_p()
        _ck(self._L.tc_create(C.byref(h), device), "tc_create")
        self.h = h
        self.n = self.D = self.k = 0

    def close(self):
        if getattr(self, "h", None):
            self._L.tc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # --- setup ------------------------------------------------------------
    def tc_init_graph(self, n, rowptr=None, colidx=None, dense=None):
        rp = None if rowptr is None else np.ascontiguousarray(rowptr, np.int32)
        ci = None if colidx is None else np.ascontiguousarray(colidx, np.int32)
        de = None if dense is None else np.ascontiguousarray(dense, np.uint8)
        _ck(self._L.tc_init_graph(self.h, int(n), _ptr(rp), _ptr(ci), _ptr(de)), "tc_init_graph")
        self.n = int(n)

    def tc_init_population(self, seed: int, D: int, k: int, p: tc_params | None = None):
        _ck(self._L.tc_init_population(self.h, seed, D, k, None if p is None else C.byref(p)),
            "tc_init_population")
        self.D, self.k = D, k
        self.cmax = 1  # a new population takes one colour per vertex

    def tc_set_params(self, p: tc_params):
        _ck(self._L.tc_set_params(self.h, C.byref(p)), "tc_set_params")

    def tc_set_stream(self, stream_handle: int | None):
        _ck(self._L.tc_set_stream(self.h, stream_handle), "tc_set_stream")

    def tc_set_graph_chunk(self, chunk: int):
        _ck(self._L.tc_set_graph_chunk(self.h, chunk), "tc_set_graph_chunk")

    def tc_set_wait_limit(self, ns: int):
        """Limit (ns) of every bounded device wait; 0 restores one second."""
        _ck(self._L.tc_set_wait_limit(self.h, ns), "tc_set_wait_limit")

    # --- iterate ------------------------------------------------------------
    def tc_step(self, n_iters: int) -> int:
        done = C.c_int64()
        _ck(self._L.tc_step(self.h, n_iters, C.byref(done)), "tc_step")
        return done.value

    def tc_best(self):
        col = np.empty(self.n, np.int32)
        fc, fe, t = C.c_int64(), C.c_int64(), C.c_int64()
        d = C.c_int32()
        _ck(self._L.tc_best(self.h, _ptr(col), C.byref(fc), C.byref(fe), C.byref(d), C.byref(t)),
            "tc_best")
        return dict(coloring=col, conflicts=fc.value, equity=fe.value, individual=d.value,
                    iteration=t.value)

    def tc_get_state(self, W_out=None):
        W = W_out if W_out is not None else np.empty((self.D, self.n, self.k), np.float32)
        t = C.c_int64()
        _ck(self._L.tc_get_state(self.h, _ptr(W), C.byref(t)), "tc_get_state")
        return W, t.value

    def tc_set_state(self, W=None, t: int | None = None):
        Wc = None if W is None else np.ascontiguousarray(W, np.float32)
        if Wc is not None and Wc.size != self.D * self.n * self.k:
            raise ValueError("W has the wrong size")
        tt = None if t is None else C.byref(C.c_int64(t))
        _ck(self._L.tc_set_state(self.h, _ptr(Wc), tt), "tc_set_state")

    def tc_get_state_dev(self, ptr: int):
        _ck(self._L.tc_get_state_dev(self.h, C.c_void_p(ptr)), "tc_get_state_dev")

    def tc_set_state_dev(self, ptr: int):
        _ck(self._L.tc_set_state_dev(self.h, C.c_void_p(ptr)), "tc_set_state_dev")

    def tc_evaluate(self, want_G: bool = True, want_M: bool = True):
        D, n, k = self.D, self.n, self.k
        out = dict(colors=np.empty((D, n), np.int32), gamma_own=np.empty((D, n), np.int32),
                   f_color=np.empty(D, np.int32), f_eq=np.empty(D, np.int32),
                   Mt=np.empty((n, n), np.int32) if want_M else None,
                   G=np.empty((D, n, k), np.float32) if want_G else None,
                   loss=np.empty(4, np.float32))
        _ck(self._L.tc_evaluate(self.h, _ptr(out["colors"]), _ptr(out["gamma_own"]),
                                _ptr(out["f_color"]), _ptr(out["f_eq"]), _ptr(out["Mt"]),
                                _ptr(out["G"]), _ptr(out["loss"])), "tc_evaluate")
        return out

    def tc_step_async(self, n_iters: int):
        _ck(self._L.tc_step_async(self.h, n_iters), "tc_step_async")

    def tc_set_timing(self, on: bool):
        _ck(self._L.tc_set_timing(self.h, int(on)), "tc_set_timing")

    def tc_kernel_times(self):
        ms = np.zeros(8, np.float64)
        cnt = np.zeros(8, np.int64)
        _ck(self._L.tc_kernel_times(self.h, _ptr(ms), _ptr(cnt)), "tc_kernel_times")
        return ms, cnt

    def tc_st_grad_dev(self, gradW_ptr: int, loss_ptr: int | None):
        _ck(self._L.tc_st_grad_dev(self.h, C.c_void_p(gradW_ptr),
                                   None if loss_ptr is None else C.c_void_p(loss_ptr)), "tc_st_grad_dev")

    def tc_relaxed_dev(self, W_ptr: int, tau: float, t: int, loss_ptr: int, gradW_ptr: int):
        _ck(self._L.tc_relaxed_dev(self.h, C.c_void_p(W_ptr), tau, t, C.c_void_p(loss_ptr),
                                   C.c_void_p(gradW_ptr)), "tc_relaxed_dev")

    def tc_kdescent(self, seed: int, D: int, k_start: int, k_min: int, max_iters: int,
                    p: tc_params | None = None):
        """Decreasing-k descent: (k_best or -1, its colouring or None, iterations run)."""
        kb, it = C.c_int32(), C.c_int64()
        col = np.empty(self.n, np.int32)
        _ck(self._L.tc_kdescent(self.h, seed, D, k_start, k_min, max_iters, None if p is None else C.byref(p),
                                C.byref(kb), _ptr(col), C.byref(it)), "tc_kdescent")
        # the context keeps the population of the last k tried
        last = k_min if kb.value == k_min else (kb.value - 1 if kb.value > 0 else k_start)
        self.D, self.k = D, last
        self.cmax = 1
        return kb.value, (col if kb.value > 0 else None), it.value

    def tc_dense_plan(self):
        """The autotuned plan of the dense contractions (see tenscol.h)."""
        plan = np.zeros(9, np.int32)
        us = np.zeros(3, np.float32)
        _ck(self._L.tc_dense_plan(self.h, _ptr(plan), _ptr(us)), "tc_dense_plan")
        return dict(gamma_tile_m=int(plan[0]), gamma_tile_n=int(plan[1]), gamma_cluster=int(plan[2]),
                    mtilde_tile_m=int(plan[3]), mtilde_tile_n=int(plan[4]), mtilde_cluster=int(plan[5]),
                    mtilde_splits=int(plan[6]), fused=bool(plan[7]), candidates=int(plan[8]),
                    gamma_us=float(us[0]), mtilde_us=float(us[1]), fused_us=float(us[2]))

    def tc_dense_set_plan(self, gamma, mtilde, mtilde_splits, fused=False):
        """Pins the plan: `gamma` and `mtilde` are (unit rows, column tile,
        cluster) triples, e.g. (128, 256, 4) or (256, 256, 2) for a CTA pair;
        fused: both contractions in one launch (one shape for both)."""
        plan = np.array([*gamma, *mtilde, mtilde_splits, int(fused)], np.int32)
        _ck(self._L.tc_dense_set_plan(self.h, _ptr(plan)), "tc_dense_set_plan")

    def tc_set_color_costs(self, z):
        """Colour costs z_l of the minimum sum colouring (TC_MSCP), one per colour."""
        z = np.ascontiguousarray(z, np.int32)
        _ck(self._L.tc_set_color_costs(self.h, _ptr(z), int(z.size)), "tc_set_color_costs")

    def tc_set_trace(self, capacity: int, every: int = 1):
        """Record (t, min f, argmin, its f_color and additive term, L, kappa,
        varpi) every `every` iterations in a device ring of `capacity`."""
        _ck(self._L.tc_set_trace(self.h, int(capacity), int(every)), "tc_set_trace")

    def tc_get_trace(self):
        """The retained trace records, oldest first, as a list of dicts."""
        n = C.c_int()
        _ck(self._L.tc_get_trace(self.h, None, 0, C.byref(n)), "tc_get_trace")
        buf = (tc_trace_entry * max(1, n.value))()
        _ck(self._L.tc_get_trace(self.h, buf, n.value, C.byref(n)), "tc_get_trace")
        return [{f: getattr(buf[r], f) for f, _ in tc_trace_entry._fields_ if f != "pad"} for r in range(n.value)]

    def tc_set_demands(self, demand):
        """Multicolouring: vertex i takes demand[i] colours (dense forms, k-COL)."""
        dm = np.ascontiguousarray(demand, np.int32)
        _ck(self._L.tc_set_demands(self.h, _ptr(dm), int(dm.size)), "tc_set_demands")
        self.cmax = int(dm.max()) if dm.size else 1

    def tc_best_multi(self):
        """Best-so-far multicolouring: colour sets (n x cmax, -1 padded) and counts."""
        stride = max(1, getattr(self, "cmax", 1))
        col = np.empty((self.n, stride), np.int32)
        fc, t = C.c_int64(), C.c_int64()
        d = C.c_int32()
        _ck(self._L.tc_best_multi(self.h, _ptr(col), stride, C.byref(fc), C.byref(d), C.byref(t)),
            "tc_best_multi")
        return dict(colors=col, conflicts=fc.value, individual=d.value, iteration=t.value)

    def tc_get_multicolors(self):
        """Current colour sets of the population: D x n x cmax, -1 padded."""
        stride = max(1, getattr(self, "cmax", 1))
        col = np.empty((self.D, self.n, stride), np.int32)
        _ck(self._L.tc_get_multicolors(self.h, _ptr(col), stride), "tc_get_multicolors")
        return col

    def tc_launch_count(self) -> int:
        c = C.c_int64()
        _ck(self._L.tc_launch_count(self.h, C.byref(c)), "tc_launch_count")
        return c.value


class TensColBatch:
    """Several contexts (instances of uneven n, k, D) stepped together by one
    CUDA-graph launch per `chunk` iterations (tc_batch_* of the C ABI).  The
    member contexts stay owned by the caller and must outlive the batch."""

    def __init__(self, device: int = 0):
        self._L = load()
        h = C.c_void_p()
        _ck(self._L.tc_batch_create(C.byref(h), device), "tc_batch_create")
        self.h = h
        self.members = []

    def add(self, ctx: "TensCol"):
        _ck(self._L.tc_batch_add(self.h, ctx.h), "tc_batch_add")
        self.members.append(ctx)

    def step(self, n_iters: int, chunk: int = 0):
        _ck(self._L.tc_batch_step(self.h, n_iters, chunk), "tc_batch_step")

    def size(self) -> int:
        c = C.c_int()
        _ck(self._L.tc_batch_size(self.h, C.byref(c)), "tc_batch_size")
        return c.value

    def close(self):
        if getattr(self, "h", None):
            self._L.tc_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
