"""FP64 CPU oracle for Graph Normalization -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library
(``paper_2605_05330_gb300``) and never imports it.

The arithmetic lives in ``gn_oracle.c`` (plain sequential C, FP64, x-space,
following Def. WRGN, Sec. 6 and the appendix module of arXiv 2605.05330).
This module is argument marshalling for it (ctypes + numpy), plus the FP64
reference forms in ``grad.py`` (unrolled-GN gradients) and ``mpnn.py``
(message-passing warm-start network).

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
against closed forms, worked examples, theorems and brute force, except where
a docstring says "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gn_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

# oracle-local status values (mirror of gn_oracle.h; names match the CUDA library's)
STATUS = {
    0: "OK",
    1: "WARN_NOT_CONVERGED",
    2: "WARN_NOT_BINARY",
    3: "WARN_NOT_MAXIMAL",
    -1: "ERR_ARG",
    -2: "ERR_NOT_SIMPLE",
    -3: "ERR_WEIGHT",
    -4: "ERR_NOT_NORMALIZABLE",
    -7: "ERR_NOT_INDEPENDENT",
}
GAMMA_PURSUIT = 0
GAMMA_FIXED = 1


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (no FMA contraction: identical on x86 and Arm)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "gn_oracle.h"))
    ):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [("gamma_mode", ctypes.c_int), ("gamma0", ctypes.c_double),
                ("gamma1", ctypes.c_double), ("ramp_iters", ctypes.c_int),
                ("check_every", ctypes.c_int), ("theta_bin", ctypes.c_double)]


class _Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int), ("binary", ctypes.c_int),
                ("status", ctypes.c_int), ("resid_inf", ctypes.c_double),
                ("resid_l1", ctypes.c_double), ("objective", ctypes.c_double),
                ("energy", ctypes.c_double), ("safe_div_hits", ctypes.c_longlong)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        lib.gno_validate.argtypes = [ctypes.c_int, P, P, P]
        lib.gno_validate.restype = ctypes.c_int
        lib.gno_gamma.argtypes = [ctypes.POINTER(_Params), ctypes.c_int]
        lib.gno_gamma.restype = ctypes.c_double
        lib.gno_step.argtypes = [ctypes.c_int, P, P, P, ctypes.c_double, P, P, P]
        lib.gno_step.restype = None
        lib.gno_run.argtypes = [ctypes.c_int, P, P, P, P, ctypes.c_int, ctypes.c_double,
                                ctypes.POINTER(_Params), ctypes.c_int, P, ctypes.POINTER(_Info),
                                P, P, ctypes.c_int]
        lib.gno_run.restype = ctypes.c_int
        lib.gno_objective.argtypes = [ctypes.c_int, P, P]
        lib.gno_objective.restype = ctypes.c_double
        lib.gno_energy.argtypes = [ctypes.c_int, P, P, P, ctypes.c_double, P]
        lib.gno_energy.restype = ctypes.c_double
        lib.gno_extract_is.argtypes = [ctypes.c_int, P, P, P, P, P, P, P, P]
        lib.gno_extract_is.restype = ctypes.c_int
        lib.gno_stability.argtypes = [ctypes.c_int, P, P, P, ctypes.c_double, P]
        lib.gno_stability.restype = ctypes.c_double
        lib.gno_mwis_enumerate.argtypes = [ctypes.c_int, P, P, P, ctypes.c_double, ctypes.c_int,
                                           P, P, P]
        lib.gno_mwis_enumerate.restype = ctypes.c_int
        lib.gno_hungarian.argtypes = [ctypes.c_int, P, P]
        lib.gno_hungarian.restype = ctypes.c_double
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _csr(row_ptr, col_idx):
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    if ci.size == 0:
        ci = np.zeros(1, dtype=np.int32)  # valid pointer for an edgeless graph
    return rp, ci


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def params(gamma_mode=GAMMA_PURSUIT, gamma0=0.9, gamma1=1.5, ramp_iters=1000, check_every=1,
           theta_bin=1e-4) -> _Params:
    """Run parameters.  Defaults: the paper's pursuit 0.9 -> 1.5 over 1000 iterations (Sec. 6)."""
    return _Params(gamma_mode, gamma0, gamma1, ramp_iters, check_every, theta_bin)


def validate(row_ptr, col_idx, w) -> str:
    rp, ci = _csr(row_ptr, col_idx)
    return STATUS[_load().gno_validate(len(rp) - 1, _p(rp), _p(ci), _p(_f64(w)))]


def gamma(p: _Params, k: int) -> float:
    return _load().gno_gamma(ctypes.byref(p), k)


def step(row_ptr, col_idx, w, gamma_value, x):
    """One WRGN step (Def. WRGN) in FP64; returns (x_next, safe_div_hits)."""
    rp, ci = _csr(row_ptr, col_idx)
    n = len(rp) - 1
    v = np.sqrt(_f64(w))
    x = _f64(x)
    xn = np.empty(n, dtype=np.float64)
    hits = ctypes.c_longlong(0)
    _load().gno_step(n, _p(rp), _p(ci), _p(v), float(gamma_value), _p(x), _p(xn),
                     ctypes.cast(ctypes.pointer(hits), ctypes.c_void_p))
    return xn, int(hits.value)


def run(row_ptr, col_idx, w, x0=None, max_iters=2000, tol=1e-7, p: _Params | None = None,
        start_iter=0, trace_len=0):
    """Iterated WRGN with the stop test; returns (x, info dict[, trace_obj, trace_energy])."""
    rp, ci = _csr(row_ptr, col_idx)
    n = len(rp) - 1
    p = p if p is not None else params()
    x_out = np.empty(max(n, 1), dtype=np.float64)
    x0a = _f64(x0) if x0 is not None else None
    info = _Info()
    tobj = np.zeros(trace_len, dtype=np.float64) if trace_len else None
    ten = np.zeros(trace_len, dtype=np.float64) if trace_len else None
    st = _load().gno_run(n, _p(rp), _p(ci), _p(_f64(w)), _p(x0a), int(max_iters), float(tol),
                         ctypes.byref(p), int(start_iter), _p(x_out), ctypes.byref(info),
                         _p(tobj), _p(ten), int(trace_len))
    d = {f: getattr(info, f) for f, _ in _Info._fields_}
    d["status"] = STATUS[st]
    if trace_len:
        return x_out[:n], d, tobj, ten
    return x_out[:n], d


def objective(w, x) -> float:
    w = _f64(w)
    return _load().gno_objective(len(w), _p(w), _p(_f64(x)))


def energy(row_ptr, col_idx, w, gamma_value, x) -> float:
    rp, ci = _csr(row_ptr, col_idx)
    return _load().gno_energy(len(rp) - 1, _p(rp), _p(ci), _p(_f64(w)), float(gamma_value),
                              _p(_f64(x)))


def extract_is(row_ptr, col_idx, w, x):
    """Round at 1/2, check independence and maximality; returns (status, mask, members, W)."""
    rp, ci = _csr(row_ptr, col_idx)
    n = len(rp) - 1
    mask = np.zeros(max(n, 1), dtype=np.uint8)
    members = np.zeros(max(n, 1), dtype=np.int32)
    count = ctypes.c_int32(0)
    weight = ctypes.c_double(0.0)
    st = _load().gno_extract_is(n, _p(rp), _p(ci), _p(_f64(w)), _p(_f64(x)), _p(mask),
                                _p(members), ctypes.cast(ctypes.pointer(count), ctypes.c_void_p),
                                ctypes.cast(ctypes.pointer(weight), ctypes.c_void_p))
    return STATUS[st], mask[:n], members[: count.value], weight.value


def stability(row_ptr, col_idx, w, gamma_value, mask) -> float:
    rp, ci = _csr(row_ptr, col_idx)
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    return _load().gno_stability(len(rp) - 1, _p(rp), _p(ci), _p(_f64(w)), float(gamma_value),
                                 _p(m))


def mwis_enumerate(row_ptr, col_idx, w, rel_tol=1e-12, max_out=64):
    """Brute-force MWIS (n <= 31): returns (W*, list of maximiser masks as bool arrays)."""
    rp, ci = _csr(row_ptr, col_idx)
    n = len(rp) - 1
    out = np.zeros(max_out, dtype=np.uint32)
    nb = ctypes.c_int(0)
    best = ctypes.c_double(0.0)
    st = _load().gno_mwis_enumerate(n, _p(rp), _p(ci), _p(_f64(w)), float(rel_tol), max_out,
                                    _p(out), ctypes.cast(ctypes.pointer(nb), ctypes.c_void_p),
                                    ctypes.cast(ctypes.pointer(best), ctypes.c_void_p))
    if st != 0:
        raise ValueError(STATUS[st])
    masks = [np.array([(int(m) >> i) & 1 for i in range(n)], dtype=bool)
             for m in out[: min(nb.value, max_out)]]
    return best.value, masks


def hungarian(cost):
    """Min-cost assignment of a k x k matrix; returns (total, assign[row] = col)."""
    c = _f64(cost)
    k = c.shape[0]
    assign = np.zeros(k, dtype=np.int32)
    total = _load().gno_hungarian(k, _p(c), _p(assign))
    return total, assign


def random_start(u):
    """The appendix module's random simplex start, FP64: p = -log u; p / max(p) over all draws;
    clamp to [1e-3, 1].  (Pinned: exponential draws divided by their maximum lie in (0, 1], and
    the clamp is the module's.)"""
    p = -np.log(np.asarray(u, dtype=np.float64))
    p = p / p.max()
    return np.clip(p, 1e-3, 1.0)
