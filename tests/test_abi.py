"""The C-ABI library loads and exports every entry point include/*.h declares (no GPU)."""
import ctypes
import glob
import os
import re

import pytest

from tests.conftest import ROOT


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(gn_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libgn():
    from paper_2605_05330_gb300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_boundary():
    names = _declared()
    for f in ("gn_create", "gn_run", "gn_extract_is", "gn_objective", "gn_backward", "gn_destroy",
              "gn_last_error"):
        assert f in names


def test_library_exports_every_declared_symbol(libgn):
    missing = [n for n in sorted(_declared()) if not hasattr(libgn, n)]
    assert not missing, missing


def test_binding_defaults(libgn):
    from paper_2605_05330_gb300 import gn
    p = gn.default_params()
    assert p.gamma0 == 0.9 and p.gamma1 == 1.5 and p.ramp_iters == 1000
    assert p.check_every == 10 and abs(p.theta_bin - 1e-4) < 1e-18
    assert gn.lib().gn_last_error() is not None


def test_create_rejects_bad_arguments_on_the_host(libgn):
    """gn_create's argument checks come before any device call, so they run here without a GPU:
    each bad argument gives GN_ERR_ARG, no handle, and a message."""
    P = ctypes.c_void_p

    class Opts(ctypes.Structure):
        _fields_ = [("reorder", ctypes.c_int), ("gather", ctypes.c_int)]

    libgn.gn_create.argtypes = [ctypes.POINTER(P), ctypes.c_int32, P, P, P, ctypes.c_int, ctypes.c_int, P]
    libgn.gn_create.restype = ctypes.c_int
    libgn.gn_create_ex.argtypes = [ctypes.POINTER(P), ctypes.c_int32, P, P, P, ctypes.c_int,
                                   ctypes.POINTER(Opts), P]
    libgn.gn_create_ex.restype = ctypes.c_int
    libgn.gn_last_error.restype = ctypes.c_char_p
    rp = (ctypes.c_int32 * 3)(0, 1, 2)
    ci = (ctypes.c_int32 * 2)(1, 0)
    w = (ctypes.c_float * 2)(1.0, 2.0)
    a = [ctypes.cast(x, P) for x in (rp, ci, w)]
    GN_ERR_ARG = -1
    cases = {
        "n < 0": (-1, a[0], a[1], a[2], 0, 0),
        "n = 2^31 - 1": (2 ** 31 - 1, a[0], a[1], a[2], 0, 0),
        "row_ptr NULL": (2, None, a[1], a[2], 0, 0),
        "w NULL": (2, a[0], a[1], None, 0, 0),
        "bad memory kind": (2, a[0], a[1], a[2], 7, 0),
        "bad reorder": (2, a[0], a[1], a[2], 0, 9),
    }
    for what, (n, r, c, ww, mem, reorder) in cases.items():
        h = P(1234)
        st = libgn.gn_create(ctypes.byref(h), n, r, c, ww, mem, reorder, None)
        assert st == GN_ERR_ARG and not h.value, what
        assert libgn.gn_last_error(), what
    assert libgn.gn_create(None, 2, a[0], a[1], a[2], 0, 0, None) == GN_ERR_ARG
    assert b"NULL" in libgn.gn_last_error()
    h = P(1234)
    st = libgn.gn_create_ex(ctypes.byref(h), 2, a[0], a[1], a[2], 0, ctypes.byref(Opts(0, 99)), None)
    assert st == GN_ERR_ARG and not h.value
    assert b"gather" in libgn.gn_last_error()
    # the batch and the warm-start network check their arguments the same way
    libgn.gn_batch_create.argtypes = [ctypes.POINTER(P), ctypes.c_int32, P, P, P, P, P, P, ctypes.c_int, P]
    libgn.gn_batch_create.restype = ctypes.c_int
    off = ctypes.cast((ctypes.c_int64 * 2)(0, 2), P)
    for what, (count, vo, eo, mem) in {"count < 0": (-1, off, off, 0), "vtx_off NULL": (1, None, off, 0),
                                       "ent_off NULL": (1, off, None, 0), "bad memory kind": (1, off, off, 5)}.items():
        h = P(1234)
        st = libgn.gn_batch_create(ctypes.byref(h), count, vo, eo, a[0], a[1], a[2], None, mem, None)
        assert st == GN_ERR_ARG and not h.value, what
    libgn.gn_mpnn_create.argtypes = [ctypes.POINTER(P), P, P]
    libgn.gn_mpnn_create.restype = ctypes.c_int
    h = P(1234)
    assert libgn.gn_mpnn_create(ctypes.byref(h), None, None) == GN_ERR_ARG and not h.value


def test_null_handles_are_rejected_on_the_host(libgn):
    """Every entry point that takes a handle answers a NULL one with GN_ERR_ARG (the queries with
    0, the destructors with nothing) before any device call, so this runs without a GPU."""
    L, d, f = libgn, ctypes.c_double, ctypes.c_float
    for destroy in (L.gn_destroy, L.gn_batch_destroy, L.gn_mpnn_destroy):
        destroy(None)
    for query in (L.gn_gather_mode, L.gn_halo_exchange, L.gn_num_vertices, L.gn_vertex_order_source):
        assert query(None) == 0
    L.gn_num_entries.restype = ctypes.c_int64
    assert L.gn_num_entries(None) == 0
    calls = {
        "gn_set_io": lambda: L.gn_set_io(None, 0),
        "gn_set_weights": lambda: L.gn_set_weights(None, None),
        "gn_vertex_order": lambda: L.gn_vertex_order(None, None),
        "gn_run": lambda: L.gn_run(None, None, 10, d(1e-7), None, 0, None, None),
        "gn_extract_is": lambda: L.gn_extract_is(None, None, None, None, None, None),
        "gn_objective": lambda: L.gn_objective(None, None, d(1.5), None, None),
        "gn_backward": lambda: L.gn_backward(None, None, None, None),
        "gn_run_noalloc": lambda: L.gn_run_noalloc(-1, None, None, None, None, 10, d(1e-7), None, 0, None, None,
                                                   None),
        "gn_batch_run": lambda: L.gn_batch_run(None, None, 10, d(1e-7), None, None, None),
        "gn_batch_set_threads": lambda: L.gn_batch_set_threads(None, 256),
        "gn_batch_set_packing": lambda: L.gn_batch_set_packing(None, 64),
        "gn_batch_packing": lambda: L.gn_batch_packing(None, None, None),
        "gn_batch_tune": lambda: L.gn_batch_tune(None, None, 10, None),
        "gn_batch_extract": lambda: L.gn_batch_extract(None, None, None, None, None),
        "gn_random_start": lambda: L.gn_random_start(ctypes.c_int64(-1), None, None, None),
        "gn_mpnn_forward": lambda: L.gn_mpnn_forward(None, None, None, None, None),
        "gn_mpnn_predict": lambda: L.gn_mpnn_predict(None, None, f(0.5), None),
        "gn_mpnn_backward": lambda: L.gn_mpnn_backward(None, None),
        "gn_mpnn_zero_grad": lambda: L.gn_mpnn_zero_grad(None),
        "gn_mpnn_step": lambda: L.gn_mpnn_step(None, f(1e-3)),
        "gn_mpnn_get_params": lambda: L.gn_mpnn_get_params(None, None),
        "gn_mpnn_get_grads": lambda: L.gn_mpnn_get_grads(None, None),
    }
    wrong = {name: st for name, st in ((name, call()) for name, call in calls.items()) if st != -1}
    assert not wrong, wrong


def test_oracle_is_not_imported_by_the_product():
    """The product path (package, bench CUDA leg) never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2605_05330_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.py"), recursive=True):
        src = open(path).read()
        assert "import oracle" not in src and "from oracle" not in src, path
