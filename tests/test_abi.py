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


def test_oracle_is_not_imported_by_the_product():
    """The product path (package, bench CUDA leg) never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2605_05330_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.py"), recursive=True):
        src = open(path).read()
        assert "import oracle" not in src and "from oracle" not in src, path
