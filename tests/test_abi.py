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


def test_oracle_is_not_imported_by_the_product():
    """The product path (package, bench CUDA leg) never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2605_05330_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.py"), recursive=True):
        src = open(path).read()
        assert "import oracle" not in src and "from oracle" not in src, path
