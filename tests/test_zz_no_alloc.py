"""gn_run_noalloc: the allocation-free variant of the iteration, for callers that may not call
cudaMalloc (they are handed device buffers by a host runtime that owns all allocation).  Its
scratch lives in a fixed array in the library's device globals.

Checked through the C ABI: two calls in a row (a larger graph, then a smaller one, so that the
second call starts from the first call's leftovers in the shared array) each agree with
gn_run, the allocating entry point, within the per-vertex tolerance of the parity tests, and a
graph above the fixed limit is rejected.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2605_05330_gb300 import inputs

pytestmark = pytest.mark.gpu

REL = 1e-5
FLOOR = 1e-6


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_05330_gb300 import build
    build.build()
    from paper_2605_05330_gb300 import gn
    L = gn.lib()
    P = ctypes.c_void_p
    L.gn_run_noalloc.argtypes = [ctypes.c_int32, P, P, P, P, ctypes.c_int, ctypes.c_double,
                                 ctypes.POINTER(gn.Params), ctypes.c_int, P, ctypes.POINTER(gn.RunInfo), P]
    L.gn_run_noalloc.restype = ctypes.c_int
    return torch, gn, L


def _noalloc(torch, gn, L, inst, max_iters, tol, params):
    dev = torch.device("cuda", 0)
    rp = torch.from_numpy(inst.row_ptr).to(dev)
    ci = torch.from_numpy(inst.col_idx).to(dev)
    w = torch.from_numpy(inst.w).to(dev)
    x = torch.empty(inst.n, dtype=torch.float32, device=dev)
    info = gn.RunInfo()
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    P = ctypes.c_void_p
    st = L.gn_run_noalloc(inst.n, P(rp.data_ptr()), P(ci.data_ptr()), P(w.data_ptr()), None, max_iters, tol,
                          ctypes.byref(params), 0, P(x.data_ptr()), ctypes.byref(info), stream)
    torch.cuda.synchronize()
    return st, x.cpu().numpy(), info


def _reference(gn, inst, max_iters, tol, params):
    # the allocating entry point with the same gather mode (neighbour values through L1/L2)
    g = gn.Graph(inst.row_ptr, inst.col_idx, inst.w, gather=gn.GATHER_GLOBAL)
    x, info = g.run(max_iters=max_iters, tol=tol, params=params)
    g.close()
    return x, info


def test_noalloc_matches_gn_run_on_two_calls_in_a_row(env):
    torch, gn, L = env
    cases = [(inputs.er_graph(60000, 10.0, 4321), 2000, 1e-7, gn.default_params()),
             (inputs.ba_graph(5000, 4, 4322), 40, -1.0, gn.default_params(theta_bin=-1.0, check_every=1))]
    for inst, max_iters, tol, p in cases:
        st, x, info = _noalloc(torch, gn, L, inst, max_iters, tol, p)
        assert st >= 0, L.gn_last_error()
        xr, ir = _reference(gn, inst, max_iters, tol, p)
        assert gn.STATUS[st] == ir["status"]
        assert info.iters == ir["iters"]
        err = np.abs(x.astype(np.float64) - xr)
        assert np.all(err <= REL * np.maximum(np.abs(xr.astype(np.float64)), FLOOR))
        assert np.array_equal(x > 0.5, xr > 0.5)
        assert abs(info.objective - ir["objective"]) <= 1e-9 * abs(ir["objective"])


def test_noalloc_rejects_graphs_above_its_limit(env):
    torch, gn, L = env
    n = 65537
    rp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    w = torch.ones(n, dtype=torch.float32, device="cuda")
    x = torch.empty(n, dtype=torch.float32, device="cuda")
    P = ctypes.c_void_p
    p = gn.default_params()
    st = L.gn_run_noalloc(n, P(rp.data_ptr()), None, P(w.data_ptr()), None, 100, 1e-7, ctypes.byref(p), 0,
                          P(x.data_ptr()), None, None)
    assert gn.STATUS[st] == "ERR_TOO_LARGE"
    assert b"65536" in L.gn_last_error()
