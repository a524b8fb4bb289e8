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


def _call(torch, gn, L, n, rp, ci, w, x0, max_iters, tol, params, start_iter, x):
    P = ctypes.c_void_p
    info = gn.RunInfo()
    st = L.gn_run_noalloc(n, P(rp.data_ptr()), P(ci.data_ptr()) if ci is not None else None, P(w.data_ptr()),
                          P(x0.data_ptr()) if x0 is not None else None, max_iters, tol, ctypes.byref(params),
                          start_iter, P(x.data_ptr()), ctypes.byref(info), None)
    torch.cuda.synchronize()
    return gn.STATUS[st], info


def test_noalloc_start_state_and_resumed_runs(env):
    """A caller's x0 (with a zero entry that a positive neighbour makes normalizable, Def. 1)
    and a run that starts at start_iter > 0 from a saved FP32 state: both as gn_run on a
    GN_GATHER_GLOBAL handle."""
    torch, gn, L = env
    inst = inputs.er_graph(4000, 8.0, 4331)
    dev = torch.device("cuda", 0)
    rp = torch.from_numpy(inst.row_ptr).to(dev)
    ci = torch.from_numpy(inst.col_idx).to(dev)
    w = torch.from_numpy(inst.w).to(dev)
    x0 = torch.from_numpy(inputs.uniforms(inst.n, 4332)).to(dev)
    x0[3] = 0.0
    assert int(inst.row_ptr[4] - inst.row_ptr[3]) > 0
    g = gn.Graph(rp, ci, w, gather=gn.GATHER_GLOBAL)
    pk = gn.default_params(theta_bin=-1.0, check_every=1)
    x = torch.empty(inst.n, dtype=torch.float32, device=dev)
    st, info = _call(torch, gn, L, inst.n, rp, ci, w, x0, 20, -1.0, pk, 0, x)
    xr, ir = g.run(x0=x0, max_iters=20, tol=-1.0, params=pk)
    assert st == ir["status"] and info.iters == ir["iters"] == 20
    xn, xrn = x.cpu().numpy().astype(np.float64), xr.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(xn - xrn) <= REL * np.maximum(np.abs(xrn), FLOOR))
    # resume from the 300-step state at start_iter = 300, to a binary state
    xs, _ = g.run(max_iters=300, tol=-1.0)
    xs = xs.clone()
    st, info = _call(torch, gn, L, inst.n, rp, ci, w, xs, 2000, 1e-7, gn.default_params(), 300, x)
    xr, ir = g.run(x0=xs, max_iters=2000, start_iter=300)
    assert st == ir["status"] == "OK" and info.iters == ir["iters"]
    assert np.array_equal(x.cpu().numpy() > 0.5, xr.cpu().numpy() > 0.5)
    g.close()


def test_noalloc_rejects_bad_inputs_and_leaves_the_output(env):
    """Weights that are not positive and finite (GN_ERR_WEIGHT), a CSR that is not simple
    (asymmetric, or with a self-loop: GN_ERR_NOT_SIMPLE), a row_ptr that decreases further on
    (GN_ERR_ARG, the rows are bounded by row_ptr[n] before their entries are read) and a wait
    that times out (GN_ERR_TIMEOUT, through the test hook that makes the first grid barrier
    unreachable): each returns its status, leaves x_out as it was, and the next call works."""
    torch, gn, L = env
    dev = torch.device("cuda", 0)
    inst = inputs.er_graph(3000, 6.0, 4341)
    rp = torch.from_numpy(inst.row_ptr).to(dev)
    ci = torch.from_numpy(inst.col_idx).to(dev)
    w = torch.from_numpy(inst.w).to(dev)
    p = gn.default_params()
    x = torch.full((inst.n,), 7.0, dtype=torch.float32, device=dev)

    def untouched():
        return bool(torch.all(x == 7.0).item())

    for bad in (0.0, -1.0, float("inf"), float("nan")):
        wb = w.clone()
        wb[5] = bad
        st, _ = _call(torch, gn, L, inst.n, rp, ci, wb, None, 100, 1e-7, p, 0, x)
        assert st == "ERR_WEIGHT" and untouched()
    # asymmetric: drop one direction of an edge; self-loop: a row that lists itself
    tiny_rp = torch.tensor([0, 1, 1], dtype=torch.int32, device=dev)
    tiny_ci = torch.tensor([1], dtype=torch.int32, device=dev)
    tiny_w = torch.ones(2, dtype=torch.float32, device=dev)
    x2 = torch.full((2,), 7.0, dtype=torch.float32, device=dev)
    st, _ = _call(torch, gn, L, 2, tiny_rp, tiny_ci, tiny_w, None, 10, 1e-7, p, 0, x2)
    assert st == "ERR_NOT_SIMPLE" and bool(torch.all(x2 == 7.0).item())
    loop_rp = torch.tensor([0, 1, 2], dtype=torch.int32, device=dev)
    loop_ci = torch.tensor([0, 1], dtype=torch.int32, device=dev)
    st, _ = _call(torch, gn, L, 2, loop_rp, loop_ci, tiny_w, None, 10, 1e-7, p, 0, x2)
    assert st == "ERR_NOT_SIMPLE" and bool(torch.all(x2 == 7.0).item())
    # row 0 claims [0, 2^30) although row_ptr[n] = 10 and col_idx holds 10 entries
    dec_rp = torch.tensor([0, 1 << 30, 10], dtype=torch.int32, device=dev)
    dec_ci = torch.ones(10, dtype=torch.int32, device=dev)
    st, _ = _call(torch, gn, L, 2, dec_rp, dec_ci, tiny_w, None, 10, 1e-7, p, 0, x2)
    assert st == "ERR_ARG" and bool(torch.all(x2 == 7.0).item())
    # a barrier nothing can satisfy: bounded wait, status returned, context usable
    pt = gn.default_params(debug_unreachable_barrier=1, spin_limit=2000)
    st, _ = _call(torch, gn, L, inst.n, rp, ci, w, None, 100, 1e-7, pt, 0, x)
    assert st == "ERR_TIMEOUT" and untouched()
    st, info = _call(torch, gn, L, inst.n, rp, ci, w, None, 2000, 1e-7, p, 0, x)
    assert st == "OK" and info.iters > 0 and bool(torch.all((x >= 0) & (x <= 1)).item())
