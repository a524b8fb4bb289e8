"""Everything a run reports besides the iterate, against the FP64 oracle, through the C ABI.

* After k in {1, 5, 20} fixed steps: the L-inf and L1 residuals of x^{k+1} - x^k (the stop
  test), the objective sum w x (Thm. 3), the energy E~ of the state entering the last step at
  that step's gamma (Sec. 3) and the safe-division count (the appendix module's mask).  The
  bounds follow from the per-vertex iterate bar |x_gpu - x_oracle| <= 1e-5 max(|x|, 1e-6) plus
  the FP32 rounding of each per-row term (the kernel forms terms in FP32 and accumulates them in
  float pairs, about 2^-44 relative per addition, far below one FP32 rounding of a term).
* gn_objective called on the library directly (ctypes, host buffers): its FP64 objective and
  energy against gno_objective / gno_energy on the same FP32 state.
* gn_extract_is on a dependent set and on a non-maximal set (Sec. 2): the oracle's statuses
  and masks.
* The safe division (d <= 1e-9 sets x = 1/2) on a start whose denominators all fall below the
  threshold, and mixed with a component that never reaches it.
* Instances on which an own state limited to FP32's exponent range ends differently from the
  FP64 run (more safe-division hits, another iteration count or other members; non-members
  that decay below 2^-126 and would later come back): the GPU's hits, iterations and set are
  the oracle's, in every kernel that runs whole runs.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2605_05330_gb300 import inputs
from tests.test_gpu_parity import FLOOR, GATHERS, K_ITERATE, REL, _tie_free, assert_close_rel, dev_graph, fixed_steps, to_np

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24


@pytest.fixture(scope="module")
def gn():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_05330_gb300 import build
    build.build()
    from paper_2605_05330_gb300 import gn as gnmod
    return gnmod


INSTANCES = {
    "er2000": lambda: inputs.workload_er_small(),
    "udg20k": lambda: inputs.unit_disk_graph(20000, 100000, 1240),
    "ba20k": lambda: inputs.ba_graph(20000, 5, 1241),
    "assign24": lambda: inputs.assignment_graph(24, 1242),
}


def _d_x(inst, gamma, x):
    """x-space denominators d_i = x_i + gamma sum_j sqrt(w_j / w_i) x_j (for error bounds only)."""
    w = inst.w.astype(np.float64)
    deg = np.diff(inst.row_ptr)
    rows = np.repeat(np.arange(inst.n), deg)
    nb = np.zeros(inst.n)
    np.add.at(nb, rows, np.sqrt(w[inst.col_idx]) * x[inst.col_idx])
    return x + gamma * nb / np.sqrt(w)


@pytest.mark.parametrize("gather", ["halo", "global"])
@pytest.mark.parametrize("k", [1, 5, K_ITERATE])
@pytest.mark.parametrize("which", list(INSTANCES))
def test_reported_scalars_match_oracle(gn, which, k, gather):
    inst = INSTANCES[which]()
    g = dev_graph(gn, inst, gather=GATHERS[gather])
    run_kw, pk = fixed_steps(k)
    x, info = g.run(params=gn.default_params(**pk), **run_kw)
    xo, io = oracle.run(inst.row_ptr, inst.col_idx, inst.w, p=oracle.params(**pk), **run_kw)
    # the state entering the last step, from the oracle
    if k == 1:
        xp = 1.0 / (np.diff(inst.row_ptr) + 1.0)
    else:
        xp, _ = oracle.run(inst.row_ptr, inst.col_idx, inst.w, p=oracle.params(**pk), max_iters=k - 1, tol=-1.0)
    assert_close_rel(to_np(x), xo)
    assert info["iters"] == io["iters"] == k
    assert info["safe_div_hits"] == io["safe_div_hits"]
    m = np.maximum(np.abs(xo), FLOOR) + np.maximum(np.abs(xp), FLOOR)
    # L-inf residual: both values within the iterate bar, the difference rounded once
    assert abs(info["resid_inf"] - io["resid_inf"]) <= REL * m.max() + 2 * EPS32 * max(io["resid_inf"], 1e-30)
    # L1 residual: the sum of the same per-row bounds
    assert abs(info["resid_l1"] - io["resid_l1"]) <= REL * m.sum() + 2 * EPS32 * io["resid_l1"]
    w = inst.w.astype(np.float64)
    # objective: the iterate bar on w x', then the FP32 product and the per-thread FP32 additions
    ob = REL * np.sum(w * np.maximum(xo, FLOOR)) + 16 * EPS32 * io["objective"]
    assert abs(info["objective"] - io["objective"]) <= ob
    # energy: term_i = w x (d_x / 2 - 1); each factor within the iterate bar (d through the
    # neighbours' x), then FP32 roundings of y, d, v and of the per-thread additions
    gam = oracle.gamma(oracle.params(**pk), k - 1)
    d = _d_x(inst, gam, xp)
    scale = np.sum(w * xp * (0.5 * d + 1.0))
    assert abs(info["energy"] - io["energy"]) <= (2 * REL + 24 * EPS32) * scale


def _abi(gn):
    L = gn.lib()
    return L, ctypes.c_void_p


@pytest.mark.parametrize("which", ["er2000", "ba20k", "assign24"])
def test_objective_through_the_c_abi(gn, which):
    """gn_create (GN_HOST) and gn_objective on host buffers, without the binding's classes."""
    inst = INSTANCES[which]()
    L, P = _abi(gn)
    h = P()
    rp = np.ascontiguousarray(inst.row_ptr, np.int32)
    ci = np.ascontiguousarray(inst.col_idx, np.int32)
    w = np.ascontiguousarray(inst.w, np.float32)
    st = L.gn_create(ctypes.byref(h), inst.n, rp.ctypes.data_as(P), ci.ctypes.data_as(P), w.ctypes.data_as(P),
                     gn.HOST, 0, None)
    assert st == 0, L.gn_last_error()
    try:
        rng = np.random.default_rng(31)
        states = [(1.0 / (np.diff(rp) + 1.0)).astype(np.float32), rng.random(inst.n).astype(np.float32)]
        for xs in states:
            for gam in (0.9, 1.5):
                o = ctypes.c_double()
                e = ctypes.c_double()
                st = L.gn_objective(h, xs.ctypes.data_as(P), gam, ctypes.cast(ctypes.pointer(o), P),
                                    ctypes.cast(ctypes.pointer(e), P))
                assert st == 0, L.gn_last_error()
                x64 = xs.astype(np.float64)
                oo = oracle.objective(inst.w, x64)
                eo = oracle.energy(inst.row_ptr, inst.col_idx, inst.w, gam, x64)
                # both FP64 on the same FP32 state; v from its float pair (2^-48) on the GPU
                wd = inst.w.astype(np.float64)
                scale = np.sum(wd * x64 * (0.5 * _d_x(inst, gam, x64) + 1.0))
                assert abs(o.value - oo) <= 1e-13 * oo
                assert abs(e.value - eo) <= 1e-12 * scale
        # NULL state: the state left by the last run (here after 7 fixed steps)
        p = gn.default_params(theta_bin=-1.0, check_every=1)
        xr = np.empty(inst.n, np.float32)
        info = gn.RunInfo()
        st = L.gn_run(h, None, 7, -1.0, ctypes.byref(p), 0, xr.ctypes.data_as(P), ctypes.byref(info))
        assert st >= 0, L.gn_last_error()
        o = ctypes.c_double()
        st = L.gn_objective(h, None, 1.5, ctypes.cast(ctypes.pointer(o), P), None)
        assert st == 0
        assert abs(o.value - oracle.objective(inst.w, xr.astype(np.float64))) <= 1e-13 * o.value
    finally:
        L.gn_destroy(h)


def test_extract_failure_branches(gn):
    """A state whose rounding has an edge inside S (GN_ERR_NOT_INDEPENDENT) and one whose
    rounding leaves a vertex with no neighbour in S (GN_WARN_NOT_MAXIMAL): statuses, masks,
    counts and W(S) as the oracle's, through the C ABI with host buffers."""
    inst = inputs.er_graph(3000, 8.0, 1501)
    L, P = _abi(gn)
    h = P()
    rp = np.ascontiguousarray(inst.row_ptr, np.int32)
    ci = np.ascontiguousarray(inst.col_idx, np.int32)
    w = np.ascontiguousarray(inst.w, np.float32)
    assert L.gn_create(ctypes.byref(h), inst.n, rp.ctypes.data_as(P), ci.ctypes.data_as(P), w.ctypes.data_as(P),
                       gn.HOST, 0, None) == 0
    try:
        # a maximal independent set from the oracle's run, then two damaged copies
        xo, _ = oracle.run(inst.row_ptr, inst.col_idx, inst.w, p=oracle.params(check_every=10))
        base = (xo > 0.5).astype(np.float32)
        i = int(np.nonzero(base > 0.5)[0][0])
        j = int(ci[rp[i]])                      # a neighbour of a member: not a member
        dep = base.copy()
        dep[j] = 0.75                           # now an edge i-j inside S
        nonmax = base.copy()
        nonmax[i] = 0.5                         # exactly 1/2 rounds out: i and maybe others uncovered
        cases = {"OK": base, "ERR_NOT_INDEPENDENT": dep, "WARN_NOT_MAXIMAL": nonmax}
        for want, xs in cases.items():
            mask = np.zeros(inst.n, np.uint8)
            mem = np.zeros(inst.n, np.int32)
            cnt = ctypes.c_int32()
            wt = ctypes.c_double()
            st = L.gn_extract_is(h, xs.ctypes.data_as(P), mask.ctypes.data_as(P), mem.ctypes.data_as(P),
                                 ctypes.cast(ctypes.pointer(cnt), P), ctypes.cast(ctypes.pointer(wt), P))
            sto, masko, memo, Wo = oracle.extract_is(inst.row_ptr, inst.col_idx, inst.w, xs.astype(np.float64))
            assert sto == want
            assert gn.STATUS[st] == sto
            np.testing.assert_array_equal(mask, masko)
            assert cnt.value == len(memo)
            np.testing.assert_array_equal(mem[: cnt.value], memo)
            assert wt.value == pytest.approx(Wo, rel=1e-14)
    finally:
        L.gn_destroy(h)


@pytest.mark.parametrize("gather", ["halo", "global"])
def test_safe_division_matches_oracle(gn, gather):
    """x0 = 1e-12 on a weighted path P4: every denominator (B y)_i is below 1e-9 at the first
    step, so every vertex is set to 1/2 and counted; a second component with an ordinary start
    never reaches the threshold.  Iterates and hit counts against the oracle for k in {1, 2, 5}."""
    p4 = inputs.small_graph("P4", 4, [(0, 1), (1, 2), (2, 3)], w=[3.0, 1.0, 2.0, 5.0])
    er = inputs.er_graph(400, 6.0, 1502)
    inst = inputs.disjoint_union([p4, er])
    x0 = np.concatenate([np.full(4, 1e-12), 1.0 / (np.diff(er.row_ptr) + 1.0)]).astype(np.float32)
    g = dev_graph(gn, inst, gather=GATHERS[gather])
    import torch
    for k in (1, 2, 5):
        run_kw, pk = fixed_steps(k)
        x, info = g.run(x0=torch.from_numpy(x0).cuda(), params=gn.default_params(**pk), **run_kw)
        xo, io = oracle.run(inst.row_ptr, inst.col_idx, inst.w, x0=x0.astype(np.float64), p=oracle.params(**pk),
                            **run_kw)
        assert io["safe_div_hits"] >= 4
        assert info["safe_div_hits"] == io["safe_div_hits"]
        assert_close_rel(to_np(x), xo)
        if k == 1:
            np.testing.assert_array_equal(to_np(x)[:4], np.full(4, 0.5, np.float32))


# unit-disk, ER and BA instances (seeded; all tie-free) on which the run's outcome depends on
# keeping deeply decayed states: with FP32's exponent range each of them ends with more
# safe-division hits, another iteration count or other members than the FP64 run
DEEP = {
    "udg5k_s2009": lambda: inputs.unit_disk_graph(5000, 25000, 2009),
    "udg5k_s2001": lambda: inputs.unit_disk_graph(5000, 25000, 2001),
    "er3k_s2011": lambda: inputs.er_graph(3000, 10.0, 2011),
    "er3k_s2016": lambda: inputs.er_graph(3000, 10.0, 2016),
    "ba5k_s2026": lambda: inputs.ba_graph(5000, 4, 2026),
}


@pytest.mark.parametrize("which", list(DEEP))
def test_deep_decay_follows_oracle(gn, which):
    inst = DEEP[which]()
    p = dict(check_every=10)
    xo, io = oracle.run(inst.row_ptr, inst.col_idx, inst.w, max_iters=2000, tol=1e-7, p=oracle.params(**p))
    set_o = oracle.extract_is(inst.row_ptr, inst.col_idx, inst.w, xo)[1]
    assert io["status"] == "OK"
    assert _tie_free(inst, oracle.params(**p))
    runs = []
    for gather in ("halo", "global"):
        g = dev_graph(gn, inst, gather=GATHERS[gather])
        runs.append((gather, g, gn.default_params(**p)))
    runs.append(("cta", runs[0][1], gn.default_params(kernel=gn.KERNEL_CTA, **p)))
    for name, g, prm in runs:
        x, info = g.run(max_iters=2000, tol=1e-7, params=prm)
        st, mask, members, cnt, W = g.extract_is()
        assert (name, info["safe_div_hits"], info["iters"]) == (name, io["safe_div_hits"], io["iters"])
        np.testing.assert_array_equal(to_np(mask), set_o)
    # the batched form on the same instances
    b = gn.Batch([inst])
    xb, infos = b.run(max_iters=2000, tol=1e-7, params=gn.default_params(**p))
    assert infos[0]["safe_div_hits"] == io["safe_div_hits"] and infos[0]["iters"] == io["iters"]
    np.testing.assert_array_equal(np.asarray(xb) > 0.5, set_o.astype(bool))


@pytest.mark.parametrize("which", ["udg20k_rcm", "ba20k_s1295", "er3k_s2011"])
def test_host_pipeline_through_the_c_abi(gn, which):
    """The path a caller with host data takes (the one the end-to-end bench times): gn_create
    from host CSR buffers, gn_run to a binary state with the default synchronisation, the state
    back in a host buffer, gn_extract_is into host buffers, gn_destroy, without the binding's
    classes.  Against the oracle's run to the same stop: the same iteration count and safe-division
    hits, an independent set (checked by the oracle) and, on a tie-free instance, the oracle's
    set and weight."""
    inst, reorder = {"udg20k_rcm": lambda: (inputs.unit_disk_graph(20000, 100000, 1294), 1),
                     "ba20k_s1295": lambda: (inputs.ba_graph(20000, 5, 1295), 0),
                     "er3k_s2011": lambda: (inputs.er_graph(3000, 9.0, 2011), 0)}[which]()
    L, P = _abi(gn)
    rp = np.ascontiguousarray(inst.row_ptr, np.int32)
    ci = np.ascontiguousarray(inst.col_idx, np.int32)
    w = np.ascontiguousarray(inst.w, np.float32)
    h = P()
    st = L.gn_create(ctypes.byref(h), inst.n, rp.ctypes.data_as(P), ci.ctypes.data_as(P), w.ctypes.data_as(P),
                     gn.HOST, reorder, None)
    assert st == 0, L.gn_last_error()
    try:
        x = np.empty(inst.n, np.float32)
        info = gn.RunInfo()
        p = gn.default_params()
        st = L.gn_run(h, None, 2000, 1e-7, ctypes.byref(p), 0, x.ctypes.data_as(P), ctypes.byref(info))
        assert st == 0, L.gn_last_error()
        mask = np.empty(inst.n, np.uint8)
        members = np.empty(inst.n, np.int32)
        cnt = ctypes.c_int32()
        wt = ctypes.c_double()
        st = L.gn_extract_is(h, None, mask.ctypes.data_as(P), members.ctypes.data_as(P),
                             ctypes.cast(ctypes.pointer(cnt), P), ctypes.cast(ctypes.pointer(wt), P))
        assert st >= 0, L.gn_last_error()
    finally:
        L.gn_destroy(h)
    po = oracle.params(check_every=10)  # the library's default cadence of the stop test
    xo, io = oracle.run(inst.row_ptr, inst.col_idx, inst.w, max_iters=2000, tol=1e-7, p=po)
    assert info.iters == io["iters"]
    assert info.safe_div_hits == io["safe_div_hits"]
    # the GPU's set, judged by the oracle's exact check of the same state
    sto, masko_of_gpu, _, wo_of_gpu = oracle.extract_is(inst.row_ptr, inst.col_idx, inst.w, x.astype(np.float64))
    assert sto in ("OK", "WARN_NOT_MAXIMAL")
    np.testing.assert_array_equal(mask.astype(bool), np.asarray(masko_of_gpu).astype(bool))
    assert sorted(members[:cnt.value].tolist()) == np.nonzero(mask)[0].tolist()
    assert abs(wt.value - wo_of_gpu) <= 1e-12 * max(1.0, wo_of_gpu)
    if _tie_free(inst, po):
        _, masko, _, wo = oracle.extract_is(inst.row_ptr, inst.col_idx, inst.w, xo)
        np.testing.assert_array_equal(mask.astype(bool), np.asarray(masko).astype(bool))
        assert abs(wt.value - wo) <= 1e-9 * wo
