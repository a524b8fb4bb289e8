"""Batched GN against the FP64 oracle (per instance) and against the single-graph path.

The batch path runs the same per-vertex arithmetic as gn_run: CSR instances use the same
lanes-per-row split and summation order as gn_run's global-gather mode, so their iterates are
bit-identical to it; assignment instances use row and column sums instead of an edge list and
agree with the oracle within the per-vertex tolerance of the parity tests.
"""
import numpy as np
import pytest

import oracle
from paper_2605_05330_gb300 import inputs
from tests.test_gpu_parity import K_ITERATE, assert_close_rel, fixed_steps

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gn():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_05330_gb300 import build
    build.build()
    from paper_2605_05330_gb300 import gn as gnmod
    return gnmod


def small_specs(count=24, seed=777):
    specs = inputs.batch_specs(count, seed=seed, k_hi=16)
    # keep the test quick: cap ER sizes
    out = []
    for i, s in enumerate(specs):
        if isinstance(s, tuple):
            out.append(s)
        elif s.n <= 1500:
            out.append(s)
        else:
            out.append(inputs.er_graph(1500, 10.0, seed + 1000 + i))
    return out


def as_csr(spec):
    return inputs.assignment_instance(spec) if isinstance(spec, tuple) else spec


def batch_items(specs):
    return [s[:3] if isinstance(s, tuple) else s for s in specs]


def split(x, vtx):
    return [np.asarray(x[vtx[i]:vtx[i + 1]]) for i in range(len(vtx) - 1)]


@pytest.mark.parametrize("k", [1, 5, K_ITERATE])
def test_batch_iterates_match_oracle(gn, k):
    specs = small_specs()
    b = gn.Batch(batch_items(specs))
    run_kw, pk = fixed_steps(k)
    x, infos = b.run(params=gn.default_params(**pk), **run_kw)
    for s, xi, inf in zip(specs, split(x, b.vtx_off), infos):
        inst = as_csr(s)
        xo, io = oracle.run(inst.row_ptr, inst.col_idx, inst.w, p=oracle.params(**pk), **run_kw)
        assert inf["iters"] == k
        assert_close_rel(xi, xo)


def test_batch_final_sets_match_oracle(gn):
    specs = small_specs(seed=778)
    b = gn.Batch(batch_items(specs))
    x, infos = b.run(max_iters=2000, tol=1e-7)
    st, mask, counts, weights, statuses = b.extract()
    assert st in ("OK", "WARN_NOT_MAXIMAL")
    p = oracle.params(check_every=10)
    agree = 0
    for i, (s, xi, inf) in enumerate(zip(specs, split(x, b.vtx_off), infos)):
        inst = as_csr(s)
        # extraction agrees bit for bit with the oracle's rounding of the same state
        sto, masko, memo, Wo = oracle.extract_is(inst.row_ptr, inst.col_idx, inst.w, xi)
        np.testing.assert_array_equal(mask[b.vtx_off[i]:b.vtx_off[i + 1]], masko)
        assert counts[i] == len(memo) and abs(weights[i] - Wo) <= 1e-9 * Wo
        assert gn.STATUS[int(statuses[i])] == sto
        xo, io = oracle.run(inst.row_ptr, inst.col_idx, inst.w, max_iters=2000, tol=1e-7, p=p)
        assert inf["status"] == io["status"] == "OK"
        same = np.array_equal(xi > 0.5, xo > 0.5)
        agree += same
        if same:
            assert inf["iters"] == io["iters"]
        assert abs(inf["objective"] - io["objective"]) <= 1e-3 * io["objective"]
        if isinstance(s, tuple):  # assignment: a permutation
            P = (xi > 0.5).reshape(s[1], s[1])
            assert np.all(P.sum(0) == 1) and np.all(P.sum(1) == 1)
    assert agree >= len(specs) - 1


def test_batch_csr_equals_single_graph_path(gn):
    specs = [s for s in small_specs(seed=779) if not isinstance(s, tuple)][:6]
    b = gn.Batch(specs)
    x, infos = b.run(max_iters=2000)
    for s, xi, inf in zip(specs, split(x, b.vtx_off), infos):
        g = gn.Graph(s.row_ptr, s.col_idx, s.w, gather=gn.GATHER_GLOBAL)
        xs, ins = g.run(max_iters=2000)
        np.testing.assert_array_equal(xi, xs)
        assert inf["iters"] == ins["iters"]


def test_assignment_structured_matches_csr_form(gn):
    specs = [s for s in inputs.batch_specs(40, seed=780, k_hi=24) if isinstance(s, tuple)][:8]
    run_kw, pk = fixed_steps(20)
    bs = gn.Batch(batch_items(specs))
    bc = gn.Batch([inputs.assignment_instance(s) for s in specs])
    xs, _ = bs.run(params=gn.default_params(**pk), **run_kw)
    xc, _ = bc.run(params=gn.default_params(**pk), **run_kw)
    assert_close_rel(xs, xc.astype(np.float64))


def test_batch_graph_replay_tune_and_device_io(gn):
    import torch
    specs = small_specs(seed=781)
    b = gn.Batch(batch_items(specs))
    x1, i1 = b.run()
    x2, i2 = b.run()                 # replay of the captured graph
    np.testing.assert_array_equal(x1, x2)
    t = b.tune(max_iters=100)
    assert t in (256, 512, 1024)
    x3, i3 = b.run()
    np.testing.assert_array_equal(x1, x3)  # the CTA size does not change the arithmetic
    bd = gn.Batch(batch_items(specs), device=True)
    x4, i4 = bd.run()
    np.testing.assert_array_equal(x1, x4.cpu().numpy())
    assert [d["iters"] for d in i1] == [d["iters"] for d in i4]


@pytest.mark.parametrize("threads", [256, 512])
def test_warp_packing_is_bit_identical(gn, threads):
    """Instance packing: the small instances run a warp each, several per CTA, after the CTA
    queue; both kinds give the iterates and stop of CTA mode bit for bit, for fixed steps and for
    the run to a binary state."""
    specs = [s for s in small_specs(count=48, seed=783)]
    items = batch_items(specs)
    b = gn.Batch(items)
    b.set_threads(threads)
    run_kw, pk = fixed_steps(20)
    ref = [b.run(params=gn.default_params(**pk), **run_kw), b.run(max_iters=2000, tol=1e-7)]
    thr = 128 if threads == 512 else 256
    b.set_packing(thr)
    wm, moved = b.packing()
    assert wm == thr and moved > 0
    # both kinds have instances this small (whether each fits a warp's share is the library's call)
    small = {isinstance(s, tuple) for s in specs if (s[1] * s[1] if isinstance(s, tuple) else s.n) <= thr}
    assert small == {True, False}
    got = [b.run(params=gn.default_params(**pk), **run_kw), b.run(max_iters=2000, tol=1e-7)]
    for (xa, ia), (xb, ib) in zip(ref, got):
        np.testing.assert_array_equal(xa, xb)
        assert [d["iters"] for d in ia] == [d["iters"] for d in ib]
        assert [d["safe_div_hits"] for d in ia] == [d["safe_div_hits"] for d in ib]
    st, mask, counts, weights, statuses = b.extract()
    assert st in ("OK", "WARN_NOT_MAXIMAL")


def test_batch_validation(gn):
    good = inputs.er_graph(50, 4, 782)
    bad = inputs.GraphInstance("asym", np.array([0, 1, 1], np.int32), np.array([1], np.int32),
                               np.ones(2, np.float32))
    with pytest.raises(gn.GNError) as e:
        gn.Batch([good, bad])
    assert e.value.status == "ERR_NOT_SIMPLE"
    with pytest.raises(gn.GNError) as e:
        gn.Batch([good, ("assignment", 3, np.zeros(9, np.float32))])
    assert e.value.status == "ERR_WEIGHT"


def test_random_start_and_multi_start(gn):
    """The random simplex start on the GPU equals the oracle's (FP32 log vs FP64), and every start
    of the multi-start batch follows the oracle from the same start."""
    import torch
    u = inputs.uniforms(5000, 31)
    x0 = gn.random_start(torch.from_numpy(u).cuda()).cpu().numpy()
    np.testing.assert_allclose(x0, oracle.random_start(u), rtol=2e-6, atol=1e-9)
    inst = inputs.er_graph(300, 8.0, 32)
    W, mask, info, ws = gn.multi_start(inst, starts=8, seed=33)
    u = inputs.uniforms(8 * inst.n, 33)
    starts = oracle.random_start(u).reshape(8, inst.n).astype(np.float32)
    for s in range(8):
        xo, io = oracle.run(inst.row_ptr, inst.col_idx, inst.w, x0=starts[s], max_iters=2000, tol=1e-7,
                            p=oracle.params(check_every=10))
        Wo = oracle.extract_is(inst.row_ptr, inst.col_idx, inst.w, xo)[3]
        assert abs(ws[s] - Wo) <= 1e-3 * Wo
    assert W == ws.max()


def test_assignment_up_to_k96_in_one_launch(gn):
    """The stress end of the batched config's assignment sizes: k = 96 (9216 vertices, 1.75M
    entries in CSR form), 90 and 72 next to a CSR instance in one launch.  The structured form
    keeps five state arrays per vertex in shared memory, so they fit; each instance follows the
    oracle and ends on a permutation."""
    specs = []
    for i, k in enumerate((96, 90, 72)):
        rng = inputs.rng_for(4000 + i)
        cost = rng.random((k, k))
        w = (2.0 - cost).astype(np.float32).reshape(-1)
        specs.append(("assignment", k, w, (2.0 - w.astype(np.float64)).reshape(k, k)))
    specs.append(inputs.er_graph(3000, 10.0, 4010))
    b = gn.Batch(batch_items(specs))
    run_kw, pk = fixed_steps(K_ITERATE)
    x, infos = b.run(params=gn.default_params(**pk), **run_kw)
    for s, xi, inf in zip(specs, split(x, b.vtx_off), infos):
        inst = as_csr(s)
        xo, io = oracle.run(inst.row_ptr, inst.col_idx, inst.w, p=oracle.params(**pk), **run_kw)
        assert inf["iters"] == K_ITERATE
        assert_close_rel(xi, xo)
    x, infos = b.run(max_iters=2000, tol=1e-7)
    for s, xi, inf in zip(specs, split(x, b.vtx_off), infos):
        assert inf["status"] == "OK"
        if isinstance(s, tuple):
            P = (xi > 0.5).reshape(s[1], s[1])
            assert np.all(P.sum(0) == 1) and np.all(P.sum(1) == 1)
