"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the passage it follows.  None of them re-types the oracle's update
formula: they use worked examples printed in the paper (tests/golden), closed
forms derived by hand, theorems (descent, mass growth, stability, Motzkin-Straus),
identities stated in the appendices evaluated with dense numpy algebra, library
routines (numpy normalisation, scipy assignment) and brute force.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2605_05330_gb300 import inputs
from tests.conftest import read_golden


def _graph_from_golden(g):
    inst = inputs.small_graph("golden", int(g["n"][0]), g["edges"], [float(t) for t in g["w"]])
    return inst


@pytest.mark.parametrize("fixture", ["wrgn_edge_step.txt", "wrgn_star_step.txt",
                                     "gn_fixed_point_7node.txt", "gn_p3_fixed_point.txt"])
def test_step_worked_examples(fixture):
    """Def. 3 (WRGN) / App. A worked examples: one step equals the hand-computed values."""
    g = read_golden(fixture)
    inst = _graph_from_golden(g)
    x = np.array([float(t) for t in g["x"]])
    xn, hits = oracle.step(inst.row_ptr, inst.col_idx, inst.w, float(g["gamma"][0]), x)
    want = np.array([float(t) for t in g["x_next"]])
    assert hits == 0
    np.testing.assert_allclose(xn, want, rtol=1e-15, atol=0)


def test_p3_closed_sum_of_zero_vertex():
    """App. A: at (1,0,1) on P3 the zero vertex has closed neighbourhood sum 2, so it
    contracts by 1/2 per step when perturbed (Jacobian entry 1/(B x*)_i, Lemma 1)."""
    g = read_golden("gn_p3_fixed_point.txt")
    inst = _graph_from_golden(g)
    eps = 1e-9
    xn, _ = oracle.step(inst.row_ptr, inst.col_idx, inst.w, 1.0, np.array([1.0, eps, 1.0]))
    assert abs(xn[1] / eps - 1.0 / float(g["closed_sum_middle"][0])) < 1e-8


def test_complete_graph_is_simplex_normalisation():
    """Sec. 2: on K_n with gamma = 1 and unit weights one step is x / sum(x)."""
    n = 7
    inst = inputs.small_graph("K7", n, [(i, j) for i in range(n) for j in range(i + 1, n)])
    x = np.random.default_rng(3).random(n) + 0.1
    xn, _ = oracle.step(inst.row_ptr, inst.col_idx, inst.w, 1.0, x)
    np.testing.assert_allclose(xn, x / np.sum(x), rtol=1e-14)
    # binary fixed points of K_n are the one-hot vectors
    e = np.zeros(n); e[2] = 1.0
    xn, _ = oracle.step(inst.row_ptr, inst.col_idx, inst.w, 1.0, e)
    np.testing.assert_array_equal(xn, e)


def test_complete_graph_weighted_is_tilted_normalisation():
    """Def. WRGN on K_n with gamma = 1: every vertex's weighted closed sum is the whole
    weighted state, so x_i' = v_i x_i / sum_j v_j x_j, i.e. x' = y / sum(y) on the simplex."""
    n = 6
    inst = inputs.small_graph("K6", n, [(i, j) for i in range(n) for j in range(i + 1, n)],
                              w=np.arange(1, n + 1, dtype=np.float32) ** 2)
    x = np.random.default_rng(4).random(n) + 0.1
    v = np.sqrt(inst.w.astype(np.float64))
    xn, _ = oracle.step(inst.row_ptr, inst.col_idx, inst.w, 1.0, x)
    np.testing.assert_allclose(xn, v * x / np.dot(v, x), rtol=1e-14)
    assert abs(np.sum(xn) - 1.0) < 1e-14


@pytest.mark.parametrize("name,n,edges,d", [
    ("C6", 6, [(i, (i + 1) % 6) for i in range(6)], 2),
    ("petersen", 10, [(i, (i + 1) % 5) for i in range(5)] + [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
     + [(i, i + 5) for i in range(5)], 3),
    ("K33", 6, [(i, j) for i in range(3) for j in range(3, 6)], 3),
])
@pytest.mark.parametrize("gamma", [1.0, 1.5])
def test_regular_graph_uniform_atom(name, n, edges, d, gamma):
    """App. A: a d-regular graph is normalised by a uniform vector; any uniform x maps to
    1/(1 + gamma d) in one step and stays there (uniform weights)."""
    inst = inputs.small_graph(name, n, edges)
    assert set(np.diff(inst.row_ptr).tolist()) == {d}
    x = np.full(n, 0.37)
    x1, _ = oracle.step(inst.row_ptr, inst.col_idx, inst.w, gamma, x)
    np.testing.assert_allclose(x1, 1.0 / (1.0 + gamma * d), rtol=1e-15)
    x2, _ = oracle.step(inst.row_ptr, inst.col_idx, inst.w, gamma, x1)
    np.testing.assert_allclose(x2, x1, rtol=1e-15)
    # the run reports a converged, non-binary state (the symmetric trap)
    xo, info = oracle.run(inst.row_ptr, inst.col_idx, inst.w, x0=x, max_iters=50, tol=1e-12,
                          p=oracle.params(gamma_mode=oracle.GAMMA_FIXED, gamma1=gamma))
    assert info["status"] == "WARN_NOT_BINARY" and info["converged"] == 1
    np.testing.assert_allclose(xo, 1.0 / (1.0 + gamma * d), rtol=1e-15)


def _k2(w0):
    return inputs.small_graph("K2", 2, [(0, 1)], w=[w0, 1.0])


def test_k2_interior_fixed_point_below_gamma_B():
    """App. H: below gamma_B the K2 energy is convex and GN converges to the apex x_a
    (printed closed form) from any start."""
    g = read_golden("k2_phase_thresholds.txt")
    w0 = float(g["w0"][0])
    inst = _k2(w0)
    gam = 0.25
    for start in ([0.9, 0.1], [0.05, 0.95], [0.5, 0.5]):
        x, info = oracle.run(inst.row_ptr, inst.col_idx, inst.w, x0=start, max_iters=5000, tol=1e-15,
                             p=oracle.params(gamma_mode=oracle.GAMMA_FIXED, gamma1=gam))
        assert info["converged"] == 1
        p1 = x[1] * 1.0 / (w0 * x[0] + x[1])      # simplex state p_i ~ w_i x_i
        assert abs(p1 - float(g["apex_gamma_1/4"][0])) < 1e-12


@pytest.mark.parametrize("gam", [0.6, 1.0, 1.25, 1.5, 1.9])
def test_k2_heavier_wins_between_gamma_B_and_gamma_D(gam):
    """App. H: for gamma_B < gamma < gamma_D every start converges to the MIS {0} (heavier)."""
    g = read_golden("k2_phase_thresholds.txt")
    w0 = float(g["w0"][0])
    assert float(g["gamma_B"][0]) < gam < float(g["gamma_D"][0])
    inst = _k2(w0)
    for start in ([0.01, 0.99], [0.2, 0.9], [0.5, 0.5]):
        x, info = oracle.run(inst.row_ptr, inst.col_idx, inst.w, x0=start, max_iters=200000,
                             tol=0.0, p=oracle.params(gamma_mode=oracle.GAMMA_FIXED, gamma1=gam))
        assert x[0] > 1 - 1e-3 and x[1] < 1e-3, (gam, start, x)


def test_k2_separatrix_above_gamma_D():
    """App. H: above gamma_D both MIS are stable; the apex x_a = 5/7 (gamma = 3) separates
    their basins on the simplex."""
    g = read_golden("k2_phase_thresholds.txt")
    w0 = float(g["w0"][0])
    inst = _k2(w0)
    xa = float(g["apex_gamma_3"][0])
    for p1, winner in ((xa - 0.02, 0), (xa + 0.02, 1)):
        start = [(1 - p1) / w0, p1]                # w_i x_i = p_i
        x, info = oracle.run(inst.row_ptr, inst.col_idx, inst.w, x0=start, max_iters=10000, tol=0.0,
                             p=oracle.params(gamma_mode=oracle.GAMMA_FIXED, gamma1=3.0))
        assert info["status"] == "OK"
        assert x[winner] > 0.999 and x[1 - winner] < 1e-3


def test_k2_equal_weights_larger_start_wins():
    """App. H, unweighted K2 with gamma > 1: the larger initial value wins."""
    inst = _k2(1.0)
    x, info = oracle.run(inst.row_ptr, inst.col_idx, inst.w, x0=[0.51, 0.49], max_iters=5000,
                         tol=0.0, p=oracle.params(gamma_mode=oracle.GAMMA_FIXED, gamma1=1.5))
    assert info["status"] == "OK" and x[0] > 0.999


def test_scale_invariance_bit_exact():
    """Sec. 2 property iv: N(alpha x) = N(x); exact in FP64 for alpha a power of two."""
    inst = inputs.er_graph(60, 5, 11)
    x = np.random.default_rng(1).random(inst.n) + 1e-3
    a, _ = oracle.step(inst.row_ptr, inst.col_idx, inst.w, 1.3, x)
    for alpha in (0.25, 8.0, 2.0 ** -20):
        b, _ = oracle.step(inst.row_ptr, inst.col_idx, inst.w, 1.3, x * alpha)
        np.testing.assert_array_equal(a, b)


def test_support_invariance_and_boundedness():
    """Sec. 2 properties i and ii: values stay in [0,1] and zeros stay zero, positives positive."""
    inst = inputs.er_graph(80, 6, 12)
    rng = np.random.default_rng(2)
    x = rng.random(inst.n) * 5
    x[rng.random(inst.n) < 0.3] = 0.0
    # keep it normalizable: every vertex with a zero closed neighbourhood gets a value
    for i in range(inst.n):
        nb = inst.col_idx[inst.row_ptr[i]:inst.row_ptr[i + 1]]
        if x[i] == 0 and np.all(x[nb] == 0):
            x[i] = 1.0
    for _ in range(30):
        xn, hits = oracle.step(inst.row_ptr, inst.col_idx, inst.w, 1.2, x)
        assert hits == 0
        assert np.all((xn >= 0) & (xn <= 1))
        np.testing.assert_array_equal(xn > 0, x > 0)
        x = xn


def test_component_independence_bit_exact():
    """Sec. 2 property iii: the union of disjoint graphs evolves as the parts do, exactly."""
    parts = [inputs.er_graph(40, 4, 21), inputs.er_graph(25, 3, 22), inputs.small_graph("iso", 3, [])]
    uni = inputs.disjoint_union(parts)
    xs = [np.random.default_rng(7 + i).random(p.n) + 0.05 for i, p in enumerate(parts)]
    xu = np.concatenate(xs)
    for k in range(40):
        gam = 0.9 + 0.6 * k / 39
        xu, _ = oracle.step(uni.row_ptr, uni.col_idx, uni.w, gam, xu)
        xs = [oracle.step(p.row_ptr, p.col_idx, p.w, gam, x)[0] for p, x in zip(parts, xs)]
    np.testing.assert_array_equal(xu, np.concatenate(xs))
    # isolated vertices go to 1 in one step (closed sum = own value)
    assert np.all(xs[2] == 1.0)


def _dense(inst):
    n = inst.n
    A = np.zeros((n, n))
    for i in range(n):
        A[i, inst.col_idx[inst.row_ptr[i]:inst.row_ptr[i + 1]]] = 1.0
    return A


@pytest.mark.parametrize("seed", [31, 32, 33])
def test_preconditioned_gradient_identity(seed):
    """App. C: y^{k+1} - y^k = -diag(y^{k+1} / v) grad E~(y^k), grad E~ = (I + gamma A) y - v."""
    inst = inputs.er_graph(50, 6, seed)
    A = _dense(inst)
    v = np.sqrt(inst.w.astype(np.float64))
    x = np.random.default_rng(seed).random(inst.n) + 0.05
    gam = 1.37
    xn, _ = oracle.step(inst.row_ptr, inst.col_idx, inst.w, gam, x)
    y, yn = v * x, v * xn
    grad = (np.eye(inst.n) + gam * A) @ y - v
    np.testing.assert_allclose(yn - y, -(yn / v) * grad, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("seed", [41, 42])
def test_replicator_identity(seed):
    """Thm. 5 / App. I: with p = v y / M_v and f_i = v_i / ((I + gamma A)(p / v))_i, the next
    weighted mass is the average fitness, M_v^{k+1} = sum_i p_i f_i, and p' = p f / fbar."""
    inst = inputs.er_graph(40, 5, seed)
    A = _dense(inst)
    v = np.sqrt(inst.w.astype(np.float64))
    x = np.random.default_rng(seed).random(inst.n) + 0.05
    gam = 1.2
    xn, _ = oracle.step(inst.row_ptr, inst.col_idx, inst.w, gam, x)
    y, yn = v * x, v * xn
    M = np.dot(v, y)
    p = v * y / M
    f = v / ((np.eye(inst.n) + gam * A) @ (p / v))
    fbar = np.dot(p, f)
    assert abs(np.dot(v, yn) - fbar) < 1e-12 * fbar
    np.testing.assert_allclose(v * yn / np.dot(v, yn), p * f / fbar, rtol=1e-12)


@pytest.mark.parametrize("seed", [51, 52, 53, 54])
def test_energy_descent_and_mass_growth_fixed_gamma(seed):
    """Thm. 1 (strict energy descent) and Thm. 3 (weighted mass strictly increases from the
    first image of the map on), at fixed gamma."""
    inst = inputs.er_graph(120, 8, seed)
    T = 300
    x, info, tobj, ten = oracle.run(
        inst.row_ptr, inst.col_idx, inst.w, x0=np.random.default_rng(seed).random(inst.n) + 0.01,
        max_iters=T, tol=-1.0, p=oracle.params(gamma_mode=oracle.GAMMA_FIXED, gamma1=1.5,
                                               theta_bin=-1.0), trace_len=T)
    assert info["iters"] == T
    dE = np.diff(ten)
    dM = np.diff(tobj)
    scale = np.abs(ten).max()
    assert np.all(dE <= 1e-13 * scale)
    assert np.all(dE[:20] < 0)
    assert np.all(dM >= -1e-13 * tobj.max())
    assert np.all(dM[:20] > 0)


@pytest.mark.parametrize("seed", range(61, 69))
def test_final_state_is_stable_mis(seed):
    """Thm. 4 (binary regularisation) and Thm. 6 (tilted Motzkin-Straus): the pursuit run ends
    on a binary MIS M with stab(M) > 1, E~ = -W(M)/2 and Q(r) = 1/W(M) at r = y / M_v."""
    inst = inputs.er_graph(150, 7, seed)
    p = oracle.params()
    x, info = oracle.run(inst.row_ptr, inst.col_idx, inst.w, max_iters=3000, tol=1e-12, p=p)
    assert info["status"] == "OK" and info["binary"] == 1
    st, mask, members, W = oracle.extract_is(inst.row_ptr, inst.col_idx, inst.w, x)
    assert st == "OK"
    gam = oracle.gamma(p, info["iters"] - 1)
    assert oracle.stability(inst.row_ptr, inst.col_idx, inst.w, gam, mask) > 1.0
    xb = mask.astype(np.float64)
    assert abs(oracle.energy(inst.row_ptr, inst.col_idx, inst.w, gam, xb) + W / 2) < 1e-9 * W
    A = _dense(inst)
    v = np.sqrt(inst.w.astype(np.float64))
    r = v * xb / np.dot(inst.w.astype(np.float64), xb)
    Q = r @ ((np.eye(inst.n) + gam * A) @ r)
    assert abs(Q - 1.0 / W) < 1e-12 / W
    assert abs(info["objective"] - W) < 1e-3 * W


def _brute_mwis_python(inst):
    n = inst.n
    best, arg = -1.0, None
    w = inst.w.astype(np.float64)
    edges = [(i, j) for i in range(n) for j in inst.col_idx[inst.row_ptr[i]:inst.row_ptr[i + 1]] if i < j]
    for bits in itertools.product((0, 1), repeat=n):
        if any(bits[i] and bits[j] for i, j in edges):
            continue
        s = sum(w[i] for i in range(n) if bits[i])
        if s > best:
            best, arg = s, bits
    return best, arg


@pytest.mark.parametrize("seed", [71, 72, 73])
def test_brute_force_enumerator_matches_exhaustive_python(seed):
    """The C enumerator against exhaustive Python over all 2^n subsets (n = 12)."""
    inst = inputs.er_graph(12, 3, seed)
    W, masks = oracle.mwis_enumerate(inst.row_ptr, inst.col_idx, inst.w)
    Wp, _ = _brute_mwis_python(inst)
    assert abs(W - Wp) < 1e-9


@pytest.mark.parametrize("seed", range(81, 91))
def test_gn_bounded_by_mwis_and_every_mwis_stable(seed):
    """Thm. 4 (optimality): every MWIS is gamma-stable with stab >= gamma > 1; GN returns an
    independent set of weight <= W* (n <= 20)."""
    inst = inputs.er_graph(18 + seed % 3, 3.5, seed)
    W, masks = oracle.mwis_enumerate(inst.row_ptr, inst.col_idx, inst.w)
    for gam in (1.05, 1.5):
        for m in masks:
            assert oracle.stability(inst.row_ptr, inst.col_idx, inst.w, gam, m.astype(np.uint8)) >= gam - 1e-12
    x, info = oracle.run(inst.row_ptr, inst.col_idx, inst.w, max_iters=3000)
    st, mask, members, Wgn = oracle.extract_is(inst.row_ptr, inst.col_idx, inst.w, x)
    assert st == "OK"
    assert Wgn <= W + 1e-9


def test_hungarian_against_library_and_permutations():
    """Textbook Hungarian (Sec. 1) against scipy's assignment solver and brute force (k <= 7)."""
    from scipy.optimize import linear_sum_assignment
    rng = np.random.default_rng(5)
    for k in (1, 2, 3, 5, 7):
        c = rng.random((k, k))
        tot, asg = oracle.hungarian(c)
        assert sorted(asg.tolist()) == list(range(k))
        best = min(sum(c[i, p[i]] for i in range(k)) for p in itertools.permutations(range(k)))
        assert abs(tot - best) < 1e-12
    for k in (16, 40):
        c = rng.random((k, k))
        tot, asg = oracle.hungarian(c)
        r, cidx = linear_sum_assignment(c)
        assert abs(tot - c[r, cidx].sum()) < 1e-10


@pytest.mark.parametrize("k", [8, 10, 12])
def test_assignment_fixed_point_is_permutation(k):
    """Sec. 2 (cross-normalisation on L(K_{k,k})): GN ends on a MIS of the rook graph, i.e. a
    permutation matrix, whose weight is bounded by the Hungarian optimum (w = 2 - cost)."""
    inst = inputs.assignment_graph(k, 100 + k)
    x, info = oracle.run(inst.row_ptr, inst.col_idx, inst.w, max_iters=3000)
    assert info["status"] == "OK"
    st, mask, members, W = oracle.extract_is(inst.row_ptr, inst.col_idx, inst.w, x)
    assert st == "OK"
    P = mask.reshape(k, k)
    assert np.all(P.sum(0) == 1) and np.all(P.sum(1) == 1)
    tot, _ = oracle.hungarian(inst.meta["cost"])
    assert W <= 2 * k - tot + 1e-6


def test_cross_normalisation_row_column_sums():
    """Sec. 2: on L(K_{k,k}) with gamma = 1, w = 1 the step divides W_ij by its row sum plus
    column sum minus W_ij."""
    k = 5
    rp, ci = inputs.rook_csr(k)
    Wm = np.random.default_rng(9).random((k, k)) + 0.1
    xn, _ = oracle.step(rp, ci, np.ones(k * k), 1.0, Wm.reshape(-1))
    want = Wm / (Wm.sum(1, keepdims=True) + Wm.sum(0, keepdims=True) - Wm)
    np.testing.assert_allclose(xn.reshape(k, k), want, rtol=1e-14)


def test_nonmember_decay_rate():
    """Thm. 4 proof (App. G): near a binary fixed point M a non-member contracts by
    1 / (gamma * sum_{j in N(i) cap M} sqrt(w_j / w_i)) per step (Jacobian diagonal)."""
    inst = inputs.er_graph(40, 4, 91)
    gam = 1.5
    p = oracle.params(gamma_mode=oracle.GAMMA_FIXED, gamma1=gam, theta_bin=1e-9)
    x, info = oracle.run(inst.row_ptr, inst.col_idx, inst.w, max_iters=400, tol=-1, p=p)
    st, mask, _, _ = oracle.extract_is(inst.row_ptr, inst.col_idx, inst.w, x)
    assert st == "OK"
    xn, _ = oracle.step(inst.row_ptr, inst.col_idx, inst.w, gam, x)
    w = inst.w.astype(np.float64)
    checked = 0
    for i in range(inst.n):
        if mask[i] or x[i] < 1e-290:      # skip values that underflowed towards denormals
            continue
        nb = inst.col_idx[inst.row_ptr[i]:inst.row_ptr[i + 1]]
        rate = 1.0 / (gam * sum(math.sqrt(w[j] / w[i]) for j in nb if mask[j]))
        assert abs(xn[i] / x[i] - rate) < 1e-6 * rate
        checked += 1
    assert checked > 5


def test_gamma_schedule():
    """Sec. 6 / appendix module: linear pursuit 0.9 -> 1.5 over 1000 iterations, then held."""
    p = oracle.params()
    assert oracle.gamma(p, 0) == 0.9
    assert abs(oracle.gamma(p, 999) - 1.5) < 1e-15
    assert abs(oracle.gamma(p, 1500) - 1.5) < 1e-15
    assert abs(oracle.gamma(p, 333) - (0.9 + 0.6 * 333 / 999)) < 1e-15
    q = oracle.params(gamma_mode=oracle.GAMMA_FIXED, gamma1=1.3)
    assert oracle.gamma(q, 0) == 1.3 and oracle.gamma(q, 10 ** 6) == 1.3


def test_safe_division():
    """Appendix module: a weighted-state denominator <= 1e-9 sets the value to 0.5 (counted)."""
    inst = inputs.small_graph("P4", 4, [(0, 1), (1, 2), (2, 3)])
    xn, hits = oracle.step(inst.row_ptr, inst.col_idx, inst.w, 1.5, np.full(4, 1e-12))
    assert hits == 4 and np.all(xn == 0.5)
    xn, hits = oracle.step(inst.row_ptr, inst.col_idx, inst.w, 1.5, np.full(4, 1e-6))
    assert hits == 0


def test_validation_errors():
    """Sec. 2 (simple undirected graph, w > 0) and Def. 1 (normalizable start)."""
    ok = inputs.small_graph("P3", 3, [(0, 1), (1, 2)])
    assert oracle.validate(ok.row_ptr, ok.col_idx, ok.w) == "OK"
    assert oracle.validate([0, 1, 1], [1], [1, 1]) == "ERR_NOT_SIMPLE"          # asymmetric
    assert oracle.validate([0, 1, 2], [0, 0], [1, 1]) == "ERR_NOT_SIMPLE"       # self-loop
    assert oracle.validate([0, 2, 4], [1, 1, 0, 0], [1, 1]) == "ERR_NOT_SIMPLE"  # duplicate
    assert oracle.validate([0, 1, 2], [1, 0], [1, 0]) == "ERR_WEIGHT"
    assert oracle.validate([0, 1, 2], [1, 0], [1, float("nan")]) == "ERR_WEIGHT"
    assert oracle.validate([0, 1, 2], [1, 5], [1, 1]) == "ERR_ARG"
    x, info = oracle.run(ok.row_ptr, ok.col_idx, ok.w, x0=[0.0, 0.0, 1.0])
    assert info["status"] == "ERR_NOT_NORMALIZABLE"
    x, info = oracle.run(ok.row_ptr, ok.col_idx, ok.w, x0=[0.5, -0.1, 1.0])
    assert info["status"] == "ERR_NOT_NORMALIZABLE"
    x, info = oracle.run(ok.row_ptr, ok.col_idx, ok.w, x0=[0.0, 1.0, 0.0])
    assert info["status"] in ("OK", "WARN_NOT_CONVERGED")


def test_resume_is_bit_exact():
    """The schedule is a function of the absolute iteration index, so a run split at K and
    resumed from x^K with start_iter = K equals the uninterrupted run."""
    inst = inputs.er_graph(300, 8, 95)
    p = oracle.params(check_every=10)
    x_full, info_full = oracle.run(inst.row_ptr, inst.col_idx, inst.w, max_iters=400, tol=-1, p=p)
    xa, ia = oracle.run(inst.row_ptr, inst.col_idx, inst.w, max_iters=170, tol=-1, p=p)
    assert ia["iters"] == 170
    xb, ib = oracle.run(inst.row_ptr, inst.col_idx, inst.w, x0=xa, max_iters=400, tol=-1, p=p,
                        start_iter=170)
    np.testing.assert_array_equal(xb, x_full)
    assert ia["iters"] + ib["iters"] == info_full["iters"]


def test_stop_cadence_and_default_start():
    """The stop test runs every check_every iterations; x0 = NULL is 1/(deg+1)."""
    inst = inputs.er_graph(400, 10, 97)
    p = oracle.params(check_every=7)
    x, info = oracle.run(inst.row_ptr, inst.col_idx, inst.w, max_iters=2000, p=p)
    assert info["status"] == "OK" and info["iters"] % 7 == 0
    deg = np.diff(inst.row_ptr)
    x2, info2 = oracle.run(inst.row_ptr, inst.col_idx, inst.w, x0=1.0 / (deg + 1.0), max_iters=2000, p=p)
    np.testing.assert_array_equal(x, x2)
    # check_every = 1 stops at the first binary iteration <= the cadence-7 stop
    x3, info3 = oracle.run(inst.row_ptr, inst.col_idx, inst.w, max_iters=2000, p=oracle.params())
    assert info3["iters"] <= info["iters"] and info["iters"] - info3["iters"] < 7


def test_zero_iterations_and_edgeless():
    inst = inputs.small_graph("E5", 5, [])
    x, info = oracle.run(inst.row_ptr, inst.col_idx, inst.w, max_iters=0)
    assert info["iters"] == 0 and info["status"] == "WARN_NOT_CONVERGED"
    x, info = oracle.run(inst.row_ptr, inst.col_idx, inst.w, max_iters=100)
    np.testing.assert_array_equal(x, np.ones(5))
    empty = inputs.small_graph("E0", 0, [])
    x, info = oracle.run(empty.row_ptr, empty.col_idx, empty.w, max_iters=10)
    assert x.size == 0


def test_random_start():
    """Appendix module: exponential draws -log u scaled by their maximum and clamped to
    [1e-3, 1]; the largest draw maps to exactly 1, tiny draws to the 1e-3 floor, and the
    order of the draws is reversed (larger u, smaller p)."""
    u = np.array([0.5, 0.25, 1.0 - 1e-12, 0.9999, 1e-6])
    x = oracle.random_start(u)
    assert x[4] == 1.0                                  # smallest u has the largest -log u
    assert abs(x[0] - np.log(2) / np.log(1e6)) < 1e-15  # -log(1/2) / -log(1e-6)
    assert x[2] == 1e-3 and x[3] == 1e-3                # clamped
    assert np.all(np.diff(oracle.random_start(np.array([0.1, 0.2, 0.3, 0.4]))) < 0)


@pytest.mark.parametrize("seed", [201, 202])
def test_unrolled_gradient_against_central_differences(seed):
    """The FP64 reference gradients of L = g . x_T (T unrolled WRGN steps) agree with central
    finite differences of the forward in FP64 (w and x0 directions)."""
    torch = pytest.importorskip("torch")
    from oracle import grad
    inst = inputs.er_graph(25, 4, seed)
    rng = np.random.default_rng(seed)
    x0 = rng.random(inst.n) + 0.1
    g = rng.standard_normal(inst.n)
    gam = grad.gammas(30)
    w = inst.w.astype(np.float64)
    L, dw, dx0, xT = grad.loss_and_grads(inst.row_ptr, inst.col_idx, w, x0, g, gam)

    def f(wv, xv):
        with torch.no_grad():
            xt = grad.unrolled(inst.row_ptr, inst.col_idx, torch.tensor(wv), torch.tensor(xv), gam)
        return float(np.dot(g, xt.numpy()))
    # the forward equals the C oracle's iteration
    xo, _ = oracle.run(inst.row_ptr, inst.col_idx, w, x0=x0, max_iters=30, tol=-1,
                       p=oracle.params(theta_bin=-1.0))
    np.testing.assert_allclose(xT, xo, rtol=1e-12, atol=1e-300)
    for i in range(0, inst.n, 5):
        h = 1e-6 * w[i]
        e = np.zeros(inst.n); e[i] = h
        fd = (f(w + e, x0) - f(w - e, x0)) / (2 * h)
        assert abs(fd - dw[i]) <= 1e-6 * max(1.0, abs(dw[i]))
        h = 1e-6 * x0[i]
        e = np.zeros(inst.n); e[i] = h
        fd = (f(w, x0 + e) - f(w, x0 - e)) / (2 * h)
        assert abs(fd - dx0[i]) <= 1e-6 * max(1.0, abs(dx0[i]))


def test_mpnn_reference_gradient_against_central_differences():
    """The FP64 warm-start network's autograd gradient agrees with central differences of its
    loss (FP64 weights, no bf16 rounding), on a small unit-disk graph."""
    pytest.importorskip("torch")
    from oracle import mpnn
    inst = inputs.unit_disk_graph(60, 150, 301)
    rng = np.random.default_rng(302)
    theta = (rng.standard_normal(mpnn.num_params()) * 0.2).astype(np.float64)
    t = (rng.random(inst.n) < 0.3).astype(np.float64)
    p, loss, g = mpnn.forward(inst.row_ptr, inst.col_idx, inst.w, theta.astype(np.float32), t, bf16=False)
    th32 = theta.astype(np.float32).astype(np.float64)
    for idx in rng.choice(len(theta), 25, replace=False):
        h = 1e-4
        e = np.zeros(len(theta)); e[idx] = h
        lp = mpnn.forward(inst.row_ptr, inst.col_idx, inst.w, th32 + e, t, bf16=False)[1]
        lm = mpnn.forward(inst.row_ptr, inst.col_idx, inst.w, th32 - e, t, bf16=False)[1]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-5 * max(1.0, abs(g[idx])), (idx, fd, g[idx])
    assert p.shape == (inst.n,) and np.all((p > 0) & (p < 1))


@pytest.mark.parametrize("a,b,gam", [(0.3, 0.7, 1.2), (0.9, 0.05, 0.8), (0.25, 0.25, 1.5)])
def test_energy_on_k2_at_fractional_states(a, b, gam):
    """Sec. 3: E~(y) = 1/2 y^T (I + gamma A) y - v^T y with y = v (.) x.  On K2 with w = (4, 1),
    v = (2, 1) and y = (2a, b), worked by hand: E~ = 1/2 (4a^2 + b^2 + 4 gamma a b) - (4a + b).
    Away from a binary state the gamma term is not zero, so a dropped or doubled gamma, or a
    wrong weight exponent, changes the value."""
    inst = inputs.small_graph("K2", 2, [(0, 1)], [4.0, 1.0])
    want = 0.5 * (4 * a * a + b * b + 4 * gam * a * b) - (4 * a + b)
    got = oracle.energy(inst.row_ptr, inst.col_idx, inst.w, gam, np.array([a, b]))
    assert got == pytest.approx(want, rel=1e-14, abs=1e-15)


@pytest.mark.parametrize("name,n,edges,d", [
    ("C7", 7, [(i, (i + 1) % 7) for i in range(7)], 2),
    ("K4", 4, [(i, j) for i in range(4) for j in range(i + 1, 4)], 3),
    ("Q3", 8, [(i, i ^ (1 << k)) for i in range(8) for k in range(3) if i < i ^ (1 << k)], 3),
])
@pytest.mark.parametrize("c,gam,wv", [(0.2, 1.5, 1.0), (0.6, 0.9, 9.0)])
def test_energy_uniform_state_on_regular_graphs(name, n, edges, d, c, gam, wv):
    """Sec. 3 energy at the uniform state x = c 1 of a d-regular graph with uniform weight w
    (the atom of App. A): y = sqrt(w) c, (I + gamma A) y = (1 + gamma d) y, so
    E~ = n w (c^2 (1 + gamma d) / 2 - c)."""
    inst = inputs.small_graph(name, n, edges, [wv] * n)
    want = n * wv * (0.5 * c * c * (1 + gam * d) - c)
    got = oracle.energy(inst.row_ptr, inst.col_idx, inst.w, gam, np.full(n, c))
    assert got == pytest.approx(want, rel=1e-14)


def test_extract_is_failure_branches():
    """Sec. 2 (independent sets) and Sec. 6 (valid MIS after rounding): on the path 0-1-2-3-4
    the rounding of (1, 0, 1, 0, 1) is a maximal independent set; raising vertex 1 above 1/2
    puts the edge 0-1 inside S (not independent); (1, 0, 0, 0, 1) leaves vertex 2 with no
    neighbour in S (not maximal); exactly 1/2 rounds out."""
    inst = inputs.small_graph("P5", 5, [(0, 1), (1, 2), (2, 3), (3, 4)], [1.0, 2.0, 3.0, 4.0, 5.0])
    rp, ci, w = inst.row_ptr, inst.col_idx, inst.w
    st, mask, mem, W = oracle.extract_is(rp, ci, w, np.array([0.9, 0.1, 0.8, 0.2, 0.7]))
    assert st == "OK" and list(mem) == [0, 2, 4] and W == 9.0
    st, mask, mem, W = oracle.extract_is(rp, ci, w, np.array([0.9, 0.6, 0.8, 0.2, 0.7]))
    assert st == "ERR_NOT_INDEPENDENT" and list(mask) == [1, 1, 1, 0, 1] and W == 11.0
    st, mask, mem, W = oracle.extract_is(rp, ci, w, np.array([0.9, 0.1, 0.5, 0.2, 0.7]))
    assert st == "WARN_NOT_MAXIMAL" and list(mem) == [0, 4] and W == 6.0
    # a dependent set is reported as such even when it is also not maximal elsewhere
    st, *_ = oracle.extract_is(rp, ci, w, np.array([0.9, 0.6, 0.0, 0.0, 0.0]))
    assert st == "ERR_NOT_INDEPENDENT"


def test_stability_exact_value():
    """Thm. 4: stab_{gamma,w}(M) = gamma min_{i not in M} sum_{j in N(i) cap M} sqrt(w_j / w_i).
    Path 0-1-2-3-4 with w = (4, 1, 9, 16, 4) and M = {0, 3}: vertex 1 sees sqrt(4/1) = 2 (its
    neighbour 2 is not in M), vertex 2 sees sqrt(16/9) = 4/3, vertex 4 sees sqrt(16/4) = 2, so
    stab = 4 gamma / 3.  Summing over all neighbours would give 5 gamma / 3, a maximum 2 gamma,
    inverted ratios gamma / 2."""
    inst = inputs.small_graph("P5", 5, [(0, 1), (1, 2), (2, 3), (3, 4)], [4.0, 1.0, 9.0, 16.0, 4.0])
    mask = np.array([1, 0, 0, 1, 0], dtype=np.uint8)
    for gam in (1.0, 1.5):
        got = oracle.stability(inst.row_ptr, inst.col_idx, inst.w, gam, mask)
        assert got == pytest.approx(4.0 * gam / 3.0, rel=1e-15)
    assert oracle.stability(inst.row_ptr, inst.col_idx, inst.w, 1.5, np.ones(5, np.uint8)) == math.inf
