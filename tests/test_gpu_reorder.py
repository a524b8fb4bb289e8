"""The handle's internal vertex orders against their definitions.  Reverse Cuthill-McKee is
searched on the device when the graph is in the search kernel's scope (at least 16,384 vertices,
degrees up to 254, levels that fit its shared-memory buffers, a level budget) and on the host
otherwise; either way the order is the one defined below, element for element.  Descending
degree is a stable sort."""
import numpy as np
import pytest

from paper_2605_05330_gb300 import inputs


def cuthill_mckee_reversed(rp, ci):
    """Each component is searched breadth-first from its unplaced vertex of least degree (ties
    by id); a vertex's unplaced neighbours follow it in increasing degree (ties in adjacency
    order); the sequence is reversed.  A plain queue, one vertex at a time."""
    n = len(rp) - 1
    deg = np.diff(rp)
    placed = np.zeros(n, bool)
    seq = []
    for s in np.argsort(deg, kind="stable"):
        if placed[s]:
            continue
        placed[s] = True
        head = len(seq)
        seq.append(int(s))
        while head < len(seq):
            u = seq[head]
            head += 1
            new = [int(v) for v in ci[rp[u]:rp[u + 1]] if not placed[v]]
            placed[new] = True
            seq.extend(sorted(new, key=lambda v: deg[v]))  # sorted() is stable
    return np.array(seq[::-1], dtype=np.int32)


def test_reference_order_small_cases():
    # path 0-1-2-3-4: start at 0 (degree 1, lowest id), the path in order, reversed
    g = inputs.small_graph("path5", 5, [(0, 1), (1, 2), (2, 3), (3, 4)])
    assert cuthill_mckee_reversed(g.row_ptr, g.col_idx).tolist() == [4, 3, 2, 1, 0]
    # star centred on 0: start at leaf 1, then the centre, then the other leaves in id order
    g = inputs.small_graph("star5", 5, [(0, 1), (0, 2), (0, 3), (0, 4)])
    assert cuthill_mckee_reversed(g.row_ptr, g.col_idx).tolist() == [4, 3, 2, 0, 1]
    # an isolated vertex (5) first, then the triangle {0, 1, 2} hanging off 3-4, children by degree
    g = inputs.small_graph("mixed", 6, [(0, 1), (1, 2), (0, 2), (2, 3), (3, 4)])
    # degrees 2 2 3 2 1 0: starts 5, then 4; 4 -> 3 -> 2 -> {0, 1}
    assert cuthill_mckee_reversed(g.row_ptr, g.col_idx).tolist() == [1, 0, 2, 3, 4, 5]


@pytest.fixture(scope="module")
def gn():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_05330_gb300 import build
    build.build()
    from paper_2605_05330_gb300 import gn as gnmod
    return gnmod


def _islands():
    """40 small unit-disk graphs and 500 isolated vertices: many components, degree-0 starts."""
    parts = [inputs.unit_disk_graph(500, 2500, 600 + i) for i in range(40)]
    parts.append(inputs.small_graph("isolated", 500, []))
    return inputs.disjoint_union(parts)


# graph, and where its reverse Cuthill-McKee order is computed
CASES = {
    "udg20k": (lambda: inputs.unit_disk_graph(20000, 100000, 5), "device"),
    "udg_1m": (inputs.workload_udg_1m, "device"),
    "islands": (_islands, "device"),
    # too many vertices for the placed-vertex bits beside the level buffers in shared memory
    "udg_islands_450k": (lambda: inputs.disjoint_union(
        [inputs.unit_disk_graph(90000, 450000, 17 + i) for i in range(5)]), "device"),
    # a level wider than the device search's shared-memory buffers
    "er30k_deg3": (lambda: inputs.er_graph(30000, 3.0, 11), "host"),
    # thousands of small components: past the device search's level budget
    "er30k_deg1": (lambda: inputs.er_graph(30000, 1.0, 12), "host"),
    # too few vertices for the device search
    "er3k": (lambda: inputs.er_graph(3000, 6.0, 13), "host"),
    # degrees above the device search's bound
    "ba20k": (lambda: inputs.ba_graph(20000, 5, 14), "host"),
    # no edges: every vertex is its own component, placed before any search
    "edgeless20k": (lambda: inputs.small_graph("edgeless20k", 20000, []), "device"),
    # a star: its centre's degree is above the bound
    "star20k": (lambda: inputs.small_graph("star20k", 20000, [(0, j) for j in range(1, 20000)]), "host"),
}


@pytest.mark.gpu
@pytest.mark.parametrize("case", sorted(CASES))
def test_rcm_order_matches_definition(gn, case):
    import torch
    make, where = CASES[case]
    inst = make()
    args = (torch.from_numpy(inst.row_ptr).cuda(), torch.from_numpy(inst.col_idx).cuda(),
            torch.from_numpy(inst.w).cuda())
    h = gn.Graph(*args, reorder=gn.REORDER_RCM)
    assert h.vertex_order_source() == where
    np.testing.assert_array_equal(h.vertex_order(), cuthill_mckee_reversed(inst.row_ptr, inst.col_idx))
    g = gn.Graph(*args, reorder=gn.REORDER_DEGREE)
    assert g.vertex_order_source() == "host"
    deg = np.diff(inst.row_ptr)
    np.testing.assert_array_equal(g.vertex_order(), np.argsort(-deg, kind="stable").astype(np.int32))
    plain = gn.Graph(*args)
    assert plain.vertex_order_source() == "none"
    np.testing.assert_array_equal(plain.vertex_order(), np.arange(inst.n, dtype=np.int32))


@pytest.mark.gpu
def test_rcm_handle_runs_like_the_oracle(gn):
    """The device-searched order changes only the internal layout: the run follows the oracle."""
    import oracle
    from tests.test_gpu_parity import K_ITERATE, assert_close_rel, fixed_steps, to_np
    inst = _islands()
    g = gn.Graph(inst.row_ptr, inst.col_idx, inst.w, reorder=gn.REORDER_RCM)
    assert g.vertex_order_source() == "device"
    run_kw, pk = fixed_steps(K_ITERATE)
    x, info = g.run(params=gn.default_params(**pk), **run_kw)
    xo, io = oracle.run(inst.row_ptr, inst.col_idx, inst.w, p=oracle.params(**pk), **run_kw)
    assert_close_rel(to_np(x), xo)
