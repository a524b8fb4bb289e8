"""Seeded synthetic inputs for Graph Normalization workloads.

This module holds no arithmetic of the method itself: it draws graphs (as
symmetric, row-sorted int32 CSR), vertex weights and raw uniform random
numbers.  It is the one module that both the CUDA path and the FP64 oracle
consume, so that both see identical inputs.

The paper's datasets (AVR, MSCD) are not available; these generators stand in
for them with the shapes its workloads have (Sec. 6 and its appendix tables:
1K-882K vertices, 2.4K-344M edges, sparse conflict graphs):

* Erdos-Renyi G(n, p) with p = avg_deg / (n - 1);
* unit-disk graphs (uniform points in the unit square, radius bisected to a
  target edge count, random vertex labels);
* Barabasi-Albert preferential attachment (heavy-tailed degrees);
* assignment conflict graphs (the line graph of K_{k,k}: cells of a k x k
  matrix, adjacent when they share a row or a column; Sec. 2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 1234


@dataclass
class GraphInstance:
    name: str
    row_ptr: np.ndarray      # int32 [n+1]
    col_idx: np.ndarray      # int32 [nnz], each row strictly increasing
    w: np.ndarray            # float32 [n], > 0
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return len(self.row_ptr) - 1

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])


def rng_for(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def csr_from_edges(n: int, a: np.ndarray, b: np.ndarray):
    """Symmetric, duplicate-free, self-loop-free CSR from an undirected edge list."""
    a = np.asarray(a, dtype=np.int64)
    b = np.asarray(b, dtype=np.int64)
    keep = a != b
    a, b = a[keep], b[keep]
    src = np.concatenate([a, b])
    dst = np.concatenate([b, a])
    key = np.unique(src * n + dst)
    src = key // n
    dst = key % n
    counts = np.bincount(src, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] > np.iinfo(np.int32).max:
        raise ValueError("graph too large for int32 CSR")
    return row_ptr.astype(np.int32), dst.astype(np.int32)


def er_edges(n: int, avg_deg: float, rng: np.random.Generator):
    """G(n, p), p = avg_deg/(n-1): a Binomial number of distinct uniform vertex pairs."""
    if n < 2:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    pairs = n * (n - 1) // 2
    p = min(1.0, avg_deg / (n - 1))
    m = int(rng.binomial(pairs, p))
    keys = np.zeros(0, dtype=np.int64)
    while keys.size < m:
        need = m - keys.size
        i = rng.integers(0, n, size=need + need // 8 + 16)
        j = rng.integers(0, n, size=i.size)
        ok = i != j
        lo = np.minimum(i[ok], j[ok])
        hi = np.maximum(i[ok], j[ok])
        new = lo * n + hi
        keys = np.unique(np.concatenate([keys, new]))
    if keys.size > m:
        keys = rng.permutation(keys)[:m]
    return keys // n, keys % n


def er_graph(n: int, avg_deg: float, seed: int, w_lo=1.0, w_hi=100.0, name=None) -> GraphInstance:
    rng = rng_for(seed)
    a, b = er_edges(n, avg_deg, rng)
    rp, ci = csr_from_edges(n, a, b)
    w = rng.uniform(w_lo, w_hi, size=n).astype(np.float32)
    return GraphInstance(name or f"er_n{n}_d{avg_deg:g}", rp, ci, w,
                         {"kind": "er", "seed": seed, "avg_deg": avg_deg})


def _udg_pairs(pts: np.ndarray, r: float):
    from scipy.spatial import cKDTree
    tree = cKDTree(pts)
    return tree.query_pairs(r, output_type="ndarray")


def udg_radius(pts: np.ndarray, target_edges: int, rel_tol: float = 0.002, max_steps: int = 40):
    """Bisect the radius so that the unit-disk graph of pts has target_edges edges (+-rel_tol)."""
    from scipy.spatial import cKDTree
    n = len(pts)
    tree = cKDTree(pts)
    r0 = math.sqrt(2.0 * target_edges / (math.pi * n * max(n - 1, 1)))
    lo, hi = 0.5 * r0, 2.0 * r0
    r = r0
    for _ in range(max_steps):
        cnt = (int(tree.count_neighbors(tree, r)) - n) // 2
        if abs(cnt - target_edges) <= rel_tol * target_edges:
            break
        if cnt < target_edges:
            lo = r
        else:
            hi = r
        r = 0.5 * (lo + hi)
    return r


def unit_disk_graph(n: int, target_edges: int, seed: int, weights: str = "lognormal",
                    name=None) -> GraphInstance:
    """Uniform points in [0,1]^2, edge iff distance <= r, r bisected to target_edges.

    Vertex labels are the (random) draw order; weights lognormal(0, 1) by default."""
    rng = rng_for(seed)
    pts = rng.random((n, 2))
    r = udg_radius(pts, target_edges)
    pr = _udg_pairs(pts, r)
    rp, ci = csr_from_edges(n, pr[:, 0], pr[:, 1])
    if weights == "lognormal":
        w = rng.lognormal(0.0, 1.0, size=n).astype(np.float32)
    else:
        w = rng.uniform(1.0, 100.0, size=n).astype(np.float32)
    return GraphInstance(name or f"udg_n{n}", rp, ci, w,
                         {"kind": "udg", "seed": seed, "radius": r, "edges": int(ci.size // 2)})


def ba_graph(n: int, m: int, seed: int, name=None) -> GraphInstance:
    """Barabasi-Albert: a star on m+1 vertices, then each new vertex links to m distinct
    earlier vertices drawn with probability proportional to degree.  Weights U[1,100]."""
    rng = rng_for(seed)
    n_edges = m + (n - m - 1) * m
    ea = np.empty(n_edges, dtype=np.int64)
    eb = np.empty(n_edges, dtype=np.int64)
    ends = np.empty(2 * n_edges, dtype=np.int64)   # every edge endpoint: degree-weighted urn
    ea[:m] = 0
    eb[:m] = np.arange(1, m + 1)
    ends[0:2 * m:2] = 0
    ends[1:2 * m:2] = np.arange(1, m + 1)
    e = m
    draws = rng.random((max(n - m - 1, 0), 3 * m))
    extra = rng_for(seed + 7919)
    for t in range(m + 1, n):
        L = 2 * e
        cand = ends[(draws[t - m - 1] * L).astype(np.int64)]
        chosen = []
        seen = set()
        for c in cand.tolist():
            if c not in seen:
                seen.add(c)
                chosen.append(c)
                if len(chosen) == m:
                    break
        while len(chosen) < m:
            c = int(ends[extra.integers(0, L)])
            if c not in seen:
                seen.add(c)
                chosen.append(c)
        ea[e:e + m] = t
        eb[e:e + m] = chosen
        ends[2 * e:2 * (e + m):2] = t
        ends[2 * e + 1:2 * (e + m):2] = chosen
        e += m
    rp, ci = csr_from_edges(n, ea, eb)
    w = rng.uniform(1.0, 100.0, size=n).astype(np.float32)
    return GraphInstance(name or f"ba_n{n}_m{m}", rp, ci, w, {"kind": "ba", "seed": seed, "m": m})


def rook_csr(k: int):
    """CSR of the assignment conflict graph L(K_{k,k}): vertex r*k + c is cell (r, c);
    two cells are adjacent iff they share a row or a column (Sec. 2)."""
    idx = np.arange(k * k)
    r = idx // k
    c = idx % k
    same = (r[:, None] == r[None, :]) | (c[:, None] == c[None, :])
    np.fill_diagonal(same, False)
    src, dst = np.nonzero(same)
    counts = np.bincount(src, minlength=k * k)
    rp = np.zeros(k * k + 1, dtype=np.int32)
    np.cumsum(counts, out=rp[1:])
    return rp, dst.astype(np.int32)


def assignment_graph(k: int, seed: int, name=None) -> GraphInstance:
    """k x k assignment instance: cost ~ U[0,1], vertex weight w = 2 - cost in (1, 2]."""
    rng = rng_for(seed)
    cost = rng.random((k, k))
    rp, ci = rook_csr(k)
    w = (2.0 - cost).astype(np.float32).reshape(-1)
    return GraphInstance(name or f"assign_k{k}", rp, ci, w,
                         {"kind": "assignment", "seed": seed, "k": k,
                          "cost": (2.0 - w.astype(np.float64)).reshape(k, k)})


def uniforms(n: int, seed: int) -> np.ndarray:
    """Raw U(0,1) float32 numbers in (0, 1) for the random simplex start (passed to both sides)."""
    u = rng_for(seed).random(n).astype(np.float32)
    return np.clip(u, np.float32(1e-7), np.float32(1.0 - 6e-8))


def normal(n: int, seed: int) -> np.ndarray:
    return rng_for(seed).standard_normal(n).astype(np.float32)


# ---------------------------------------------------------------------------------------------
# workload recipes


def workload_er_small(seed: int = SEED_BASE) -> GraphInstance:
    """ER n=2000, average degree 10, w ~ U[1,100]."""
    return er_graph(2000, 10.0, seed, name="er_n2000_d10")


def workload_udg_1m(seed: int = SEED_BASE, n: int = 200_000, edges: int = 1_000_000) -> GraphInstance:
    """Unit-disk n=200,000, |E| ~ 1.0M, w ~ lognormal(0,1), random labels."""
    return unit_disk_graph(n, edges, seed, name=f"udg_n{n}_e{edges}")


def workload_ba_1m(seed: int = SEED_BASE + 1, n: int = 200_000, m: int = 5) -> GraphInstance:
    """Barabasi-Albert n=200,000, m=5 (|E| ~ 1.0M), w ~ U[1,100]."""
    return ba_graph(n, m, seed, name=f"ba_n{n}_m{m}")


def batch_sizes(count: int, seed: int = SEED_BASE, n_lo=64, n_hi=4096, k_lo=8, k_hi=64):
    """Instance recipe of the batched workload: n log-uniform in [n_lo, n_hi]; even ids are
    ER (average degree U[6,16]), odd ids assignment graphs with k = clamp(round(sqrt(n)))."""
    rng = rng_for(seed)
    n = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=count))
    deg = rng.uniform(6.0, 16.0, size=count)
    out = []
    for i in range(count):
        if i % 2 == 0:
            out.append(("er", int(round(n[i])), float(deg[i])))
        else:
            k = int(min(max(round(math.sqrt(n[i])), k_lo), k_hi))
            out.append(("assignment", k, 0.0))
    return out


def workload_batch(count: int = 4096, seed: int = SEED_BASE, k_hi: int = 64):
    """The batched workload: `count` mixed ER / assignment instances (seed base + id each)."""
    insts = []
    for i, (kind, size, deg) in enumerate(batch_sizes(count, seed, k_hi=k_hi)):
        if kind == "er":
            insts.append(er_graph(size, deg, seed + 1 + i, name=f"b{i}_er{size}"))
        else:
            insts.append(assignment_graph(size, seed + 1 + i, name=f"b{i}_as{size}"))
    return insts


def batch_specs(count: int = 4096, seed: int = SEED_BASE, k_hi: int = 64):
    """The batched workload without edge lists for the assignment instances: ER instances as
    GraphInstance, assignment instances as ("assignment", k, w, cost) with w = 2 - cost."""
    out = []
    for i, (kind, size, deg) in enumerate(batch_sizes(count, seed, k_hi=k_hi)):
        if kind == "er":
            out.append(er_graph(size, deg, seed + 1 + i, name=f"b{i}_er{size}"))
        else:
            rng = rng_for(seed + 1 + i)
            cost = rng.random((size, size))
            w = (2.0 - cost).astype(np.float32).reshape(-1)
            out.append(("assignment", size, w, (2.0 - w.astype(np.float64)).reshape(size, size)))
    return out


def assignment_instance(spec) -> GraphInstance:
    """The CSR form of an ("assignment", k, w, cost) spec."""
    _, k, w, cost = spec
    rp, ci = rook_csr(k)
    return GraphInstance(f"assign_k{k}", rp, ci, np.asarray(w, np.float32),
                         {"kind": "assignment", "k": k, "cost": cost})


def workload_diff(seed: int = SEED_BASE, n: int = 50_000, avg_deg: float = 12.0):
    """Differentiable workload: ER n=50,000 average degree 12, w ~ U[1,100], g ~ N(0,1)."""
    g = er_graph(n, avg_deg, seed, name=f"er_n{n}_d{avg_deg:g}")
    return g, normal(n, seed + 99)


def bfs_ball(inst: GraphInstance, root: int, size: int) -> GraphInstance:
    """Induced subgraph on the first `size` vertices reached by BFS from root (CSR order)."""
    rp, ci = inst.row_ptr, inst.col_idx
    order = [root]
    seen = {root}
    head = 0
    while head < len(order) and len(order) < size:
        u = order[head]
        head += 1
        for j in ci[rp[u]:rp[u + 1]].tolist():
            if j not in seen:
                seen.add(j)
                order.append(j)
                if len(order) == size:
                    break
    verts = np.array(sorted(order), dtype=np.int64)
    pos = -np.ones(inst.n, dtype=np.int64)
    pos[verts] = np.arange(len(verts))
    a, b = [], []
    for li, u in enumerate(verts.tolist()):
        nb = ci[rp[u]:rp[u + 1]]
        keep = pos[nb] >= 0
        a.extend([li] * int(keep.sum()))
        b.extend(pos[nb[keep]].tolist())
    rp2, ci2 = csr_from_edges(len(verts), np.array(a, dtype=np.int64), np.array(b, dtype=np.int64))
    return GraphInstance(f"{inst.name}_ball{size}", rp2, ci2, inst.w[verts].copy(),
                         {"kind": "bfs_ball", "root": root, "verts": verts})


def disjoint_union(parts):
    """Block-diagonal union of several instances (component independence, Sec. 2 iii)."""
    rps, cis, ws = [], [], []
    off_v = 0
    off_e = 0
    for g in parts:
        rps.append(g.row_ptr[:-1].astype(np.int64) + off_e)
        cis.append(g.col_idx.astype(np.int64) + off_v)
        ws.append(g.w)
        off_v += g.n
        off_e += g.nnz
    rp = np.concatenate(rps + [np.array([off_e])]).astype(np.int32)
    ci = np.concatenate(cis).astype(np.int32) if cis else np.zeros(0, np.int32)
    return GraphInstance("union", rp, ci, np.concatenate(ws).astype(np.float32), {"kind": "union"})


def small_graph(name: str, n: int, edges, w=None) -> GraphInstance:
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2) if len(edges) else np.zeros((0, 2), np.int64)
    rp, ci = csr_from_edges(n, e[:, 0], e[:, 1])
    w = np.ones(n, np.float32) if w is None else np.asarray(w, dtype=np.float32)
    return GraphInstance(name, rp, ci, w, {"kind": "small"})
