"""Seeded synthetic graph generators.

These produce the *inputs* of the orbit counter and nothing else: every graph
is simple and undirected, stored as CSR with sorted rows (``rowptr`` int64 of
length n+1, ``col`` uint32 of length 2m).  No orbit-counting arithmetic lives
here, so both the CUDA path and the CPU oracle can draw their inputs from this
module without sharing any of the method.

Workload families (the paper evaluates on SNAP / Network Repository / KONECT
graphs, Sec. 6; those datasets are not available offline, so these seeded
generators stand in for them):

* ``er_gnm`` / ``er_gnp`` -- Erdos-Renyi.
* ``chung_lu`` -- power-law expected-degree graphs (web / social shapes).
* ``rmat`` -- Kronecker-style R-MAT graphs.
* ``barabasi_albert`` / ``random_geometric`` -- small-graph families used by
  the many-small-graphs batch.
* closed-form families (complete, star, cycle, path) used by pins.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "Graph", "csr_from_pairs", "er_gnm", "er_gnp", "chung_lu", "rmat",
    "barabasi_albert", "random_geometric", "complete", "star", "cycle", "path",
    "from_edge_list", "relabel", "small_graph_batch", "concat_batch",
]


class Graph:
    """Simple undirected graph in CSR form with sorted rows."""

    __slots__ = ("n", "rowptr", "col")

    def __init__(self, n: int, rowptr: np.ndarray, col: np.ndarray):
        self.n = int(n)
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.uint32)

    @property
    def m(self) -> int:
        return int(self.col.shape[0] // 2)

    def degrees(self) -> np.ndarray:
        return np.diff(self.rowptr)

    def edges(self) -> np.ndarray:
        """(m, 2) array of undirected edges u < v."""
        src = np.repeat(np.arange(self.n, dtype=np.int64), self.degrees())
        dst = self.col.astype(np.int64)
        keep = src < dst
        return np.stack([src[keep], dst[keep]], axis=1)

    def __repr__(self) -> str:
        d = self.degrees()
        dmax = int(d.max()) if self.n else 0
        return f"Graph(n={self.n}, m={self.m}, dmax={dmax})"


def csr_from_pairs(n: int, u: np.ndarray, v: np.ndarray, cap: int | None = None,
                   seed: int = 0) -> Graph:
    """Symmetrise, drop self-loops and duplicates, optionally cap degrees.

    The degree cap drops excess edges in a deterministic (seeded) order: edges
    are ranked at each endpoint in a seeded random order and an edge is kept
    only if it ranks below ``cap`` at both endpoints.
    """
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    keep = u != v
    u, v = u[keep], v[keep]
    a = np.minimum(u, v)
    b = np.maximum(u, v)
    key = np.unique(a * np.int64(n) + b)
    a = key // n
    b = key % n
    if cap is not None and key.size:
        rng = np.random.default_rng(np.uint64(seed) + np.uint64(0x9E3779B9))
        order = rng.permutation(key.size)
        # rank of each edge among the edges of each endpoint, in seeded order
        ends = np.concatenate([a, b])
        eid = np.concatenate([np.arange(key.size), np.arange(key.size)])
        pri = np.concatenate([order, order])
        srt = np.lexsort((pri, ends))
        ends_s = ends[srt]
        starts = np.searchsorted(ends_s, ends_s, side="left")
        rank = np.empty_like(srt)
        rank[srt] = np.arange(srt.size) - starts
        ok = np.ones(key.size, dtype=bool)
        np.logical_and.at(ok, eid, rank < cap)
        a, b = a[ok], b[ok]
    src = np.concatenate([a, b])
    dst = np.concatenate([b, a])
    srt = np.lexsort((dst, src))
    src, dst = src[srt], dst[srt]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(src, minlength=n), out=rowptr[1:])
    return Graph(n, rowptr, dst.astype(np.uint32))


def from_edge_list(n: int, edges) -> Graph:
    e = np.asarray(list(edges), dtype=np.int64).reshape(-1, 2)
    return csr_from_pairs(n, e[:, 0], e[:, 1])


def relabel(g: Graph, perm: np.ndarray) -> Graph:
    """Graph with vertex x renamed perm[x]."""
    e = g.edges()
    perm = np.asarray(perm, dtype=np.int64)
    return csr_from_pairs(g.n, perm[e[:, 0]], perm[e[:, 1]])


def er_gnm(n: int, m: int, seed: int) -> Graph:
    """G(n, m): m distinct uniform pairs, drawn in seeded order."""
    rng = np.random.default_rng(seed)
    maxm = n * (n - 1) // 2
    if m > maxm:
        raise ValueError("m too large for n")
    got = np.empty(0, dtype=np.int64)
    while got.size < m:
        k = int((m - got.size) * 1.3) + 16
        x = rng.integers(0, n, size=k, dtype=np.int64)
        y = rng.integers(0, n, size=k, dtype=np.int64)
        ok = x != y
        key = np.minimum(x[ok], y[ok]) * n + np.maximum(x[ok], y[ok])
        allk = np.concatenate([got, key])
        _, first = np.unique(allk, return_index=True)
        got = allk[np.sort(first)]
    got = got[:m]
    return csr_from_pairs(n, got // n, got % n)


def er_gnp(n: int, p: float, seed: int) -> Graph:
    rng = np.random.default_rng(seed)
    iu, ju = np.triu_indices(n, k=1)
    keep = rng.random(iu.size) < p
    return csr_from_pairs(n, iu[keep], ju[keep])


def _powerlaw_weights(n: int, m: int, exponent: float, cap: float) -> np.ndarray:
    """Expected degrees w_i = c (i+1)^(-1/(gamma-1)) capped, with sum 2m."""
    alpha = 1.0 / (exponent - 1.0)
    base = np.arange(1, n + 1, dtype=np.float64) ** (-alpha)
    lo, hi = 0.0, 2.0 * m / base.sum() * 1e6
    for _ in range(200):
        c = 0.5 * (lo + hi)
        s = np.minimum(c * base, cap).sum()
        if s < 2.0 * m:
            lo = c
        else:
            hi = c
    return np.minimum(hi * base, cap)


def chung_lu(n: int, m: int, exponent: float, cap: int, seed: int) -> Graph:
    """Chung-Lu graph: ~m edges, expected degrees power-law with ``exponent``,
    weights capped at ``cap`` and realised degrees hard-capped at ``cap``."""
    rng = np.random.default_rng(seed)
    w = _powerlaw_weights(n, m, exponent, float(cap))
    w = w[rng.permutation(n)]
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    u = np.searchsorted(cdf, rng.random(m), side="right")
    v = np.searchsorted(cdf, rng.random(m), side="right")
    u = np.minimum(u, n - 1)
    v = np.minimum(v, n - 1)
    return csr_from_pairs(n, u, v, cap=cap, seed=seed)


def rmat(scale: int, edge_factor: int, a: float, b: float, c: float,
         seed: int, cap: int | None = None) -> Graph:
    """R-MAT graph with 2^scale vertices and edge_factor * 2^scale draws."""
    rng = np.random.default_rng(seed)
    n = 1 << scale
    m = edge_factor * n
    u = np.zeros(m, dtype=np.int64)
    v = np.zeros(m, dtype=np.int64)
    for lvl in range(scale):
        r = rng.random(m)
        bit_u = r >= a + b                     # quadrants c, d
        bit_v = ((r >= a) & (r < a + b)) | (r >= a + b + c)   # quadrants b, d
        u |= bit_u.astype(np.int64) << lvl
        v |= bit_v.astype(np.int64) << lvl
    perm = rng.permutation(n)
    return csr_from_pairs(n, perm[u], perm[v], cap=cap, seed=seed)


def barabasi_albert(n: int, m0: int, seed: int) -> Graph:
    """Preferential attachment: each new vertex joins m0 distinct targets."""
    rng = np.random.default_rng(seed)
    m0 = max(1, min(m0, n - 1))
    us, vs = [], []
    repeated = list(range(m0))       # start: a star-free seed set of m0 vertices
    for x in range(m0, n):
        targets = set()
        while len(targets) < m0:
            targets.add(repeated[int(rng.integers(0, len(repeated)))])
        for t in targets:
            us.append(x)
            vs.append(t)
        repeated.extend(targets)
        repeated.extend([x] * m0)
    return csr_from_pairs(n, np.array(us), np.array(vs))


def random_geometric(n: int, radius: float, seed: int) -> Graph:
    rng = np.random.default_rng(seed)
    p = rng.random((n, 2))
    d2 = ((p[:, None, :] - p[None, :, :]) ** 2).sum(-1)
    iu, ju = np.triu_indices(n, k=1)
    keep = d2[iu, ju] <= radius * radius
    return csr_from_pairs(n, iu[keep], ju[keep])


def complete(n: int) -> Graph:
    iu, ju = np.triu_indices(n, k=1)
    return csr_from_pairs(n, iu, ju)


def star(k: int) -> Graph:
    """Centre 0 joined to leaves 1..k."""
    return csr_from_pairs(k + 1, np.zeros(k, dtype=np.int64), np.arange(1, k + 1))


def cycle(n: int) -> Graph:
    x = np.arange(n)
    return csr_from_pairs(n, x, (x + 1) % n)


def path(n: int) -> Graph:
    x = np.arange(n - 1)
    return csr_from_pairs(n, x, x + 1)


def small_graph_batch(count: int, nmin: int, nmax: int, seed: int):
    """Many small graphs: a third each ER (average degree 4..12), BA (m0 in
    2..5) and 2-D random geometric (radius for average degree 6).

    Returns a list of Graph objects (used for modest counts; the large batch
    workload goes through ``concat_batch`` the same way)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(nmin, nmax + 1))
        fam = i % 3
        s = int(rng.integers(0, 2**31 - 1))
        if fam == 0:
            deg = float(rng.uniform(4.0, 12.0))
            m = min(int(round(deg * n / 2)), n * (n - 1) // 2)
            out.append(er_gnm(n, m, s))
        elif fam == 1:
            out.append(barabasi_albert(n, int(rng.integers(2, 6)), s))
        else:
            r = float(np.sqrt(6.0 / (np.pi * (n - 1))))
            out.append(random_geometric(n, r, s))
    return out


def concat_batch(graphs):
    """Concatenate graphs: per-graph local row offsets and local vertex ids.

    Returns (rowptr_cat uint32[sum(n_g+1)], col_cat uint32[sum 2m_g],
    vtx_off int64[G+1], edge_off int64[G+1])."""
    G = len(graphs)
    vtx_off = np.zeros(G + 1, dtype=np.int64)
    edge_off = np.zeros(G + 1, dtype=np.int64)
    for i, g in enumerate(graphs):
        vtx_off[i + 1] = vtx_off[i] + g.n
        edge_off[i + 1] = edge_off[i] + g.col.shape[0]
    rowptr_cat = np.concatenate([g.rowptr.astype(np.uint32) for g in graphs]) if G else np.zeros(0, np.uint32)
    col_cat = np.concatenate([g.col for g in graphs]) if G else np.zeros(0, np.uint32)
    return rowptr_cat, col_cat, vtx_off, edge_off
