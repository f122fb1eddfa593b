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

import math

import numpy as np

__all__ = [
    "Graph", "csr_from_pairs", "er_gnm", "er_gnp", "chung_lu", "rmat",
    "barabasi_albert", "random_geometric", "complete", "star", "cycle", "path",
    "from_edge_list", "relabel", "small_graph_batch", "concat_batch",
    "small_graph_batch_tensors", "batch_graph",
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


def _batch_csr_torch(ns, gid, a, b):
    """Per-graph local edges (graph id, a, b) as torch int64 tensors ->
    batch CSR (rowptr_cat int32-bits-of-uint32, col_cat, vtx_off int64,
    edge_off int64), loops and duplicates removed."""
    import torch
    dev = ns.device
    G = ns.numel()
    vtx_off = torch.zeros(G + 1, dtype=torch.int64, device=dev)
    vtx_off[1:] = torch.cumsum(ns, 0)
    keep = a != b
    gid, a, b = gid[keep], a[keep], b[keep]
    lo = torch.minimum(a, b)
    hi = torch.maximum(a, b)
    N = int(vtx_off[-1].item())
    key = torch.unique((vtx_off[gid] + lo) * N + (vtx_off[gid] + hi))
    ga = key // N
    gb = key % N
    src = torch.cat([ga, gb])
    dst = torch.cat([gb, ga])
    order = torch.argsort(src * N + dst)
    src, dst = src[order], dst[order]
    deg = torch.bincount(src, minlength=N)
    grow = torch.zeros(N + 1, dtype=torch.int64, device=dev)
    grow[1:] = torch.cumsum(deg, 0)
    edge_off = grow[vtx_off]
    reps = ns + 1
    gid_rows = torch.repeat_interleave(torch.arange(G, device=dev), reps)
    first_row = torch.zeros(G, dtype=torch.int64, device=dev)
    first_row[1:] = torch.cumsum(reps, 0)[:-1]
    local = torch.arange(gid_rows.numel(), device=dev) - first_row[gid_rows]
    rowptr_cat = grow[vtx_off[gid_rows] + local] - edge_off[gid_rows]
    gid_slots = torch.repeat_interleave(torch.arange(G, device=dev), edge_off[1:] - edge_off[:-1])
    col_cat = dst - vtx_off[gid_slots]
    return (rowptr_cat.to(torch.int32), col_cat.to(torch.int32), vtx_off, edge_off)


def small_graph_batch_tensors(count: int, nmin: int, nmax: int, seed: int, device="cpu"):
    """The many-small-graphs workload in batch CSR form, generated with torch
    on `device` (seeded): graph g has n_g ~ U[nmin, nmax] vertices;
    g % 3 == 0: Erdos-Renyi with average degree ~ U[4, 12] (distinct uniform
    pairs); g % 3 == 1: Barabasi-Albert, each new vertex joins m0 ~ U{2..5}
    distinct targets drawn in proportion to degree (seeded by a star on the
    first m0 vertices); g % 3 == 2: 2-D random geometric graph in the unit
    square with radius sqrt(6 / (pi (n-1))) (average degree about 6).
    Returns (rowptr_cat, col_cat, vtx_off, edge_off) torch tensors; ids are
    uint32 bit patterns in int32 tensors."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    dev = torch.device(device)
    rnd = lambda *shape: torch.rand(*shape, generator=gen, device=dev)
    ns = (nmin + (rnd(count) * (nmax - nmin + 1)).long()).clamp_(nmin, nmax)
    fam = torch.arange(count, device=dev) % 3
    pg, pa, pb = [], [], []

    # Erdos-Renyi
    er = torch.nonzero(fam == 0).flatten()
    if er.numel():
        n_er = ns[er]
        deg = 4.0 + 8.0 * rnd(er.numel())
        want = torch.minimum(torch.round(deg * n_er / 2).long(), n_er * (n_er - 1) // 2)
        draws = (want.double() * 1.4 + 8).long()
        gid = torch.repeat_interleave(er, draws)
        nn = ns[gid]
        x = (rnd(gid.numel()) * nn).long()
        y = (rnd(gid.numel()) * nn).long()
        ok = x != y
        gid, x, y = gid[ok], x[ok], y[ok]
        lo, hi = torch.minimum(x, y), torch.maximum(x, y)
        key = torch.unique((gid * 1024 + lo) * 1024 + hi)
        gid, lo, hi = key // (1024 * 1024), (key // 1024) % 1024, key % 1024
        pri = rnd(gid.numel())
        order = torch.argsort(gid.double() * 2.0 + pri)  # by graph, random within
        gid, lo, hi = gid[order], lo[order], hi[order]
        cnt = torch.bincount(gid, minlength=count)
        start = torch.zeros(count, dtype=torch.long, device=dev)
        start[1:] = torch.cumsum(cnt, 0)[:-1]
        rank = torch.arange(gid.numel(), device=dev) - start[gid]
        cap = torch.zeros(count, dtype=torch.long, device=dev)
        cap[er] = want
        sel = rank < cap[gid]
        pg.append(gid[sel]); pa.append(lo[sel]); pb.append(hi[sel])

    # Barabasi-Albert, all graphs grown in lock-step
    ba = torch.nonzero(fam == 1).flatten()
    if ba.numel():
        B = ba.numel()
        m0 = 2 + (rnd(B) * 4).long().clamp_(0, 3)
        nb = ns[ba]
        L = int((2 * m0 * nb).max().item()) + 16
        rep = torch.zeros((B, L), dtype=torch.long, device=dev)
        ln = torch.zeros(B, dtype=torch.long, device=dev)
        rows = torch.arange(B, device=dev)
        for k in range(1, 5):  # seed star: 0 - k for k < m0
            s = rows[m0 > k]
            pg.append(ba[s]); pa.append(torch.zeros_like(s)); pb.append(torch.full_like(s, k))
            rep[s, ln[s]] = 0
            rep[s, ln[s] + 1] = k
            ln[s] += 2
        kcol = torch.arange(5, device=dev)
        for t in range(2, int(nb.max().item())):
            act = rows[(nb > t) & (m0 <= t)]
            if act.numel() == 0:
                continue
            k = m0[act]
            need = kcol[None, :] < k[:, None]                 # (A, 5)
            tg = torch.full((act.numel(), 5), -1, dtype=torch.long, device=dev)
            todo = need.clone()
            for _ in range(64):
                if not bool(todo.any()):
                    break
                idx = (rnd(act.numel(), 5) * ln[act][:, None]).long()
                cand = torch.gather(rep[act], 1, idx)
                tg = torch.where(todo, cand, tg)
                # a slot is a duplicate if an earlier slot of its row holds the same target
                same = (tg[:, :, None] == tg[:, None, :]) & need[:, :, None] & need[:, None, :]
                earlier = torch.tril(torch.ones(5, 5, dtype=torch.bool, device=dev), -1)
                todo = (same & earlier[None]).any(2)
            r_i, c_i = torch.nonzero(need, as_tuple=True)
            gsel = act[r_i]
            pg.append(ba[gsel]); pa.append(torch.full_like(gsel, t)); pb.append(tg[r_i, c_i])
            pos = ln[gsel] + 2 * c_i
            rep[gsel, pos] = tg[r_i, c_i]
            rep[gsel, pos + 1] = t
            ln[act] += 2 * k

    # random geometric, grouped by size
    rg = torch.nonzero(fam == 2).flatten()
    if rg.numel():
        sizes = torch.unique(ns[rg]).tolist()
        for nval in sizes:
            grp = rg[ns[rg] == nval]
            n = int(nval)
            pts = rnd(grp.numel(), n, 2)
            d2 = torch.cdist(pts.double(), pts.double()) ** 2
            r2 = 6.0 / (math.pi * (n - 1))
            iu = torch.triu(torch.ones(n, n, dtype=torch.bool, device=dev), 1)
            gi, ii, jj = torch.nonzero((d2 <= r2) & iu[None], as_tuple=True)
            pg.append(grp[gi]); pa.append(ii); pb.append(jj)

    gid = torch.cat(pg) if pg else torch.zeros(0, dtype=torch.long, device=dev)
    a = torch.cat(pa) if pa else torch.zeros(0, dtype=torch.long, device=dev)
    b = torch.cat(pb) if pb else torch.zeros(0, dtype=torch.long, device=dev)
    return _batch_csr_torch(ns, gid.long(), a.long(), b.long())


def batch_graph(rowptr_cat, col_cat, vtx_off, edge_off, g: int) -> Graph:
    """Graph g of a batch (numpy arrays or CPU tensors) in CSR form."""
    rowptr_cat, col_cat, vtx_off, edge_off = (np.asarray(x) for x in
                                              (rowptr_cat, col_cat, vtx_off, edge_off))
    n = int(vtx_off[g + 1] - vtx_off[g])
    r0 = int(vtx_off[g] + g)
    rp = rowptr_cat[r0:r0 + n + 1].astype(np.uint32).astype(np.int64)
    col = col_cat[int(edge_off[g]):int(edge_off[g + 1])].astype(np.uint32)
    return Graph(n, rp, col)
