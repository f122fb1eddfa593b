"""Test-side readers for the paper's printed data (tests/golden) and an
independent brute-force classifier built on networkx isomorphism."""
import itertools
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_matrix(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([int(x) for x in line.split()])
    return np.array(rows, dtype=np.int64)


def read_patterns():
    """List of (k, edges[(a,b)] 0-based, {vertex: orbit}) from Fig. node_orbits."""
    pats = []
    for line in open(os.path.join(GOLDEN, "patterns.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        left, right = line.split("|")
        f = left.split()
        k = int(f[1])
        edges = [(int(e[0]) - 1, int(e[1]) - 1) for e in f[2:]]
        labels = {int(t.split(":")[0]) - 1: int(t.split(":")[1]) for t in right.split()}
        pats.append((k, edges, labels))
    return pats


def nx_orbit_table():
    """Orbit number of every vertex of every pattern, from networkx automorphisms."""
    import networkx as nx
    from networkx.algorithms.isomorphism import GraphMatcher
    out = []
    for k, edges, labels in read_patterns():
        h = nx.Graph()
        h.add_nodes_from(range(k))
        h.add_edges_from(edges)
        cls = {v: {v} for v in range(k)}
        for mp in GraphMatcher(h, h).isomorphisms_iter():
            for a, b in mp.items():
                cls[a].add(b)
        orb = [-1] * k
        for v, num in labels.items():
            for x in cls[v]:
                orb[x] = num
        out.append((h, orb))
    return out


def nx_brute_force(g):
    """Induced orbit counts by enumerating every vertex subset of size 2..5,
    testing connectivity and matching against the patterns with networkx."""
    import networkx as nx
    from networkx.algorithms.isomorphism import GraphMatcher
    table = nx_orbit_table()
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    G.add_edges_from(map(tuple, g.edges().tolist()))
    out = np.zeros((g.n, 73), dtype=np.int64)
    for k in range(2, 6):
        for S in itertools.combinations(range(g.n), k):
            sub = G.subgraph(S)
            if not nx.is_connected(sub):
                continue
            for h, orb in table:
                if h.number_of_nodes() != k or h.number_of_edges() != sub.number_of_edges():
                    continue
                gm = GraphMatcher(sub, h)
                if gm.is_isomorphic():
                    for a, b in gm.mapping.items():
                        out[a, orb[b]] += 1
                    break
            else:
                raise AssertionError("unclassified subset")
    return out
