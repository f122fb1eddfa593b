"""Pins of the oracle's edge orbits E0..E11 (Fig. edge_orbits, Lem. 4edgeorbit).

The brute force enumerates non-induced copies by the Definition that follows
Fig. edge_orbits; the formula path applies Lem. 4edgeorbit to the oracle's base
counts.  Both are checked against hand counts on the patterns themselves,
against each other on random graphs, and against the vertex-orbit brute force
(each copy of a pattern has a fixed number of edges in each edge orbit)."""
import numpy as np
import pytest

from paper_1911_10616_gb300 import graphgen as gg

# edge orbit -> (pattern, vertex orbit of one end, of the other, edges of the
# orbit in one copy, symmetric ends); the pattern edge counts are those of
# Fig. edge_orbits (2-path: 2 edges; triangle: 3; 3-path: 2 end + 1 middle;
# 3-star: 3; 4-cycle: 4; paw: 1 + 1 + 2; diamond: 4 + 1; 4-clique: 6)
EDGE_ORBITS = {
    0: (1, 2, 1, 2, False), 1: (2, 3, 3, 3, True), 2: (3, 5, 4, 2, False),
    3: (3, 5, 5, 1, True), 4: (4, 7, 6, 3, False), 5: (5, 8, 8, 4, True),
    6: (6, 11, 9, 1, False), 7: (6, 10, 10, 1, True), 8: (6, 11, 10, 2, False),
    9: (7, 13, 12, 4, False), 10: (7, 13, 13, 1, True), 11: (8, 14, 14, 6, True),
}
# one vertex orbit of each pattern and its size (Fig. node_orbits)
PATTERN_ORBIT = {1: (2, 1), 2: (3, 3), 3: (5, 2), 4: (7, 1), 5: (8, 4), 6: (11, 1),
                 7: (13, 2), 8: (14, 4)}


def slot(g, u, v):
    rp, col = g.rowptr, g.col
    row = col[rp[u]:rp[u + 1]]
    return int(rp[u] + np.searchsorted(row, v))


def test_paw_by_hand(oracle_mod):
    # pendant 0, centre 1, triangle 1-2-3: one paw, nothing else of 4 vertices
    g = gg.from_edge_list(4, [(0, 1), (1, 2), (1, 3), (2, 3)])
    for E in (oracle_mod.edge_orbits_brute(g), oracle_mod.edge_orbits_formula(g)):
        assert E[slot(g, 1, 0), 6] == 1 and E[slot(g, 0, 1), 6] == 0   # pendant edge
        assert E[slot(g, 2, 3), 7] == 1 and E[slot(g, 3, 2), 7] == 1   # opposite the centre
        assert E[slot(g, 1, 2), 8] == 1 and E[slot(g, 2, 1), 8] == 0   # at the centre
        assert E[:, 9:].sum() == 0                                     # no diamond, no K4
        # 2-paths: centre 1 has three neighbours, each edge at 1 lies on two
        assert E[slot(g, 1, 0), 0] == 2 and E[slot(g, 0, 1), 0] == 0
        # the 3-path 0-1-2-3 and 0-1-3-2: edge (1,2) is a middle edge once
        assert E[slot(g, 1, 2), 3] == 1 and E[slot(g, 2, 1), 3] == 1
        # 3-star at 1 with leaves 0, 2, 3: each edge at 1 once
        assert E[slot(g, 1, 0), 4] == 1 and E[slot(g, 0, 1), 4] == 0


def test_path_by_hand(oracle_mod):
    g = gg.path(4)  # 0-1-2-3
    for E in (oracle_mod.edge_orbits_brute(g), oracle_mod.edge_orbits_formula(g)):
        assert E[slot(g, 1, 0), 2] == 1 and E[slot(g, 0, 1), 2] == 0  # end edge, 1 inner
        assert E[slot(g, 1, 2), 3] == 1 and E[slot(g, 2, 1), 3] == 1  # middle edge
        assert E[slot(g, 1, 2), 2] == 0
        assert E[:, [1, 4, 5, 6, 7, 8, 9, 10, 11]].sum() == 0


def test_cliques_closed_forms(oracle_mod):
    for k in (4, 5, 6):
        g = gg.complete(k)
        E = oracle_mod.edge_orbits_brute(g)
        assert (E == E[0]).all()                      # every slot alike
        t = k - 2
        assert E[0, 1] == t and E[0, 11] == (t * (t - 1)) // 2   # triangles, 4-cliques
        assert E[0, 10] == (t * (t - 1)) // 2         # diamonds with the edge as chord
        assert E[0, 5] == 2 * (t * (t - 1)) // 2      # 4-cycles through the edge


def _random_graphs():
    rng = np.random.default_rng(77)
    out = [gg.complete(5), gg.star(6), gg.cycle(4), gg.cycle(6), gg.path(6),
           gg.from_edge_list(5, [(0, 1), (0, 2), (0, 3), (0, 4), (1, 2), (2, 3), (3, 4), (4, 1)])]
    for i in range(25):
        n = int(rng.integers(5, 13))
        out.append(gg.er_gnp(n, float(rng.uniform(0.2, 0.7)), 300 + i))
    return out


def test_brute_equals_lemma(oracle_mod):
    for g in _random_graphs():
        b = oracle_mod.edge_orbits_brute(g)
        f = oracle_mod.edge_orbits_formula(g)
        bad = np.argwhere(b != f)
        assert bad.size == 0, f"{g}: (slot, orbit) {bad[:6].tolist()}"


def test_totals_match_vertex_orbits(oracle_mod):
    # each non-induced copy of a pattern puts a fixed number of edges in each
    # of its edge orbits; the copies are counted independently by the
    # vertex-orbit brute force (sum of DM over one orbit / orbit size)
    for g in _random_graphs()[:12]:
        E = oracle_mod.edge_orbits_brute(g)
        _, dm = oracle_mod.brute_force(g, noninduced=True)
        for i, (pat, _, _, per_copy, sym) in EDGE_ORBITS.items():
            o, size = PATTERN_ORBIT[pat]
            copies = int(dm[:, o].sum()) // size
            assert int(E[:, i].sum()) == copies * per_copy * (2 if sym else 1), (g, i)


def test_symmetric_orbits_agree_across_slots(oracle_mod):
    g = gg.er_gnp(12, 0.5, 9)
    E = oracle_mod.edge_orbits_brute(g)
    rev = np.array([slot(g, int(g.col[s]), u) for u in range(g.n)
                    for s in range(g.rowptr[u], g.rowptr[u + 1])])
    for i, (_, _, _, _, sym) in EDGE_ORBITS.items():
        if sym:
            assert np.array_equal(E[:, i], E[rev, i]), i

