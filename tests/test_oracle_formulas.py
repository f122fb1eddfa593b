"""Pins of the oracle's implementation of the paper's method (Lem.
4vertexorbit, Lem. 4edgeorbit, Thm. 5vertexorbit, Thm. 5-Cycle-Clique, the
induced transform of App. A) against the brute-force definition."""
import numpy as np
import pytest

from paper_1911_10616_gb300 import graphgen as gg
from tests import _paper


def test_noninduced_equations_each_orbit(oracle_mod):
    # every DM equation separately against non-induced brute force
    for seed in range(12):
        rng = np.random.default_rng(seed)
        g = gg.er_gnp(int(rng.integers(8, 13)), float(rng.uniform(0.3, 0.7)), 300 + seed)
        _, dm_bf = oracle_mod.brute_force(g, noninduced=True)
        dm, _ = oracle_mod.formulas(g)
        bad = np.where((dm != dm_bf).any(0))[0]
        assert bad.size == 0, f"orbits {bad.tolist()} disagree"


def test_small_random_graphs_config(oracle_mod):
    # 50 random G(n in [8,30], p in [0.2,0.6]) graphs
    rng = np.random.default_rng(2024)
    for i in range(50):
        n = int(rng.integers(8, 31))
        p = float(rng.uniform(0.2, 0.6))
        g = gg.er_gnp(n, p, 1000 + i)
        _, dim = oracle_mod.formulas(g)
        assert np.array_equal(dim, oracle_mod.brute_force(g)), (n, p)


def test_er_2000_10000(oracle_mod):
    g = gg.er_gnm(2000, 10000, 1)
    _, dim = oracle_mod.formulas(g)
    assert np.array_equal(dim, oracle_mod.brute_force(g))


def test_special_graphs(oracle_mod):
    graphs = [gg.complete(7), gg.star(8), gg.cycle(5), gg.cycle(9), gg.path(8)]
    graphs += [gg.from_edge_list(k, e) for k, e, _ in _paper.read_patterns()]
    for g in graphs:
        _, dim = oracle_mod.formulas(g)
        assert np.array_equal(dim, oracle_mod.brute_force(g))


def test_hubby_graph(oracle_mod):
    # power-law with a dense hub core: exercises 5-cycles / 5-cliques / W4
    g = gg.chung_lu(60, 400, 1.9, 40, 5)
    _, dim = oracle_mod.formulas(g)
    assert np.array_equal(dim, oracle_mod.brute_force(g))


def test_orbit26_worked_example(oracle_mod):
    # Eq. orb26 on the bull H12 itself: each orbit-26 vertex is in exactly one
    # non-induced bull.  On a diamond with a pendant at each chord vertex the
    # diamond shrinkage term 2*DM13 of Eq. orb26 is exercised.
    k, edges, _ = _paper.read_patterns()[12]
    g = gg.from_edge_list(k, edges)
    dm, _ = oracle_mod.formulas(g)
    assert dm[2, 26] == 1 and dm[3, 26] == 1
    g2 = gg.from_edge_list(6, [(0, 1), (0, 2), (1, 2), (1, 3), (2, 3), (1, 4), (2, 5)])
    dm2, _ = oracle_mod.formulas(g2)
    _, dm_bf = oracle_mod.brute_force(g2, noninduced=True)
    assert dm2[1, 26] == dm_bf[1, 26] and dm2[1, 13] == 1


def test_relabel_invariance(oracle_mod):
    g = gg.chung_lu(300, 1500, 2.1, 60, 9)
    _, dim = oracle_mod.formulas(g)
    perm = np.random.default_rng(3).permutation(g.n)
    _, dim2 = oracle_mod.formulas(gg.relabel(g, perm))
    assert np.array_equal(dim2[perm], dim)
