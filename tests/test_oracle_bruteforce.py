"""Pins of the oracle's brute force (the definition) against closed forms,
an independent networkx enumeration, and invariants."""
from math import comb

import numpy as np
import pytest

from paper_1911_10616_gb300 import graphgen as gg
from tests import _paper


def only(vec, expect):
    out = np.zeros(73, np.int64)
    for k, v in expect.items():
        out[k] = v
    return np.array_equal(vec, out), out


@pytest.mark.parametrize("n", [5, 6, 7, 9])
def test_complete_graph(oracle_mod, n):
    dim = oracle_mod.brute_force(gg.complete(n))
    ok, want = only(dim[0], {0: n - 1, 3: comb(n - 1, 2), 14: comb(n - 1, 3), 72: comb(n - 1, 4)})
    assert ok, (dim[0], want)
    assert (dim == dim[0]).all()


@pytest.mark.parametrize("k", [1, 2, 3, 4, 6, 9])
def test_star(oracle_mod, k):
    dim = oracle_mod.brute_force(gg.star(k))
    ok, _ = only(dim[0], {0: k, 2: comb(k, 2), 7: comb(k, 3), 23: comb(k, 4)})
    assert ok, dim[0]
    ok, _ = only(dim[1], {0: 1, 1: k - 1, 6: comb(k - 1, 2), 22: comb(k - 1, 3)})
    assert ok, dim[1]


@pytest.mark.parametrize("n", [6, 7, 10])
def test_long_cycle(oracle_mod, n):
    dim = oracle_mod.brute_force(gg.cycle(n))
    ok, _ = only(dim[0], {0: 2, 1: 2, 2: 1, 4: 2, 5: 2, 15: 2, 16: 2, 17: 1})
    assert ok, dim[0]
    assert (dim == dim[0]).all()


def test_short_cycles(oracle_mod):
    assert only(oracle_mod.brute_force(gg.cycle(3))[0], {0: 2, 3: 1})[0]
    assert only(oracle_mod.brute_force(gg.cycle(4))[0], {0: 2, 1: 2, 2: 1, 8: 1})[0]
    assert only(oracle_mod.brute_force(gg.cycle(5))[0],
                {0: 2, 1: 2, 2: 1, 4: 2, 5: 2, 34: 1})[0]


def test_path(oracle_mod):
    dim = oracle_mod.brute_force(gg.path(7))
    # end vertex: edge, 2-path end, 3-path end, 4-path end
    assert only(dim[0], {0: 1, 1: 1, 4: 1, 15: 1})[0]
    # second vertex: 2-path centre and end, 3-path middle and end, 4-path 16 and 15
    assert only(dim[1], {0: 2, 1: 1, 2: 1, 4: 1, 5: 1, 15: 1, 16: 1})[0]
    # middle vertex 3 of 0..6: the 4-path windows starting at 0, 1, 2 put it
    # second-from-end, centre, second-from-end
    assert only(dim[3], {0: 2, 1: 2, 2: 1, 4: 2, 5: 2, 16: 2, 17: 1})[0]


def test_each_pattern_contains_itself_once(oracle_mod):
    k, orb, _ = oracle_mod.pattern_orbits()
    for j, (kk, edges, _) in enumerate(_paper.read_patterns()):
        g = gg.from_edge_list(kk, edges)
        dim = oracle_mod.brute_force(g)
        lo, hi = {2: (0, 1), 3: (1, 4), 4: (4, 15), 5: (15, 73)}[kk]
        for x in range(kk):
            row = dim[x, lo:hi]
            assert row.sum() == 1 and row[orb[j, x] - lo] == 1, (j, x)


@pytest.mark.parametrize("seed", range(6))
def test_matches_networkx_enumeration(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(6, 9))
    g = gg.er_gnp(n, float(rng.uniform(0.3, 0.7)), seed)
    assert np.array_equal(oracle_mod.brute_force(g), _paper.nx_brute_force(g))


def test_invariants_random(oracle_mod):
    k, orb, sz = oracle_mod.pattern_orbits()
    for seed in range(10):
        g = gg.er_gnp(14, 0.35, 50 + seed)
        dim = oracle_mod.brute_force(g)
        assert (dim >= 0).all()
        assert np.array_equal(dim[:, 0], g.degrees())
        tot = dim.sum(0)
        for j in range(30):
            orbits = sorted(set(orb[j, : k[j]]))
            copies = {tot[o] // sz[o] for o in orbits}
            assert all(tot[o] % sz[o] == 0 for o in orbits)
            assert len(copies) == 1, (j, [tot[o] for o in orbits])
        # relabelling invariance
        perm = np.random.default_rng(seed).permutation(g.n)
        dim2 = oracle_mod.brute_force(gg.relabel(g, perm))
        assert np.array_equal(dim2[perm], dim)


def test_noninduced_equals_A_times_induced(oracle_mod):
    A = oracle_mod.A_matrix()
    for seed in range(5):
        g = gg.er_gnp(11, 0.5, 70 + seed)
        dim, dm = oracle_mod.brute_force(g, noninduced=True)
        assert np.array_equal(dim @ A.T, dm)
