"""Pins of the oracle's pattern/orbit tables and of its derived matrix A
against what the paper prints (Fig. node_orbits, Fig. A, Fig. Ainv)."""
import numpy as np
import pytest

from tests import _paper


def test_tables_consistent(oracle_mod):
    assert oracle_mod.tables_ok()


def test_orbits_match_networkx_automorphisms(oracle_mod):
    # Def. auto: orbits are automorphism classes; networkx computes them
    # independently from the printed edge lists.
    k, orb, sz = oracle_mod.pattern_orbits()
    table = _paper.nx_orbit_table()
    for j, (h, o) in enumerate(table):
        assert k[j] == h.number_of_nodes()
        assert list(orb[j, : k[j]]) == o, f"H{j}"
    # 73 orbits numbered 0..72, each in exactly one pattern
    seen = sorted(x for j in range(30) for x in set(orb[j, : k[j]]))
    assert seen == list(range(73))
    # sizes: e.g. K5 (orbit 72) has all 5 vertices, the star centre (23) one
    assert sz[72] == 5 and sz[23] == 1 and sz[22] == 4 and sz[54] == 3 and sz[55] == 2
    assert sz.sum() == sum(k)


def test_A_four_vertex_block_matches_fig_A(oracle_mod):
    A = oracle_mod.A_matrix()
    figA = _paper.read_matrix("fig_A_4vertex.txt")
    blk = A[4:15, 4:15]
    mask = np.ones_like(figA, dtype=bool)
    mask[5 - 4, 13 - 4] = False          # printed erratum, see the fixture header
    assert np.array_equal(blk[mask], figA[mask])
    assert blk[5 - 4, 13 - 4] == 4


def test_A_inverse_matches_fig_Ainv(oracle_mod):
    A = oracle_mod.A_matrix()[4:15, 4:15]
    inv = np.rint(np.linalg.inv(A.astype(float))).astype(np.int64)
    assert np.array_equal(inv @ A, np.eye(11, dtype=np.int64))
    fig = _paper.read_matrix("fig_Ainv_4vertex.txt")
    figA = _paper.read_matrix("fig_A_4vertex.txt")
    # the printed pair is self-consistent ...
    assert np.array_equal(figA @ fig, np.eye(11, dtype=np.int64))
    # ... and equals ours except in the row of orbit 5, columns 13 and 14
    mask = np.ones_like(fig, dtype=bool)
    mask[1, 9:] = False
    assert np.array_equal(inv[mask], fig[mask])
    assert list(inv[1, 9:]) == [4, -6]


def test_A_structure(oracle_mod):
    A = oracle_mod.A_matrix()
    k, orb, _ = oracle_mod.pattern_orbits()
    size = np.zeros(73, int)
    for j in range(30):
        for x in range(k[j]):
            size[orb[j, x]] = k[j]
    # block diagonal by pattern size, unit upper triangular (orbits are
    # numbered by non-decreasing edge count, App. A)
    for i in range(73):
        assert A[i, i] == 1
        for j in range(73):
            if A[i, j]:
                assert size[i] == size[j] and i <= j
    # 3-vertex block: a triangle vertex is an end of two 2-paths and the
    # centre of one (DM1 = DIM1 + 2 DIM3, DM2 = DIM2 + DIM3)
    assert A[1, 3] == 2 and A[2, 3] == 1 and A[1, 2] == 0
    # K5 at a vertex: C(4,2)*3!... 5-cycles through a vertex of K5 = 12
    assert A[34, 72] == 12
    # K5 contains 5*3 = 15 spanning 4-paths... at a vertex: middle of P5 is
    # any of 5!/2 = 60 Hamiltonian paths with the vertex at the centre: 12
    assert A[17, 72] == 12 and A[15, 72] + A[16, 72] + A[17, 72] == 60
