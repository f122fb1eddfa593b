"""The oracle's 4-vertex-orbit mode (orbits 0..14, Thm. 4orbit) against the
brute-force definition and against the full method's first 15 columns."""
import numpy as np

from paper_1911_10616_gb300 import graphgen as gg


def _graphs():
    rng = np.random.default_rng(78)
    out = [gg.complete(5), gg.star(6), gg.cycle(4), gg.path(6)]
    for i in range(12):
        out.append(gg.er_gnp(int(rng.integers(5, 14)), float(rng.uniform(0.2, 0.7)), 500 + i))
    return out + [gg.chung_lu(800, 4000, 2.1, 60, 2)]


def test_four_vertex_only_mode(oracle_mod):
    for g in _graphs():
        got = oracle_mod.formulas4(g)
        assert np.array_equal(got, oracle_mod.formulas(g)[1][:, :15]), g
        if g.n <= 14:
            assert np.array_equal(got, oracle_mod.brute_force(g)[:, :15]), g
