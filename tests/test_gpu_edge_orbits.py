"""Parity of evoke_edge_orbit_counts (E0..E11 per slot, Lem. 4edgeorbit) with
the oracle, bit-exact, through the C ABI."""
import numpy as np
import pytest

from paper_1911_10616_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1911_10616_gb300 as ev
    ev.load()
    return ev


def gpu_edge_orbits(ev, g):
    rp, col = ev.to_device(g)
    return ev.edge_orbit_counts(rp, col, g.n, g.m).cpu().numpy()


def test_tiny_graphs_against_definition(ev, oracle_mod):
    rng = np.random.default_rng(5)
    graphs = [gg.complete(5), gg.star(6), gg.cycle(4), gg.path(5)]
    graphs += [gg.er_gnp(int(rng.integers(5, 13)), float(rng.uniform(0.2, 0.7)), 40 + i)
               for i in range(20)]
    for g in graphs:
        want = oracle_mod.edge_orbits_brute(g)
        got = gpu_edge_orbits(ev, g)
        bad = np.argwhere(got != want)
        assert bad.size == 0, f"{g}: (slot, orbit) {bad[:6].tolist()}"


@pytest.mark.parametrize("make", [
    lambda: gg.er_gnm(2000, 10000, 1),
    lambda: gg.chung_lu(20000, 100000, 2.1, 500, 3),   # relabelled inside the plan
    lambda: gg.chung_lu(3000, 30000, 1.9, 400, 11),    # dense hub core
    lambda: gg.rmat(11, 8, 0.57, 0.19, 0.19, seed=4, cap=300),
])
def test_against_lemma(ev, oracle_mod, make):
    g = make()
    want = oracle_mod.edge_orbits_formula(g)
    got = gpu_edge_orbits(ev, g)
    bad = np.argwhere(got != want)
    assert bad.size == 0, f"{g}: (slot, orbit) {bad[:6].tolist()}"


def test_edgeless_and_isolated(ev):
    import torch
    g = gg.from_edge_list(5, [])
    assert gpu_edge_orbits(ev, g).shape == (0, 12)
    g = gg.from_edge_list(6, [(1, 4)])
    got = gpu_edge_orbits(ev, g)
    assert got.shape == (2, 12) and not got.any()
