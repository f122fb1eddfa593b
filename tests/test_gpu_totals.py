"""Non-induced output (evoke_opts.noninduced: DM without A^-1) and global
pattern totals (evoke_graphlet_totals) against the oracle and closed forms."""
import itertools
from math import comb, factorial

import numpy as np
import pytest

from paper_1911_10616_gb300 import graphgen as gg
from tests import _paper

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ev():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1911_10616_gb300 as ev
    ev.load()
    return ev


@pytest.mark.parametrize("make", [
    lambda: gg.complete(7),
    lambda: gg.er_gnp(25, 0.4, 3),
    lambda: gg.er_gnm(2000, 10000, 1),
    lambda: gg.chung_lu(20000, 100000, 2.1, 500, 3),   # relabelled inside the plan
])
def test_noninduced_counts(ev, oracle_mod, make):
    g = make()
    dm, _ = oracle_mod.formulas(g)
    rp, col = ev.to_device(g)
    got = ev.count_orbits(rp, col, g.n, g.m, induced=False).cpu().numpy()
    bad = np.argwhere(got != dm)
    assert bad.size == 0, bad[:8].tolist()
    got4 = ev.count_orbits(rp, col, g.n, g.m, induced=False, orbits=15).cpu().numpy()
    assert np.array_equal(got4, dm[:, :15])


def _pattern_graphs():
    return [(k, e) for k, e, _ in _paper.read_patterns()]


def _automorphisms(k, edges):
    es = {frozenset(e) for e in edges}
    return sum(1 for p in itertools.permutations(range(k))
               if {frozenset((p[a], p[b])) for a, b in edges} == es)


def test_totals_closed_forms(ev):
    pats = _pattern_graphs()
    # K_7: every k-subset induces K_k; non-induced copies of H in K_k: k!/|Aut H|
    g = gg.complete(7)
    rp, col = ev.to_device(g)
    ind = ev.graphlet_totals(ev.count_orbits(rp, col, g.n, g.m))
    want = np.zeros(30, np.int64)
    for j, (k, e) in enumerate(pats):
        if len(e) == k * (k - 1) // 2:
            want[j] = comb(7, k)
    assert np.array_equal(ind, want)
    non = ev.graphlet_totals(ev.count_orbits(rp, col, g.n, g.m, induced=False))
    want = np.array([comb(7, k) * factorial(k) // _automorphisms(k, e) for k, e in pats])
    assert np.array_equal(non, want)
    # cycle C_9: induced paths on 2..5 vertices, nine of each
    g = gg.cycle(9)
    rp, col = ev.to_device(g)
    ind = ev.graphlet_totals(ev.count_orbits(rp, col, g.n, g.m))
    paths = {j for j, (k, e) in enumerate(pats)
             if len(e) == k - 1 and max(np.bincount(np.ravel(e), minlength=k)) <= 2}
    assert np.array_equal(ind, np.array([9 if j in paths else 0 for j in range(30)]))
    # star with L leaves: induced stars with 1..4 leaves
    g = gg.star(9)
    leaves = g.m
    rp, col = ev.to_device(g)
    ind = ev.graphlet_totals(ev.count_orbits(rp, col, g.n, g.m))
    stars = {j: comb(leaves, k - 1) for j, (k, e) in enumerate(pats)
             if len(e) == k - 1 and max(np.bincount(np.ravel(e), minlength=k)) == k - 1}
    assert np.array_equal(ind, np.array([stars.get(j, 0) for j in range(30)]))
    four = ev.graphlet_totals(ev.count_orbits(rp, col, g.n, g.m, orbits=15))
    assert np.array_equal(four, ind[:9])


def test_totals_against_oracle_and_batch(ev, oracle_mod):
    graphs = gg.small_graph_batch(40, 10, 80, seed=12)
    got = ev.graphlet_totals(ev.count_batch(*ev.batch_to_device(graphs)))
    got_non = ev.graphlet_totals(ev.count_batch(*ev.batch_to_device(graphs), induced=False))
    k, orbit_of, size = oracle_mod.pattern_orbits()
    first = [int(orbit_of[j, 0]) for j in range(30)]  # an orbit of each pattern
    want = np.zeros(30, np.int64)
    want_non = np.zeros(30, np.int64)
    for g in graphs:
        dm, dim = oracle_mod.formulas(g)
        want += np.array([dim[:, o].sum() // size[o] for o in first])
        want_non += np.array([dm[:, o].sum() // size[o] for o in first])
    assert np.array_equal(got, want)
    assert np.array_equal(got_non, want_non)


def test_inconsistent_counts_detected(ev):
    import torch
    c = torch.zeros((4, 73), dtype=torch.int64, device="cuda")
    c[0, 3] = 1  # one vertex of a triangle without the other two
    with pytest.raises(ev.EvokeError):
        ev.graphlet_totals(c)
