"""Parity of the CUDA path (through the C ABI) with the oracle: every
orbit count of every vertex must be bit-identical (exact integers)."""
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


def gpu_counts(ev, g, **kw):
    rp, col = ev.to_device(g)
    out = ev.count_orbits(rp, col, g.n, g.m, **kw)
    return out.cpu().numpy()


def check(ev, oracle_mod, g, **kw):
    _, want = oracle_mod.formulas(g)
    got = gpu_counts(ev, g, **kw)
    bad = np.argwhere(got != want)
    assert bad.size == 0, f"{g}: first mismatches (vertex, orbit) {bad[:8].tolist()}"


def test_special_graphs(ev, oracle_mod):
    graphs = [gg.complete(6), gg.complete(9), gg.star(7), gg.cycle(5), gg.cycle(8),
              gg.path(9)]
    graphs += [gg.from_edge_list(k, e) for k, e, _ in _paper.read_patterns()]
    for g in graphs:
        check(ev, oracle_mod, g)


def test_small_random_graphs(ev, oracle_mod):
    rng = np.random.default_rng(2024)
    for i in range(50):
        n = int(rng.integers(8, 31))
        g = gg.er_gnp(n, float(rng.uniform(0.2, 0.6)), 1000 + i)
        check(ev, oracle_mod, g)


def test_er_2000_10000(ev, oracle_mod):
    check(ev, oracle_mod, gg.er_gnm(2000, 10000, 1))


def test_chung_lu_medium(ev, oracle_mod):
    # power-law with hubs: many CTAs, ragged rows, dense hub core
    check(ev, oracle_mod, gg.chung_lu(20000, 100000, 2.1, 500, 3))


def test_rmat_small(ev, oracle_mod):
    check(ev, oracle_mod, gg.rmat(11, 8, 0.57, 0.19, 0.19, seed=4, cap=300))


def test_dense_core(ev, oracle_mod):
    # hub-heavy: many 5-cliques, wheels, long triangle lists
    check(ev, oracle_mod, gg.chung_lu(3000, 30000, 1.9, 400, 11))


def test_edge_orbits(ev, oracle_mod):
    g = gg.chung_lu(5000, 25000, 2.1, 200, 5)
    rp, col = ev.to_device(g)
    got = {k: v.cpu().numpy() for k, v in ev.edge_orbits(rp, col, g.n, g.m).items()}
    want = oracle_mod.edge_counts(g)
    for k in ("T", "C4", "K4", "E7", "E9"):
        assert np.array_equal(got[k], want[k]), k


def test_empty_and_isolated(ev, oracle_mod):
    import torch
    empty = gg.from_edge_list(0, [])
    assert gpu_counts(ev, empty).shape == (0, 73)
    iso = gg.from_edge_list(6, [(1, 4)])
    check(ev, oracle_mod, iso)
    check(ev, oracle_mod, gg.from_edge_list(7, []))


def test_schedule_invariance(ev, oracle_mod):
    g = gg.chung_lu(4000, 20000, 2.1, 150, 8)
    a = gpu_counts(ev, g)
    b = gpu_counts(ev, g, root_ctas=3)
    c = gpu_counts(ev, g, validate=True)
    assert np.array_equal(a, b) and np.array_equal(a, c)
    perm = np.random.default_rng(1).permutation(g.n)
    d = gpu_counts(ev, gg.relabel(g, perm))
    assert np.array_equal(d[perm], a)


def test_validation_rejects_non_simple(ev):
    import torch
    g = gg.from_edge_list(4, [(0, 1), (1, 2), (2, 3)])
    rp, col = ev.to_device(g)
    bad = col.clone()
    bad[0] = 0  # self-loop at vertex 0
    with pytest.raises(ev.EvokeError) as e:
        ev.count_orbits(rp, bad, g.n, g.m, validate=True)
    assert e.value.code == 2
    asym = gg.Graph(3, np.array([0, 1, 1, 1]), np.array([1], dtype=np.uint32))
    rp2, col2 = ev.to_device(asym)
    with pytest.raises(ev.EvokeError) as e:
        ev.count_orbits(rp2, col2, 3, 0, validate=True)
    assert e.value.code == 1  # rowptr[n] != 2m


def test_build_dag(ev):
    g = gg.chung_lu(3000, 15000, 2.1, 100, 2)
    rp, col = ev.to_device(g)
    dp, dc = ev.build_dag(rp, col, g.n, g.m)
    dp, dc = dp.cpu().numpy(), dc.cpu().numpy()
    d = g.degrees()
    e = g.edges()
    want = {}
    for a, b in e:
        s, t = (a, b) if (d[a], a) < (d[b], b) else (b, a)
        want.setdefault(int(s), []).append(int(t))
    for u in range(g.n):
        assert sorted(want.get(u, [])) == dc[dp[u]:dp[u + 1]].tolist()


def test_hub_grouped_schedule(ev, oracle_mod):
    # the root order (degree buckets, or grouped by highest-degree neighbour
    # in chunks) must not change any count
    import torch
    g = gg.chung_lu(20000, 100000, 2.1, 500, 3)
    _, want = oracle_mod.formulas(g)
    rp, col = ev.to_device(g)
    plan = ev.Plan.single(rp, col, g.n, g.m)
    out = plan.new_output()
    for sched, chunk in ((1, 1), (1, 8), (1, 64), (0, 8)):
        plan.set_schedule(sched, chunk)
        out.fill_(-1)
        plan.execute(out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), want), (sched, chunk)
    out.fill_(-1)
    plan.set_schedule(1, 16)
    plan.launch_graph(out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), want)


def test_degree_limit(ev):
    # degrees above 65,535 could wrap the 2-hop pass's 32-bit per-pair counts:
    # plans refuse them with EVOKE_ERANGE instead
    g = gg.star(70_000)
    rp, col = ev.to_device(g)
    with pytest.raises(ev.EvokeError) as info:
        ev.count_orbits(rp, col, g.n, g.m)
    assert info.value.code == 3
    h = gg.star(65_535)  # the largest accepted degree
    rp, col = ev.to_device(h)
    out = ev.count_orbits(rp, col, h.n, h.m).cpu().numpy()
    assert out[0, 0] == 65_535 and out[0, 7] == 65_535 * 65_534 * 65_533 // 6
