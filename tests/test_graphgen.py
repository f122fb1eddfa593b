"""The seeded input generators that stand in for the paper's datasets: every
graph is simple (sorted rows, no loops, no duplicates, symmetric), the same
seed gives the same graph, and each generator honours its parameters (exact
edge counts, degree caps, size ranges, batch offsets)."""
import numpy as np
import pytest

from paper_1911_10616_gb300 import graphgen as gg


def assert_simple(g):
    rp, col = g.rowptr, g.col.astype(np.int64)
    assert rp[0] == 0 and rp[-1] == col.size and (np.diff(rp) >= 0).all()
    src = np.repeat(np.arange(g.n), np.diff(rp))
    assert (col < g.n).all() and (col != src).all()           # ids in range, no loops
    for u in range(g.n) if g.n < 3000 else range(0, g.n, max(1, g.n // 3000)):
        row = col[rp[u]:rp[u + 1]]
        assert (np.diff(row) > 0).all(), u                      # sorted, no duplicates
    key = src * g.n + col
    rkey = col * g.n + src
    assert np.array_equal(np.sort(key), np.sort(rkey))          # symmetric


@pytest.mark.parametrize("make", [
    lambda s: gg.er_gnm(500, 2000, s),
    lambda s: gg.er_gnp(60, 0.2, s),
    lambda s: gg.chung_lu(5000, 25000, 2.1, 200, s),
    lambda s: gg.rmat(10, 8, 0.57, 0.19, 0.19, s, cap=150),
    lambda s: gg.barabasi_albert(300, 3, s),
    lambda s: gg.random_geometric(300, 0.1, s),
])
def test_simple_and_seeded(make):
    a, b, c = make(1), make(1), make(2)
    assert_simple(a)
    assert np.array_equal(a.rowptr, b.rowptr) and np.array_equal(a.col, b.col)
    assert not (a.rowptr.size == c.rowptr.size and np.array_equal(a.col, c.col))


def test_parameters_honoured():
    assert gg.er_gnm(400, 1234, 3).m == 1234
    g = gg.chung_lu(20000, 100000, 2.1, 300, 4)
    assert g.degrees().max() <= 300
    d = g.degrees()
    assert d.max() > 20 * d.mean()                  # heavy tail reaches the cap region
    r = gg.rmat(11, 8, 0.57, 0.19, 0.19, 5, cap=100)
    assert r.n == 2048 and r.degrees().max() <= 100
    ba = gg.barabasi_albert(200, 4, 6)
    assert ba.m == 4 * (200 - 4)                    # m0 distinct targets per new vertex
    for k in (3, 7):
        assert gg.complete(k).m == k * (k - 1) // 2
        assert gg.cycle(k).m == k and gg.path(k).m == k - 1 and gg.star(k).m == k


def test_relabel_permutes_degrees():
    g = gg.chung_lu(3000, 12000, 2.1, 100, 7)
    perm = np.random.default_rng(8).permutation(g.n)
    h = gg.relabel(g, perm)
    assert_simple(h)
    assert np.array_equal(h.degrees()[perm], g.degrees())


def test_batch_tensors_layout():
    torch = pytest.importorskip("torch")
    rpc, colc, vo, eo = gg.small_graph_batch_tensors(90, 10, 60, 9, device="cpu")
    vo, eo = vo.numpy(), eo.numpy()
    assert vo.shape == (91,) and eo.shape == (91,) and vo[0] == 0 and eo[0] == 0
    assert rpc.numel() == vo[-1] + 90 and colc.numel() == eo[-1]
    h = [x.numpy() for x in (rpc, colc)] + [vo, eo]
    for gi in range(90):
        g = gg.batch_graph(*h, gi)
        assert 10 <= g.n <= 60
        assert g.col.size == eo[gi + 1] - eo[gi]
        assert_simple(g)
    # the same seed gives the same batch
    again = gg.small_graph_batch_tensors(90, 10, 60, 9, device="cpu")
    assert all(torch.equal(x, y) for x, y in zip((rpc, colc), again[:2]))


def test_concat_batch_round_trip():
    graphs = gg.small_graph_batch(12, 10, 40, 3) + [gg.from_edge_list(0, []), gg.star(4)]
    rp, col, vo, eo = gg.concat_batch(graphs)
    for gi, g in enumerate(graphs):
        back = gg.batch_graph(rp, col, vo, eo, gi)
        assert back.n == g.n and np.array_equal(back.rowptr, g.rowptr)
        assert np.array_equal(back.col, g.col)
