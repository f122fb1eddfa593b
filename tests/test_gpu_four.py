"""The 4-vertex-orbit mode (evoke_opts.orbits = 15: orbits 0..14 of Thm. 4orbit
only, the EVOKE-4 column of the paper's runtime table) against the oracle.
A is block diagonal by pattern size, so these columns of the oracle's full
induced counts are the expected values, bit for bit."""
import ctypes

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


@pytest.mark.parametrize("make", [
    lambda: gg.complete(7),
    lambda: gg.er_gnp(25, 0.4, 3),
    lambda: gg.er_gnm(2000, 10000, 1),
    lambda: gg.chung_lu(20000, 100000, 2.1, 500, 3),   # relabelled inside the plan
    lambda: gg.chung_lu(3000, 30000, 1.9, 400, 11),
])
def test_single_graph(ev, oracle_mod, make):
    g = make()
    want = oracle_mod.formulas(g)[1][:, :15]
    rp, col = ev.to_device(g)
    got = ev.count_orbits(rp, col, g.n, g.m, orbits=15).cpu().numpy()
    assert got.shape == (g.n, 15)
    bad = np.argwhere(got != want)
    assert bad.size == 0, bad[:8].tolist()


def test_plan_and_graph_replay(ev, oracle_mod):
    import torch
    g = gg.chung_lu(5000, 25000, 2.1, 200, 5)
    want = oracle_mod.formulas(g)[1][:, :15]
    rp, col = ev.to_device(g)
    plan = ev.Plan.single(rp, col, g.n, g.m, orbits=15)
    assert plan.info()["orbits"] == 15
    out = plan.new_output()
    for run in (plan.execute, plan.execute, plan.launch_graph, plan.launch_graph):
        out.fill_(-1)
        run(out)
        plan.status()  # no 3-path count wrapped
        assert np.array_equal(out.cpu().numpy(), want)


def test_batch(ev, oracle_mod):
    graphs = gg.small_graph_batch(60, 10, 120, seed=9) + [gg.from_edge_list(3, [])]
    want = np.concatenate([oracle_mod.formulas(x)[1][:, :15] for x in graphs])
    got = ev.count_batch(*ev.batch_to_device(graphs), orbits=15).cpu().numpy()
    assert np.array_equal(got, want)


def test_bad_orbit_count_rejected(ev):
    from paper_1911_10616_gb300 import _lib
    g = gg.complete(4)
    rp, col = ev.to_device(g)
    import torch
    out = torch.empty((g.n, 73), dtype=torch.int64, device=rp.device)
    for bad in (1, 14, 16, 74):
        opts = _lib.EvokeOpts(0, 0, 0, bad)
        rc = ev.load().evoke_count_orbits(_lib._ptr(rp), _lib._ptr(col), g.n, g.m,
                                          _lib._ptr(out), ctypes.byref(opts), None)
        assert rc == 1  # EVOKE_EINVAL
    with pytest.raises(ValueError):
        ev.count_orbits(rp, col, g.n, g.m, orbits=20)
