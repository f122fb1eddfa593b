"""Batched many-small-graphs path (evoke_count_batch, plans, CUDA-graph
replay) against the oracle, graph by graph."""
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


def mixed_batch():
    graphs = [gg.from_edge_list(k, e) for k, e, _ in _paper.read_patterns()]
    graphs += [gg.from_edge_list(0, []), gg.from_edge_list(1, []), gg.from_edge_list(5, [(0, 4)]),
               gg.complete(7), gg.star(9), gg.cycle(5), gg.path(6)]
    graphs += gg.small_graph_batch(90, 10, 60, seed=5)
    return graphs


def oracle_concat(oracle_mod, graphs):
    return np.concatenate([oracle_mod.formulas(g)[1] if g.n else np.zeros((0, 73), np.int64)
                           for g in graphs])


def test_count_batch_matches_oracle(ev, oracle_mod):
    graphs = mixed_batch()
    want = oracle_concat(oracle_mod, graphs)
    got = ev.count_batch(*ev.batch_to_device(graphs), validate=True).cpu().numpy()
    bad = np.argwhere(got != want)
    assert bad.size == 0, bad[:8].tolist()


def test_batch_plan_execute_and_graph_replay(ev, oracle_mod):
    import torch
    graphs = gg.small_graph_batch(60, 10, 120, seed=9)
    want = oracle_concat(oracle_mod, graphs)
    plan = ev.Plan.batch(*ev.batch_to_device(graphs))
    out = plan.new_output()
    for _ in range(2):
        out.fill_(-1)
        plan.execute(out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), want)
    for _ in range(2):
        out.fill_(-1)
        plan.launch_graph(out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), want)
    info = plan.info()
    assert info["max_component"] == max(g.n for g in graphs)
    # a different CTA shape of the per-root pass gives the same counts
    plan.set_tuning(256, info["root_ctas_max"])
    out.fill_(-1)
    plan.execute(out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), want)
    plan.destroy()


def test_single_plan_matches_one_shot(ev, oracle_mod):
    import torch
    g = gg.chung_lu(8000, 40000, 2.1, 300, 13)
    _, want = oracle_mod.formulas(g)
    rp, col = ev.to_device(g)
    plan = ev.Plan.single(rp, col, g.n, g.m, validate=True)
    out = plan.new_output()
    plan.execute(out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), want)
    out.zero_()
    plan.launch_graph(out)
    plan.launch_graph(out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), want)
    plan.destroy()
