"""Full-size workloads in the launch configuration bench.py times (plans,
autotuned per-root shape), checked through the C ABI:

* the 1,000,000-vertex Chung-Lu graph: properties that hold at any size
  (orbit 0 is the degree; per pattern, sum_u DIM_k(u) / |orbit k| is the same
  for every orbit k of the pattern; all counts >= 0; the per-edge triangle
  counts sum to 3x the per-vertex ones; a relabelled copy gives the
  relabelled counts);
* the 200,000-graph batch: every count of a seeded sample of whole graphs,
  which the oracle computes one graph at a time, plus the invariants on all
  51 million rows."""
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


def exact_column_sums(counts):
    """Column sums as Python ints (no int64 or float rounding)."""
    c = counts.astype(np.uint64)  # counts are >= 0
    hi = (c >> np.uint64(32)).sum(0, dtype=np.uint64)
    lo = (c & np.uint64(0xFFFFFFFF)).sum(0, dtype=np.uint64)
    return [(int(h) << 32) + int(l) for h, l in zip(hi, lo)]


def pattern_consistency(oracle_mod, counts):
    """Per pattern: each orbit's column sum is divisible by the orbit's size
    and the quotients (the number of induced copies) agree."""
    k, orb, sz = oracle_mod.pattern_orbits()
    tot = exact_column_sums(counts)
    for j in range(30):
        orbits = sorted(set(orb[j, : k[j]]))
        if any(tot[o] % int(sz[o]) for o in orbits):
            return False
        if len({tot[o] // int(sz[o]) for o in orbits}) != 1:
            return False
    return True


def run_plan(ev, rp, col, n, m, configs=((512, 2, 0, 1),)):
    """Counts of one plan under each (threads, CTAs per SM, schedule, chunk)
    configuration of the per-root pass; all must agree bit for bit."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    plan = ev.Plan.single(rp, col, n, m, validate=True)
    out = plan.new_output()
    res = None
    for th, per_sm, sched, chunk in configs:
        plan.set_tuning(th, min(sms * per_sm, plan.info()["root_ctas_max"]))
        plan.set_schedule(sched, chunk)
        out.fill_(-1)
        plan.execute(out)
        plan.status()
        got = out.cpu().numpy()
        if res is None:
            res = got
        else:
            assert np.array_equal(got, res), (th, per_sm, sched, chunk)
    plan.destroy()
    return res


def test_chung_lu_1m_invariants(ev, oracle_mod):
    g = gg.chung_lu(1_000_000, 10_000_000, 2.1, 5000, 1)
    rp, col = ev.to_device(g)
    # the configuration the bench settles on (1024-thread CTAs, one per SM,
    # roots grouped by highest-degree neighbour) and the default one
    dim = run_plan(ev, rp, col, g.n, g.m, configs=((1024, 1, 1, 16), (512, 2, 0, 1)))
    assert (dim >= 0).all()
    assert np.array_equal(dim[:, 0], g.degrees())
    assert pattern_consistency(oracle_mod, dim)
    T = ev.edge_orbits(rp, col, g.n, g.m)["T"].cpu().numpy()
    # per slot T(u,v) summed over all 2m slots = 6 x triangles = 2 x sum_u T(u)
    assert int(T.sum()) == 2 * int(dim[:, 3].sum())
    # relabelling: a random permutation of the ids permutes the rows
    perm = np.random.default_rng(5).permutation(g.n)
    h = gg.relabel(g, perm)
    rp2, col2 = ev.to_device(h)
    dim2 = run_plan(ev, rp2, col2, h.n, h.m)
    assert np.array_equal(dim2[perm], dim)


def test_batch_200k_sampled_exact(ev, oracle_mod):
    import torch
    rpc, colc, vo, eo = gg.small_graph_batch_tensors(200_000, 10, 500, 1, device="cuda")
    plan = ev.Plan.batch(rpc, colc, vo, eo, validate=True)
    out = plan.new_output()
    plan.launch_graph(out)
    torch.cuda.synchronize()
    dim = out.cpu().numpy()
    plan.destroy()
    h = [x.cpu().numpy() for x in (rpc, colc, vo, eo)]
    assert (dim >= 0).all()
    rng = np.random.default_rng(11)
    sample = np.sort(rng.choice(200_000, 300, replace=False))
    for gi in sample:
        gr = gg.batch_graph(*h, gi)
        _, want = oracle_mod.formulas(gr)
        got = dim[h[2][gi]:h[2][gi + 1]]
        assert np.array_equal(got, want), gi
    assert pattern_consistency(oracle_mod, dim)
