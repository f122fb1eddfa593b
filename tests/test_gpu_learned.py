"""Learned work model: the CUDA MLP kernels against the oracle's numpy MLP,
training, the learned schedule's invariance, and what it gains over the
wedge-work estimate of the degree-bucket schedule."""
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


def test_forward_and_gradient_match_oracle(ev):
    import torch
    from oracle import mlp
    from paper_1911_10616_gb300 import _lib
    rng = np.random.default_rng(3)
    p = (rng.normal(0, 0.4, mlp.NPARAM)).astype(np.float32)
    X = rng.uniform(0, 6, (1000, 4)).astype(np.float32)   # ragged: not a multiple of 64
    T = rng.normal(8, 2, 1000).astype(np.float32)
    dp, dX, dT = (torch.from_numpy(a).cuda() for a in (p, X, T))
    y = _lib.mlp_forward(dX, dp).cpu().numpy()
    y_ref, _ = mlp.forward(p, X)
    assert np.allclose(y, y_ref, rtol=1e-4, atol=1e-4)
    g, loss = _lib.mlp_grad(dX, dT, dp)
    l_ref, g_ref = mlp.loss_and_grad(p, X, T)
    assert abs(float(loss.item()) - l_ref) <= 1e-4 * max(1.0, l_ref)
    scale = np.abs(g_ref).max()
    assert np.allclose(g.cpu().numpy(), g_ref, rtol=1e-3, atol=1e-4 * scale)


def test_training_reduces_loss(ev):
    import torch
    from paper_1911_10616_gb300 import _lib, learned
    rng = np.random.default_rng(4)
    X = rng.uniform(0, 8, (20000, 4)).astype(np.float32)
    T = (2.0 + X @ np.array([0.5, 1.0, 0.25, 0.3]) + 0.3 * np.sin(X[:, 0])).astype(np.float32)
    dX, dT = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    params = learned.init_params(0)
    losses, _ = _lib.mlp_train(dX, dT, params, epochs=30, batch=1024, lr=3e-3)
    assert losses[-1] < 0.05 * losses[0]


def test_learned_schedule_same_counts_and_gain(ev, oracle_mod):
    import torch
    from paper_1911_10616_gb300 import _lib, learned
    train = learned.training_graphs(4, scales=(13, 14), cap=5000, seed0=40)
    data = [learned.measure(g)[:2] for g in train]
    params, losses = learned.train(data, epochs=40, batch=2048)
    assert losses[-1] < losses[0]
    g = gg.rmat(14, 16, *learned.RMAT_ABC, seed=77, cap=5000)
    rp, col = ev.to_device(g)
    plan = ev.Plan.single(rp, col, g.n, g.m)
    out_deg = plan.new_output()
    plan.execute(out_deg)
    plan.set_model(params)
    out_l = plan.new_output()
    plan.execute(out_l)
    torch.cuda.synchronize()
    # the schedule never changes the counts
    assert np.array_equal(out_deg.cpu().numpy(), out_l.cpu().numpy())
    plan.destroy()
    # gain over the wedge-work estimate sum_{v in N(u)} d(v) that orders the
    # degree-bucket schedule, judged by measured per-root cycles of a graph
    # the network was not trained on: its cost prediction has a smaller error
    # than the best affine map from the estimate to log2 cycles (fitted on
    # this very graph, which favours the estimate).  Its ranking is about as
    # good as the estimate's (which is already near 0.99 here), so only a
    # floor is asserted for it.
    X, y, cyc = learned.measure(g)
    pred = _lib.mlp_forward(X, params).cpu().numpy()
    meas = y.cpu().numpy()
    busy = g.degrees() > 0
    work = learned.wedge_work(g)
    r_learned = learned.spearman(pred[busy], meas[busy])
    r_proxy = learned.spearman(work[busy], meas[busy])
    A = np.vstack([np.log2(1 + work[busy]), np.ones(busy.sum())]).T
    coef = np.linalg.lstsq(A, meas[busy], rcond=None)[0]
    mae_proxy = np.abs(A @ coef - meas[busy]).mean()
    mae_learned = np.abs(pred[busy] - meas[busy]).mean()
    print(f"spearman learned {r_learned:.4f} vs wedge work {r_proxy:.4f}; "
          f"MAE log2 cycles learned {mae_learned:.3f} vs affine wedge work {mae_proxy:.3f}")
    assert mae_learned < mae_proxy
    assert r_learned > 0.95
