"""Learned work model for the per-root pass (the persistent root queue).

Training data are measured, not modelled: an instrumented execution of the
orbit-counting plan records the clock64 cycles the per-root pass spends on
every vertex.  The targets are log2 of those cycles; the inputs the four
per-vertex features of evoke_plan_features.  Training (forward, backward,
Adam) and inference run in the library's CUDA kernels; this module only
orchestrates them.
"""
from __future__ import annotations

import numpy as np

from . import _lib, graphgen

RMAT_ABC = (0.57, 0.19, 0.19)


def init_params(seed: int, device="cuda"):
    """He-uniform initial parameters (float32, 1249 values) on `device`."""
    import torch
    rng = np.random.default_rng(seed)
    parts = [rng.uniform(-1, 1, (32, 4)) * np.sqrt(6.0 / 4), np.zeros(32),
             rng.uniform(-1, 1, (32, 32)) * np.sqrt(6.0 / 32), np.zeros(32),
             rng.uniform(-1, 1, 32) * np.sqrt(3.0 / 32), np.array([10.0])]
    p = np.concatenate([np.asarray(x, np.float64).reshape(-1) for x in parts]).astype(np.float32)
    assert p.size == _lib.MLP_PARAMS
    return torch.from_numpy(p).to(device)


def training_graphs(count: int = 20, scales=(16, 17, 18), edge_factor: int = 16,
                    cap: int = 20000, seed0: int = 1):
    """Seeded R-MAT graphs, scales cycling over `scales`."""
    a, b, c = RMAT_ABC
    return [graphgen.rmat(scales[i % len(scales)], edge_factor, a, b, c, seed=seed0 + i, cap=cap)
            for i in range(count)]


def measure(graph, warm: int = 1):
    """(features [n,4] float32, log2 cycles [n] float32, cycles int64) of one
    graph, from an instrumented execution on the current CUDA device."""
    import torch
    rp, col = _lib.to_device(graph)
    plan = _lib.Plan.single(rp, col, graph.n, graph.m)
    out = plan.new_output()
    for _ in range(warm):
        plan.execute(out)
    cyc, _ = plan.root_timing(out)
    X = plan.features()
    torch.cuda.synchronize()
    y = torch.log2(cyc.clamp(min=1).to(torch.float32))
    plan.destroy()
    return X, y, cyc


def train(datasets, epochs: int = 40, batch: int = 4096, lr: float = 3e-3, seed: int = 0):
    """Train on a list of (X, y) pairs; returns (params, per-epoch losses)."""
    import torch
    X = torch.cat([d[0] for d in datasets]).contiguous()
    y = torch.cat([d[1] for d in datasets]).contiguous()
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    perm = torch.randperm(X.shape[0], generator=g).to(X.device)
    X, y = X[perm].contiguous(), y[perm].contiguous()
    params = init_params(seed, X.device)
    params[-1] = float(y.mean().item())  # start the output bias at the mean target
    losses, _ = _lib.mlp_train(X, y, params, epochs, batch, lr)
    return params, losses


def spearman(a, b) -> float:
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    ra = np.argsort(np.argsort(a, kind="stable"), kind="stable").astype(np.float64)
    rb = np.argsort(np.argsort(b, kind="stable"), kind="stable").astype(np.float64)
    ra -= ra.mean()
    rb -= rb.mean()
    den = np.sqrt((ra * ra).sum() * (rb * rb).sum())
    return float((ra * rb).sum() / den) if den > 0 else 0.0


def wedge_work(graph) -> np.ndarray:
    """The degree-bucket schedule's cost estimate: sum_{v in N(u)} d(v)."""
    d = graph.degrees().astype(np.int64)
    src = np.repeat(np.arange(graph.n), d)
    return np.bincount(src, weights=d[graph.col.astype(np.int64)], minlength=graph.n)


def list_schedule_makespan(cost, order, workers: int) -> float:
    """Makespan of greedy list scheduling: jobs taken in `order`, each by the
    worker that frees up first (the persistent queue's behaviour), with the
    measured per-job `cost`."""
    import heapq
    cost = np.asarray(cost, np.float64)
    heap = [0.0] * workers
    for j in order:
        t = heapq.heappop(heap)
        heapq.heappush(heap, t + cost[j])
    return max(heap)
