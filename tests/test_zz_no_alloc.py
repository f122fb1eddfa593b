"""evoke_build_dag_noalloc (the allocation-free DAG build, for callers that
cannot allocate device memory) must give exactly the DAG of evoke_build_dag.

Two calls in a row on different graphs, each compared with the allocating
entry point: the second call also shows that the shared static scratch left
behind by the first call does not leak into the result.  This file is
collected last so that a failure here stops a -x run only after every other
test has run."""
import numpy as np
import pytest

from paper_1911_10616_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


def test_noalloc_dag_matches_allocating_entry_point():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1911_10616_gb300 as ev
    from paper_1911_10616_gb300 import _lib

    graphs = [gg.chung_lu(30000, 150000, 2.1, 400, 21),  # many scan tiles, ragged tail
              gg.er_gnm(2500, 9000, 22)]                 # fewer tiles than the first call
    for g in graphs:
        rp, col = ev.to_device(g)
        want_ptr, want_col = ev.build_dag(rp, col, g.n, g.m)
        dp = torch.full((g.n + 1,), -1, dtype=torch.int32, device="cuda")
        dc = torch.full((max(g.m, 1),), -1, dtype=torch.int32, device="cuda")
        _lib.build_dag_noalloc(rp, col, g.n, g.m, dp, dc)
        torch.cuda.synchronize()
        assert np.array_equal(dp.cpu().numpy(), want_ptr.cpu().numpy())
        assert np.array_equal(dc[:g.m].cpu().numpy(), want_col.cpu().numpy())
