"""The multi-rank host logic of bench.py on CPU (gloo, world size 2): ranks
are independent replicas, the job's time is the slowest rank's, and only rank
0 of the CPU reference arm does work."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from tests.conftest import ROOT


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(1.5 + rank, dist)   # rank 1 is the slower one
    same = bench.max_over_ranks(3.0, dist)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, same))


def test_max_over_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == [(0, 2.5, 3.0), (1, 2.5, 3.0)]


def test_max_over_ranks_single_process():
    import bench
    assert bench.max_over_ranks(4.25, None) == 4.25


def test_reference_arm_only_on_rank0(capsys):
    import argparse

    import bench
    args = argparse.Namespace(workload="er_2000", steps=1, warmup=0, cpu_budget=1.0, gpus=2)
    bench.run_reference(args, rank=1, world=2)   # the other ranks exit without work
    assert capsys.readouterr().out == ""


def test_traffic_gate_follows_kernel_source(tmp_path, monkeypatch):
    # the root kernel's DRAM traffic is reported from the committed ncu
    # summary only while the kernel source it was captured from is unchanged
    import shutil

    import bench
    assert isinstance(bench.measured_traffic("chung_lu_1m"), int)
    assert bench.measured_traffic("er_2000") is None
    (tmp_path / "profiles").mkdir()
    shutil.copy(os.path.join(ROOT, "profiles", "root_kernel_dram_chung_lu_1m.md"), tmp_path / "profiles")
    src = tmp_path / "paper_1911_10616_gb300" / "csrc"
    src.mkdir(parents=True)
    text = open(os.path.join(ROOT, "paper_1911_10616_gb300", "csrc", "k_root.cu")).read()
    (src / "k_root.cu").write_text(text)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert isinstance(bench.measured_traffic("chung_lu_1m"), int)
    (src / "k_root.cu").write_text(text + "\n// changed\n")
    assert bench.measured_traffic("chung_lu_1m") is None
