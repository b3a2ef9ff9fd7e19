"""The N > 1 path of bench.py on the host: two gloo ranks on the CPU join the
process group, meet at the barrier, agree on the maximum of their timings,
and compute the whole-job throughput of independent replicas from it; the
reference arm runs on rank 0 only.  No data-path collective exists: each rank
advances its own simulation."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

from conftest import ROOT


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench

    grp = bench._Group("gloo")
    assert (grp.ws, grp.rank) == (ws, rank)
    grp.barrier()
    ms = 10.0 + 5.0 * rank          # the slower rank decides the job's time
    ms_max = grp.max(ms)
    value = bench.aggregate_mlups(grp.ws, 1000, 20, ms_max)
    grp.barrier()
    grp.close()
    q.put((rank, ms_max, value))


def test_two_gloo_ranks_agree_on_max_and_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    ms_max = 10.0 + 5.0
    for rank, m, v in out:
        assert m == ms_max
        assert v == pytest.approx(2 * 1000 * 20 / (ms_max * 1e-3) / 1e6)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    called = []
    monkeypatch.setattr(bench, "_oracle_run", lambda *a, **k: called.append(a))
    a = type("A", (), {"warmup": 1, "steps": 1, "cpu_budget_s": 1.0, "workload": "config2", "gpus": 2})()
    assert bench.run_reference(a) is None
    assert not called
