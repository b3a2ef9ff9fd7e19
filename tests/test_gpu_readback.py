"""Asynchronous read-back: iblbm_read_async snapshots the node positions
behind the steps already enqueued and copies them and the capsule reductions
to the host from a read-back stream; after iblbm_sync they equal what the
synchronising getters return at the same step, also when further steps ran
while the read-backs were in flight."""
import numpy as np
import pytest
import torch

from cases import gpu_sim
from paper_1004_2416_gb300 import iblbm as B
from paper_1004_2416_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _case(prec):
    shape = (64, 48, 40)
    caps = [W.Capsule((20.3, 23.1, 19.4), 6.0, 3, W.k_s_for(0.05, 6.0)),
            W.Capsule((45.2, 24.7, 20.8), 5.0, 2, W.k_s_for(0.05, 5.0))]
    return W.Case("readback", shape, 1.0, 3, prec, 0.02, caps, 40)


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_read_async_matches_getters(prec, pinned):
    case = _case(prec)
    g = gpu_sim(case)
    g.set_taylor_recording(1, ring=64)  # records in flight on the side stream
    n, nc = g.info().n_nodes, len(case.capsules)
    if pinned:
        nodes = torch.empty(n * 3, dtype=torch.float64, pin_memory=True).numpy()
        sums = torch.empty(nc * 12, dtype=torch.float64, pin_memory=True).numpy()
    else:
        nodes = np.empty(n * 3, np.float64)
        sums = np.empty(nc * 12, np.float64)
    early = np.empty(n * 3, np.float64)
    g.step(3)
    g.read_async(early, None)      # behind three steps
    g.step(case.steps)             # several read-backs may be queued at once
    g.read_async(nodes, sums)
    g.sync()
    x = g.get_nodes()
    assert np.array_equal(nodes.reshape(-1, 3), x)
    assert not np.array_equal(early.reshape(-1, 3), x)
    for k in range(nc):
        got = B.taylor_from_sums(sums[12 * k:12 * (k + 1)])
        ref = g.taylor(k)
        for key in ("D", "theta", "V", "A", "c_x", "I_xx", "I_xz"):
            assert got[key] == ref[key], (k, key)
    g.close()


def _case_many(prec):
    """Four 2 562-node capsules: 10 248 nodes, above the count from which
    the read-back snapshot is taken by a copy kernel instead of the copy
    engine."""
    caps = [W.Capsule((15.2 + 24.0 * k, 23.6, 19.7), 6.0, 4, W.k_s_for(0.05, 6.0)) for k in range(4)]
    return W.Case("readback-many", (96, 48, 40), 1.0, 3, prec, 0.02, caps, 40)


@pytest.mark.parametrize("prec,many", [("fp64", False), ("fp32", False), ("fp16", False), ("fp32", True),
                                       ("fp64", True)])
def test_read_async_per_step_while_stepping(prec, many):
    """A read-back after each of eight steps, all in flight while the next
    steps run, against the getters of a twin run after the same steps
    (deterministic spreading: both runs have the same bits)."""
    case = _case_many(prec) if many else _case(prec)
    runs = [gpu_sim(case), gpu_sim(case)]
    for g in runs:
        g.set_deterministic_spreading(True)
    a, twin = runs
    n, nc, k_steps = a.info().n_nodes, len(case.capsules), 8
    nodes = [torch.empty(n * 3, dtype=torch.float64, pin_memory=True).numpy() for _ in range(k_steps)]
    sums = [torch.empty(nc * 12, dtype=torch.float64, pin_memory=True).numpy() for _ in range(k_steps)]
    for k in range(k_steps):
        a.step(1)
        a.read_async(nodes[k], sums[k])
    a.sync()
    for k in range(k_steps):
        twin.step(1)
        assert np.array_equal(nodes[k].reshape(-1, 3), twin.get_nodes()), k
        for c in range(nc):
            got = B.taylor_from_sums(sums[k][12 * c:12 * (c + 1)])
            ref = twin.taylor(c)
            for key in ("D", "theta", "V", "A", "c_x", "I_xx", "I_xz"):
                assert got[key] == ref[key], (k, c, key)
    for g in runs:
        g.close()


def test_read_async_arguments():
    g = gpu_sim(_case("fp32"))
    g.read_async(None, None)  # nothing to copy
    with pytest.raises(ValueError):
        g.read_async(np.empty(3, np.float64), None)  # too small
    g.close()
