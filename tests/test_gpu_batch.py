"""Batching extension: independent runs of uneven box sizes advanced together
(one persistent collide-and-stream launch per step), each run compared with
its own FP64 oracle simulation."""
import numpy as np
import pytest

import oracle as O
from cases import oracle_sim, rel_inf
from paper_1004_2416_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-4}


def _runs():
    """Four runs: cubic 24 and 32, a ragged box, an elongated box; different G."""
    out = []
    for (nx, ny, nz), r, m, G in (((24, 24, 24), 3.0, 2, 0.05), ((32, 32, 32), 4.0, 2, 0.0125),
                                  ((20, 18, 14), 2.5, 2, 0.1), ((48, 16, 40), 5.0, 3, 0.003)):
        c = W.Capsule(((nx - 1) / 2 + 0.3, (ny - 1) / 2 - 0.2, (nz - 1) / 2 + 0.1), r, m, W.k_s_for(G, r))
        out.append(W.Case(f"run{nx}x{ny}x{nz}", (nx, ny, nz), 1.0, 3, "fp32", W.u_wall_for(nz), [c], 0))
    return out


def _batch(cases, prec, autotune=False):
    from paper_1004_2416_gb300 import Sim

    b = Sim.batch([(*c.shape, c.tau, c.u_wall) for c in cases], precision=prec, delta_points=3)
    for k, c in enumerate(cases):
        for cap in c.capsules:
            cid = b.add_capsule_icosphere_in_run(k, cap.center, cap.radius, cap.subdivisions)
            b.set_skalak(cap.k_s, cap.C, cid)
    b.init_fluid(1)
    if autotune:
        b.autotune_tiles(3)
    return b


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_runs_match_their_oracles(prec):
    cases = _runs()
    b = _batch(cases, prec)
    steps = 60
    b.step(steps)
    cid = 0
    for k, c in enumerate(cases):
        o = oracle_sim(c)
        o.step(steps)
        assert rel_inf(b.get_run_velocity(k), o.get_velocity()) < TOL[prec], k
        x = b.get_nodes(cid)
        assert np.abs(x - o.get_nodes()).max() / c.capsules[0].radius < TOL[prec], k
        Tg, To = b.taylor(cid), o.taylor(0)
        assert abs(Tg["D"] - To["D"]) <= 10 * TOL[prec] * abs(To["D"]) + 1e-12, k
        cid += 1


def test_autotuned_tiles_give_the_same_trajectory():
    cases = _runs()
    a = _batch(cases, "fp64")
    t = _batch(cases, "fp64", autotune=True)
    shapes = {(32, 8), (16, 16), (8, 32), (64, 4), (128, 2), (256, 1)}
    for k in range(len(cases)):
        assert t.run_tile(k) in shapes
    a.step(40)
    t.step(40)
    for k in range(len(cases)):
        assert rel_inf(t.get_run_populations(k) - 1.0 / 19, a.get_run_populations(k) - 1.0 / 19) < 1e-12
    assert np.abs(t.get_nodes() - a.get_nodes()).max() < 1e-12


def test_config3_subset_against_oracle():
    """Four runs of the seeded 64-run batch (box 24..64, r = side/8, G
    log-uniform in [0.003, 0.1]), FP32, 30 steps."""
    cases = W.config3_cases()[:4]
    b = _batch(cases, "fp32", autotune=True)
    b.step(30)
    for k, c in enumerate(cases):
        o = oracle_sim(c)
        o.step(30)
        assert rel_inf(b.get_run_velocity(k), o.get_velocity()) < TOL["fp32"], k
        assert np.abs(b.get_nodes(k) - o.get_nodes()).max() / c.capsules[0].radius < TOL["fp32"], k


def test_batch_errors():
    from paper_1004_2416_gb300 import iblbm as B

    b = _batch(_runs(), "fp32")
    with pytest.raises(B.IblbmError) as e:
        b.get_velocity()
    assert e.value.code == B.IBLBM_ERR_STATE
    out = np.empty(3 * 24 ** 3)
    assert B.iblbm_get_run_velocity(b.handle, 4, out.ctypes.data_as(B._dp)) == B.IBLBM_ERR_ARG
    b.step(1)
    with pytest.raises(B.IblbmError) as e:
        b.autotune_tiles(2)
    assert e.value.code == B.IBLBM_ERR_STATE
    with pytest.raises(B.IblbmError):
        B.Sim.batch([(8, 8, 8, 0.4, 0.0)])


def test_batch_with_an_odd_row_length():
    """One run with rows of odd length sends the whole FP32 batch through the
    one-cell collide (every run with even rows takes two cells per thread)."""
    cases = _runs()[:2]
    c = W.Capsule((12.3, 9.8, 8.6), 3.0, 2, W.k_s_for(0.05, 3.0))
    cases.append(W.Case("run25x20x18", (25, 20, 18), 1.0, 3, "fp32", W.u_wall_for(18), [c], 0))
    b = _batch(cases, "fp32")
    b.step(40)
    for k, cs in enumerate(cases):
        o = oracle_sim(cs)
        o.step(40)
        assert rel_inf(b.get_run_velocity(k), o.get_velocity()) < TOL["fp32"], k
        assert np.abs(b.get_nodes(k) - o.get_nodes()).max() / cs.capsules[0].radius < TOL["fp32"], k


def test_batch_with_launch_overlap():
    """A batch with the step kernels launched to overlap their predecessor (the
    automatic choice for large batches) against the runs' oracles."""
    cases = _runs()
    b = _batch(cases, "fp32")
    b.set_launch_overlap(True)
    b.step(40)
    for k, c in enumerate(cases):
        o = oracle_sim(c)
        o.step(40)
        assert rel_inf(b.get_run_velocity(k), o.get_velocity()) < TOL["fp32"], k
        assert np.abs(b.get_nodes(k) - o.get_nodes()).max() / c.capsules[0].radius < TOL["fp32"], k
