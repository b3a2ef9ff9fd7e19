"""Parity at the full sizes of the suspension and batch workloads, in the
launch configuration the bench times (captured step graphs, a Taylor record
every step, the automatic kernel choices), against the FP64 oracle:

- the 256 x 128 x 128 suspension of 200 capsules (128 400 nodes, 3-point
  stencil): FP16 storage (the bench's precision) one coupled step, FP32
  storage ten steps, from a jittered state with population noise, every node
  and every cell compared;
- the 64-run batch (boxes 24..64, persistent collide, autotuned tiles):
  20 steps of all 64 runs, each against its own oracle run.

Tolerances as everywhere (relative, infinity norm): FP32 1e-5 for one step
and 1e-4 over several, FP16 storage 2e-3 for one step."""
import os

import numpy as np
import pytest

import oracle as O
from cases import gpu_sim, oracle_sim, rel_inf
from paper_1004_2416_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,steps,tol", [("fp16", 1, 2e-3), ("fp32", 10, 1e-4)])
def test_suspension_full_size(prec, steps, tol):
    case = W.config4(prec)
    o = oracle_sim(case)
    x0 = o.get_nodes() + W.jitter(o.n_nodes, 0.1, seed=97)
    f0 = o.get_f() + W.population_noise(case.shape, 1e-3, seed=98)
    g = gpu_sim(case)
    for s in (g, o):
        s.set_nodes(x0)
    g.set_populations(f0)
    o.set_f(f0)
    g.set_taylor_recording(1, 64)
    g.step(steps)
    threads = O.get_threads()
    O.set_threads(min(16, os.cpu_count() or 1))  # the oracle's lattice loops (bit-identical for any count)
    try:
        o.step(steps)
    finally:
        O.set_threads(threads)
    r = case.capsules[0].radius
    if steps == 1:
        assert rel_inf(g.get_node_forces(), o.get_node_forces()) < 1e-5
        assert rel_inf(g.get_force_field(), o.get_force_field()) < 1e-5
    assert rel_inf(g.get_velocity(), o.get_velocity()) < tol
    assert rel_inf(g.get_node_velocities(), o.get_node_velocities()) < tol
    assert np.abs(g.get_nodes() - o.get_nodes()).max() / r < tol
    _, w, _ = O.d3q19()
    wb = w[:, None, None, None]
    assert rel_inf(g.get_populations() - wb, o.get_f() - wb) < tol
    # the records of the last step against the oracle's shape measures of every capsule
    for cid in (0, 77, 199):
        steps_rec, rec = g.taylor_records(cid)
        assert steps_rec[-1] == steps
        D_o = o.taylor(cid)["D"]
        assert abs(rec[-1, 0] - D_o) <= 50 * tol * abs(D_o) + 1e-7, cid
    g.close()
    o.close()


def test_batch_full_size():
    from paper_1004_2416_gb300 import Sim

    cases = W.config3_cases()
    b = Sim.batch([(*c.shape, c.tau, c.u_wall) for c in cases], precision="fp32", delta_points=3)
    for k, c in enumerate(cases):
        for cap in c.capsules:
            cid = b.add_capsule_icosphere_in_run(k, cap.center, cap.radius, cap.subdivisions)
            b.set_skalak(cap.k_s, cap.C, cid)
    b.init_fluid(1)
    b.autotune_tiles(5)
    b.set_taylor_recording(1, 64)
    steps = 20
    b.step(steps)
    threads = O.get_threads()
    O.set_threads(min(16, os.cpu_count() or 1))
    try:
        for k, c in enumerate(cases):
            o = oracle_sim(c)
            o.step(steps)
            assert rel_inf(b.get_run_velocity(k), o.get_velocity()) < 1e-4, k
            assert np.abs(b.get_nodes(k) - o.get_nodes()).max() / c.capsules[0].radius < 1e-4, k
            assert abs(b.taylor(k)["D"] - o.taylor(0)["D"]) <= 1e-3 * abs(o.taylor(0)["D"]) + 1e-9, k
            o.close()
    finally:
        O.set_threads(threads)
    b.close()
