"""Deterministic spreading (iblbm_set_deterministic_spreading): the force
density of Eq. (forcespreading) summed in 64-bit fixed point, whose integer
additions give the same bits in any order.  Checked: two independent runs
with membranes give identical bits; a run restarted from a checkpoint
continues the uninterrupted run bit for bit with membranes (float atomics
only allow that without them); the trajectory matches the FP64 oracle at the
usual tolerances; a contribution beyond the fixed-point range is refused and
reported; batches are refused."""
import numpy as np
import pytest

import oracle as O
from cases import gpu_sim, oracle_sim, rel_inf
from paper_1004_2416_gb300 import iblbm as B
from paper_1004_2416_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _case(precision, steps=60):
    """Two capsules close enough that their stencils share cells, above 152 x
    32 nodes in all (the four-nodes-per-warp kernels) or not, by radius."""
    caps = [W.Capsule((17.3, 17.6, 13.4), 5.0, 3, W.k_s_for(0.05, 5.0)),
            W.Capsule((29.1, 18.2, 14.9), 4.0, 3, W.k_s_for(0.02, 4.0))]
    return W.Case("det", (48, 36, 28), 1.0, 3, precision, 0.02, caps, steps)


def _det_sim(case, x0=None, f0=None):
    g = gpu_sim(case)
    g.set_deterministic_spreading(True)
    if x0 is not None:
        g.set_nodes(x0)
    if f0 is not None:
        g.set_populations(f0)
    return g


def _start(case, seed):
    o = oracle_sim(case)
    x0 = o.get_nodes() + W.jitter(o.n_nodes, 0.2, seed=seed)
    f0 = o.get_f() + W.population_noise(case.shape, 1e-3, seed=seed + 1)
    return o, x0, f0


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
def test_two_runs_identical(prec):
    case = _case(prec)
    o, x0, f0 = _start(case, 11)
    out = []
    for _ in range(2):
        g = _det_sim(case, x0, f0)
        g.step(case.steps)
        out.append((g.get_populations(), g.get_nodes(), g.get_force_field(), g.get_node_velocities()))
        g.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b)
    o.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
def test_restart_bit_exact_with_membranes(prec):
    case = _case(prec)
    o, x0, f0 = _start(case, 21)
    g = _det_sim(case, x0, f0)
    g.step(37)
    ck = g.checkpoint_save()
    g.step(41)
    ref = (g.get_populations(), g.get_nodes(), g.get_force_field(), g.taylor(0)["D"])
    g2 = _det_sim(case)
    g2.checkpoint_restore(ck)
    g2.step(41)
    got = (g2.get_populations(), g2.get_nodes(), g2.get_force_field(), g2.taylor(0)["D"])
    for a, b in zip(got, ref):
        assert np.array_equal(np.asarray(a), np.asarray(b))
    g.close()
    g2.close()
    o.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-4)])
def test_against_oracle(prec, tol):
    case = _case(prec)
    o, x0, f0 = _start(case, 31)
    g = _det_sim(case, x0, f0)
    o.set_nodes(x0)
    o.set_f(f0)
    g.step(1)
    o.step(1)
    one = 1e-12 if prec == "fp64" else 1e-5
    assert rel_inf(g.get_force_field(), o.get_force_field()) < one
    g.step(case.steps - 1)
    o.step(case.steps - 1)
    assert np.abs(g.get_nodes() - o.get_nodes()).max() / 5.0 < tol
    assert rel_inf(g.get_velocity(), o.get_velocity()) < tol
    _, w, _ = O.d3q19()
    wb = w[:, None, None, None]
    assert rel_inf(g.get_populations() - wb, o.get_f() - wb) < tol
    g.close()
    o.close()


def test_out_of_range_contribution_is_reported():
    """A capsule with an absurd modulus and a strong initial strain: its node
    forces exceed the float builds' fixed-point range (2^22): those
    contributions are not added, and the next synchronising call says so."""
    c = W.Capsule((17.3, 17.6, 13.4), 5.0, 3, 1e9)
    case = W.Case("det-range", (36, 36, 28), 1.0, 3, "fp32", 0.0, [c], 1)
    o = oracle_sim(case)
    x0 = o.get_nodes() * np.array([1.1, 1.0, 1.0]) - np.array([1.73, 0.0, 0.0])
    g = _det_sim(case, x0)
    g.step(1)
    with pytest.raises(B.IblbmError) as e:
        g.sync()
    assert e.value.code == B.IBLBM_ERR_UNSTABLE and "fixed-point" in str(e.value)
    g.sync()  # the status was cleared with the report
    g.close()
    o.close()


def test_batch_and_slabs_refused():
    from paper_1004_2416_gb300 import Sim

    b = Sim.batch([(24, 24, 24, 1.0, 0.01)], precision="fp32", delta_points=3)
    with pytest.raises(B.IblbmError) as e:
        b.set_deterministic_spreading(True)
    assert e.value.code == B.IBLBM_ERR_STATE
    b.close()
    s = Sim(16, 8, 8, precision="fp32")
    s.slab_configure(16, 48)
    with pytest.raises(B.IblbmError) as e:
        s.set_deterministic_spreading(True)
    assert e.value.code == B.IBLBM_ERR_STATE
    s.close()
    s = Sim(16, 8, 8, precision="fp32")
    s.set_deterministic_spreading(True)
    with pytest.raises(B.IblbmError) as e:
        s.slab_configure(16, 48)
    assert e.value.code == B.IBLBM_ERR_STATE
    s.close()
