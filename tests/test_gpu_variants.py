"""The method variants of the paper through the C ABI against the FP64
oracle: Adams-Bashforth node advection (Sec. II.C) and the linearised
equilibrium (Sec. IV.A), on the scalar (FP64, ragged) and vectorised
(FP32/FP16, nx/4 a power of two) collide paths, across graph replays, for a
batch, and through a checkpoint restart."""
import numpy as np
import pytest

import oracle as O
from cases import gpu_sim, oracle_sim, rel_inf
from paper_1004_2416_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TRAJ = {"fp64": 1e-10, "fp32": 1e-4}


def _case(precision, shape=(40, 36, 28)):
    c = W.Capsule((19.2, 17.7, 13.6), 5.0, 3, W.k_s_for(0.05, 5.0))
    return W.Case("variant", shape, 1.0, 3, precision, 0.02, [c], 150)


@pytest.mark.parametrize("prec,shape", [("fp64", (40, 36, 28)), ("fp32", (40, 36, 28)), ("fp32", (32, 36, 28))])
@pytest.mark.parametrize("integrator,order", [(1, 2), (0, 1), (1, 1)])
def test_variants_against_oracle(prec, shape, integrator, order):
    case = _case(prec, shape)
    g = gpu_sim(case)
    g.set_integrator(integrator)
    g.set_equilibrium(order)
    o = oracle_sim(case)
    o.set_integrator(integrator)
    o.set_equilibrium(order)
    g.step(case.steps)
    o.step(case.steps)
    tol = TRAJ[prec]
    r = case.capsules[0].radius
    assert np.abs(g.get_nodes() - o.get_nodes()).max() / r < tol
    assert rel_inf(g.get_velocity(), o.get_velocity()) < tol
    assert abs(g.taylor(0)["D"] - o.taylor(0)["D"]) <= 10 * tol * abs(o.taylor(0)["D"])
    g.close()


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_linear_equilibrium_lattice_only(prec):
    """Collide-stream alone with the linearised equilibrium, random start,
    moving walls, both collide paths (vectorised nx = 64, scalar nx = 37)."""
    for shape in ((64, 9, 11), (37, 9, 11)):
        nx, ny, nz = shape
        tau, uw = 0.8, 0.03
        f0 = O.init_couette(nx, ny, nz, uw) + W.population_noise(shape, 2e-3, seed=3)
        from paper_1004_2416_gb300 import Sim

        s = Sim(nx, ny, nz, tau=tau, precision=prec, delta_points=3)
        s.set_shear_walls(uw)
        s.set_equilibrium(1)
        s.set_populations(f0)
        s.step(30)
        f = f0
        for _ in range(30):
            f = O.lbm_step(f, tau, uw, order=1)
        _, w, _ = O.d3q19()
        wb = w[:, None, None, None]
        assert rel_inf(s.get_populations() - wb, f - wb) < (1e-5 if prec == "fp32" else 3e-3)
        s.close()


def test_linear_equilibrium_in_a_batch():
    from paper_1004_2416_gb300 import Sim

    runs = [(24, 20, 22, 1.0, 0.02), (32, 16, 20, 0.9, 0.03)]
    b = Sim.batch(runs, precision="fp32", delta_points=3)
    b.set_equilibrium(1)
    b.init_fluid(1)
    b.step(25)
    for k, (nx, ny, nz, tau, uw) in enumerate(runs):
        f = O.init_couette(nx, ny, nz, uw)
        for _ in range(25):
            f = O.lbm_step(f, tau, uw, order=1)
        _, w, _ = O.d3q19()
        wb = w[:, None, None, None]
        assert rel_inf(b.get_run_populations(k) - wb, f - wb) < 1e-5
    b.close()


def test_adams_bashforth_restart_and_adjoint_refusal():
    from paper_1004_2416_gb300 import iblbm as B

    case = _case("fp64")
    a = gpu_sim(case)
    a.set_integrator(1)
    a.step(20)
    ck = a.checkpoint_save()
    a.step(20)
    x_ref = a.get_nodes()
    a.checkpoint_restore(ck)
    a.step(20)
    assert np.abs(a.get_nodes() - x_ref).max() < 1e-12
    with pytest.raises(B.IblbmError) as e:
        a.adjoint_forward(10, 5)
    assert e.value.code == B.IBLBM_ERR_STATE
    with pytest.raises(B.IblbmError) as e:
        a.set_integrator(2)
    assert e.value.code == B.IBLBM_ERR_ARG
    with pytest.raises(B.IblbmError) as e:
        a.set_equilibrium(3)
    assert e.value.code == B.IBLBM_ERR_ARG
    a.close()
