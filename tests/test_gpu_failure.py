"""Failure detection without a GPU fault: the collide kernels' density watchdog.

Every collide-and-stream kernel checks the density of each cell it updates
(Eq. lbmmomenta0) and records a non-finite value, or one outside (0.5, 2), in
the object's device status word; the next synchronising call returns
IBLBM_ERR_UNSTABLE with its message and clears the word.  The faults are
made on the host: populations uploaded through the C ABI with one cell of
density 3, or one population of 1e30 (a runaway value: out of range in the
FP64 and FP32 builds, infinite once stored as a scaled FP16 deviation).  A
NaN never reaches the device that way: the upload refuses non-finite
values.  After good populations are put back, the next step runs clean.
Nothing here traps, hangs or faults the device: the kernels only set a
bit.
"""
import numpy as np
import pytest

import oracle as O
from paper_1004_2416_gb300 import iblbm as B
from paper_1004_2416_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# one lattice shape per collide kernel family of the float builds: 4 cells
# per thread (nx/4 a power of two), 2 cells per thread (even rows), 1 cell
# (odd rows); the FP64 build takes the one-cell kernel everywhere
SHAPES = {"x4": (32, 6, 7), "pair": (20, 6, 7), "one": (21, 6, 7)}


def _bad(f, kind):
    f = f.copy()
    if kind == "huge":
        f[7, 3, 2, 5] = 1e30
    else:  # density 3 in one cell: every population of the cell scaled by 3
        f[:, 4, 1, 9] *= 3.0
    return f


def _expect_unstable(sim):
    with pytest.raises(B.IblbmError) as e:
        sim.sync()
    assert e.value.code == B.IBLBM_ERR_UNSTABLE
    assert "density" in str(e.value)
    sim.sync()  # reported once, then cleared


@pytest.mark.parametrize("kind", ["huge", "rho3"])
@pytest.mark.parametrize("family", sorted(SHAPES))
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
def test_watchdog_single_lattice(prec, family, kind):
    from paper_1004_2416_gb300 import Sim

    nx, ny, nz = SHAPES[family]
    uw = 0.02
    good = O.init_couette(nx, ny, nz, uw) + W.population_noise((nx, ny, nz), 1e-3, seed=5)
    s = Sim(nx, ny, nz, tau=1.0, precision=prec, delta_points=3)
    s.set_shear_walls(uw)
    s.set_populations(good)
    s.step(1)
    s.sync()
    s.set_populations(_bad(good, kind))
    s.step(1)
    _expect_unstable(s)
    s.set_populations(good)
    s.step(2)
    s.sync()  # clean again
    f = O.lbm_step(O.lbm_step(good, 1.0, uw), 1.0, uw)
    tol = {"fp64": 1e-12, "fp32": 1e-5, "fp16": 3e-3}[prec]
    _, w, _ = O.d3q19()
    wb = w[:, None, None, None]
    err = np.abs((s.get_populations() - wb) - (f - wb)).max() / np.abs(f - wb).max()
    assert err < tol
    s.close()


@pytest.mark.parametrize("kind", ["huge", "rho3"])
@pytest.mark.parametrize("nx1", [20, 21])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
def test_watchdog_batch(prec, nx1, kind):
    """A batch of two runs (with nx1 = 20 every row is even and the float
    builds take the two-cell batch kernel, with 21 the one-cell kernel): a
    bad cell in run 1 is reported, and after run 1 gets good populations back
    the batch steps clean."""
    from paper_1004_2416_gb300 import Sim

    specs = [(24, 8, 6, 1.0, 0.02), (nx1, 7, 9, 1.0, 0.03)]
    s = Sim.batch(specs, precision=prec, delta_points=3)
    s.init_fluid(1)
    nx, ny, nz = specs[1][:3]
    good = O.init_couette(nx, ny, nz, specs[1][4]) + W.population_noise((nx, ny, nz), 1e-3, seed=6)
    s.set_run_populations(1, good)
    s.step(1)
    s.sync()
    s.set_run_populations(1, _bad(good, kind))
    s.step(1)
    _expect_unstable(s)
    s.set_run_populations(1, good)
    s.step(1)
    s.sync()
    f = O.lbm_step(good, 1.0, specs[1][4])
    _, w, _ = O.d3q19()
    wb = w[:, None, None, None]
    tol = {"fp64": 1e-12, "fp32": 1e-5, "fp16": 3e-3}[prec]
    err = np.abs((s.get_run_populations(1) - wb) - (f - wb)).max() / np.abs(f - wb).max()
    assert err < tol
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
def test_upload_refuses_nan(prec):
    from paper_1004_2416_gb300 import Sim

    s = Sim(20, 6, 7, tau=1.0, precision=prec, delta_points=3)
    before = s.get_populations()
    f = O.init_couette(20, 6, 7, 0.02)
    for bad in (np.nan, np.inf, -np.inf):
        g = f.copy()
        g[3, 2, 1, 4] = bad
        with pytest.raises(B.IblbmError) as e:
            s.set_populations(g)
        assert e.value.code == B.IBLBM_ERR_ARG and "non-finite" in str(e.value)
        assert np.array_equal(s.get_populations(), before)  # the lattice is left as it was
    g = f.copy()
    g[18, 6, 5, 19] = np.nan  # the last value
    with pytest.raises(B.IblbmError):
        s.set_populations(g)
    s.set_populations(f)  # a clean upload after refused ones
    assert np.abs(s.get_populations() - f).max() < {"fp64": 1e-15, "fp32": 1e-7, "fp16": 1e-4}[prec]
    s.step(1)
    s.sync()
    s.close()


def test_watchdog_with_capsule_then_restore():
    """A coupled FP32 step whose lattice gets a cell of density 3 far from the
    capsule: UNSTABLE is reported; a checkpoint taken before restores a state
    that steps clean."""
    from cases import gpu_sim

    c = W.Capsule((19.2, 17.7, 13.6), 5.0, 3, W.k_s_for(0.05, 5.0))
    case = W.Case("fail", (40, 36, 28), 1.0, 3, "fp32", 0.02, [c], 4)
    s = gpu_sim(case)
    s.step(2)
    ck = s.checkpoint_save()
    f = s.get_populations()
    f[:, 25, 3, 2] *= 3.0
    s.set_populations(f)
    s.step(1)
    _expect_unstable(s)
    s.checkpoint_restore(ck)
    s.step(2)
    s.sync()
    assert s.info().step == 4
    s.close()
