"""The collide-and-stream kernel that stages its populations in shared memory
by bulk copies (Eq. lbequation with Guo forcing and moving walls, the same
arithmetic as the direct-load kernel) against the direct-load kernel, bit for
bit, and against the oracle; and its bounded wait, made to give up from the
host, returning IBLBM_ERR_TIMEOUT with the context left usable."""
import numpy as np
import pytest

import oracle as O
from cases import gpu_sim, oracle_sim, rel_inf
from paper_1004_2416_gb300 import iblbm as B
from paper_1004_2416_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# nx = 4 * lanes per row: 8 .. 1024 cells, row counts that leave the last
# tile partial and the tiles unevenly spread over the persistent blocks
SHAPES = [(8, 5, 7), (32, 9, 6), (64, 7, 5), (128, 37, 9), (256, 13, 29), (512, 3, 7), (1024, 2, 3)]


def _lattice(prec, shape, staging, steps, seed):
    from paper_1004_2416_gb300 import Sim

    nx, ny, nz = shape
    tau, uw = 0.9, 0.04
    f0 = O.init_couette(nx, ny, nz, uw) + W.population_noise(shape, 2e-3, seed=seed)
    s = Sim(nx, ny, nz, tau=tau, precision=prec, delta_points=3)
    s.set_shear_walls(uw)
    s.set_collide_staging(staging)
    s.set_populations(f0)
    s.step(steps)
    f = s.get_populations()
    name = s.collide_kernel()
    s.close()
    return f0, f, name


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
@pytest.mark.parametrize("shape", SHAPES)
def test_staged_equals_direct_and_oracle(prec, shape):
    if prec == "fp16" and shape[0] < 8:
        pytest.skip("a half row of fewer than 8 cells is not a multiple of 16 bytes")
    if prec == "fp32" and shape[0] > 512:
        pytest.skip("a float tile of 512 cells holds no row longer than 512")
    f0, a, na = _lattice(prec, shape, 0, 7, 21)
    _, b, nb = _lattice(prec, shape, 1, 7, 21)
    assert na.startswith("k_collide_stream_x4") and nb.startswith("k_collide_stream_tma"), (na, nb)
    assert np.array_equal(a, b)
    f = f0
    for _ in range(7):
        f = O.lbm_step(f, 0.9, 0.04)
    _, w, _ = O.d3q19()
    wb = w[:, None, None, None]
    assert rel_inf(b - wb, f - wb) < {"fp32": 1e-5, "fp16": 3e-3}[prec]


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_staged_coupled_steps(prec):
    """Coupled steps with a capsule (force flags, Guo term) on a lattice that
    takes the vectorised kernel: staged and direct give the same populations
    and nodes up to the order of the spreading's atomic additions."""
    c = W.Capsule((31.3, 17.6, 14.2), 5.0, 3, W.k_s_for(0.05, 5.0))
    case = W.Case("staged", (64, 36, 29), 1.0, 3, prec, 0.02, [c], 40)
    out = []
    for staging in (0, 1):
        g = gpu_sim(case)
        g.set_collide_staging(staging)
        g.step(40)
        out.append((g.get_populations(), g.get_nodes()))
        g.close()
    tol = {"fp32": 1e-5, "fp16": 2e-3}[prec]
    _, w, _ = O.d3q19()
    wb = w[:, None, None, None]
    assert rel_inf(out[1][0] - wb, out[0][0] - wb) < tol
    assert np.abs(out[1][1] - out[0][1]).max() / 5.0 < tol
    o = oracle_sim(case)
    o.step(40)
    assert np.abs(out[1][1] - o.get_nodes()).max() / 5.0 < {"fp32": 1e-4, "fp16": 2e-3}[prec]


def test_staged_wait_gives_up_and_recovers():
    """A wait limit of 0 makes every block give up at its first wait: the step
    reports IBLBM_ERR_TIMEOUT, the context stays usable, and after the limit is
    restored and good populations uploaded the next step is exact."""
    from paper_1004_2416_gb300 import Sim

    nx, ny, nz = 128, 24, 20
    f0 = O.init_couette(nx, ny, nz, 0.03) + W.population_noise((nx, ny, nz), 1e-3, seed=8)
    s = Sim(nx, ny, nz, tau=1.0, precision="fp16", delta_points=3)
    s.set_shear_walls(0.03)
    s.set_collide_staging(1)
    s.set_populations(f0)
    s.set_device_wait_limit(0)
    s.step(1)
    with pytest.raises(B.IblbmError) as e:
        s.sync()
    assert e.value.code == B.IBLBM_ERR_TIMEOUT
    s.sync()  # reported once
    s.set_device_wait_limit(1_000_000_000)
    s.set_populations(f0)
    s.step(2)
    s.sync()
    _, ref, _ = _lattice("fp16", (nx, ny, nz), 0, 0, 8)
    f = O.lbm_step(O.lbm_step(f0, 1.0, 0.03), 1.0, 0.03)
    _, w, _ = O.d3q19()
    wb = w[:, None, None, None]
    assert rel_inf(s.get_populations() - wb, f - wb) < 3e-3
    with pytest.raises(B.IblbmError) as e:
        s.set_device_wait_limit(-1)
    assert e.value.code == B.IBLBM_ERR_ARG
    s.close()


def test_staging_refused_where_unsupported():
    from paper_1004_2416_gb300 import Sim

    for args in (((40, 8, 8), "fp32"), ((32, 8, 8), "fp64"), ((1024, 2, 3), "fp32"), ((4, 8, 8), "fp16")):
        s = Sim(*args[0], precision=args[1], delta_points=3)
        with pytest.raises(B.IblbmError) as e:
            s.set_collide_staging(1)
        assert e.value.code == B.IBLBM_ERR_STATE
        s.set_collide_staging(0)
        s.set_collide_staging(-1)
        s.close()
