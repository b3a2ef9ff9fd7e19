"""GPU-vs-oracle parity through the C ABI.  Every comparison is element by
element on the same seeded inputs.  Tolerances (relative, infinity norm over
the compared array): FP64 build 1e-10 (trajectories) / 1e-12 (one step),
FP32 1e-4 (trajectories) / 1e-5 (one step); FP16 storage has its error stated
against the oracle."""
import numpy as np
import pytest

import oracle as O
from cases import gpu_sim, oracle_sim, rel_inf
from paper_1004_2416_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ONE_STEP_TOL = {"fp64": 1e-12, "fp32": 1e-5, "fp16": 2e-3}
TRAJ_TOL = {"fp64": 1e-10, "fp32": 1e-4}


def _small_case(delta=3, precision="fp32", shape=(40, 36, 28), r=5.0, m=3, G=0.05, steps=300):
    nx, ny, nz = shape
    c = W.Capsule((19.2, 17.7, 13.6), r, m, W.k_s_for(G, r))
    return W.Case("small", shape, 1.0, delta, precision, 0.02, [c], steps)


# ---- lattice only ------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(37, 19, 11), (38, 19, 11)])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
def test_lattice_only_ragged(prec, shape):
    """Collide-stream with moving walls on a ragged lattice (not a multiple of
    the 32 x 8 tile), tau != 1, random start; odd rows take the one-cell
    kernel, even rows (float builds) the two-cells-per-thread kernel."""
    tau, uw = 0.8, 0.03
    nx, ny, nz = shape
    f0 = O.init_couette(nx, ny, nz, uw) + W.population_noise(shape, 2e-3, seed=1)
    from paper_1004_2416_gb300 import Sim

    s = Sim(nx, ny, nz, tau=tau, precision=prec, delta_points=3)
    s.set_shear_walls(uw)
    s.set_populations(f0)
    s.step(40)
    f = f0
    for _ in range(40):
        f = O.lbm_step(f, tau, uw)
    c, w, _ = O.d3q19()
    g_gpu = s.get_populations() - w[:, None, None, None]
    g_ref = f - w[:, None, None, None]
    tol = {"fp64": 1e-12, "fp32": 1e-5, "fp16": 3e-3}[prec]
    assert rel_inf(g_gpu, g_ref) < tol
    u_ref = np.einsum("ia,izyx->azyx", c.astype(float), f) / f.sum(axis=0)
    assert rel_inf(s.get_velocity(), u_ref) < tol
    mass_tol = {"fp64": 1e-13, "fp32": 1e-8, "fp16": 1e-5}[prec]  # rounding of the storage type
    assert abs(s.get_density().sum() - f.sum(axis=0).sum()) / f.sum(axis=0).sum() < mass_tol


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
@pytest.mark.parametrize("shape", [(4, 3, 5), (8, 5, 7), (32, 9, 6), (64, 7, 5), (128, 5, 9),
                                   (256, 3, 7), (512, 2, 3), (1024, 1, 3)])
def test_lattice_vectorised_rows(shape, prec):
    """The 4-cells-per-thread collide-stream (nx/4 a power of two <= 32), with
    row counts that leave idle lanes in the last block."""
    nx, ny, nz = shape
    tau, uw = 0.9, 0.04
    f0 = O.init_couette(nx, ny, nz, uw) + W.population_noise(shape, 2e-3, seed=11)
    from paper_1004_2416_gb300 import Sim

    s = Sim(nx, ny, nz, tau=tau, precision=prec, delta_points=3)
    s.set_shear_walls(uw)
    s.set_populations(f0)
    s.step(23)
    f = f0
    for _ in range(23):
        f = O.lbm_step(f, tau, uw)
    _, w, _ = O.d3q19()
    wb = w[:, None, None, None]
    tol = {"fp32": 1e-5, "fp16": 3e-3}[prec]
    assert rel_inf(s.get_populations() - wb, f - wb) < tol


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
@pytest.mark.parametrize("shape", [(256, 48, 52), (512, 32, 40)])
def test_lattice_long_rows_full_blocks(shape, prec):
    """Rows of two and four warps on lattices of a few thousand rows (every
    block full): the warp-edge cells come from shared memory across the warps
    of a block."""
    nx, ny, nz = shape
    tau, uw = 0.9, 0.04
    f0 = O.init_couette(nx, ny, nz, uw) + W.population_noise(shape, 2e-3, seed=12)
    from paper_1004_2416_gb300 import Sim

    s = Sim(nx, ny, nz, tau=tau, precision=prec, delta_points=3)
    s.set_shear_walls(uw)
    s.set_populations(f0)
    s.step(3)
    f = f0
    for _ in range(3):
        f = O.lbm_step(f, tau, uw)
    _, w, _ = O.d3q19()
    wb = w[:, None, None, None]
    tol = {"fp32": 1e-5, "fp16": 3e-3}[prec]
    assert rel_inf(s.get_populations() - wb, f - wb) < tol


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
@pytest.mark.parametrize("delta", [2, 4])
def test_one_step_vectorised_path(prec, delta):
    """Coupled step on a lattice that takes the vectorised kernel (nx = 64)."""
    c = W.Capsule((31.3, 17.6, 14.2), 5.0, 3, W.k_s_for(0.05, 5.0))
    case = W.Case("vec", (64, 36, 29), 1.0, delta, prec, 0.02, [c], 1)
    g = gpu_sim(case)
    o = oracle_sim(case)
    x0 = o.get_nodes() + W.jitter(o.n_nodes, 0.15, seed=13)
    f0 = o.get_f() + W.population_noise(case.shape, 1e-3, seed=14)
    g.set_nodes(x0)
    o.set_nodes(x0)
    g.set_populations(f0)
    o.set_f(f0)
    g.step(1)
    o.step(1)
    tol = ONE_STEP_TOL[prec]
    assert rel_inf(g.get_node_forces(), o.get_node_forces()) < 1e-5
    assert rel_inf(g.get_force_field(), o.get_force_field()) < 1e-5
    _, w, _ = O.d3q19()
    wb = w[:, None, None, None]
    assert rel_inf(g.get_populations() - wb, o.get_f() - wb) < tol
    assert rel_inf(g.get_velocity(), o.get_velocity()) < tol
    assert rel_inf(g.get_node_velocities(), o.get_node_velocities()) < tol
    # a second step: the previous step's force tiles must have been cleared
    g.step(1)
    o.step(1)
    assert rel_inf(g.get_force_field(), o.get_force_field()) < 1e-5
    assert rel_inf(g.get_populations() - wb, o.get_f() - wb) < tol


@pytest.mark.parametrize("shape", [(1, 1, 4), (3, 2, 5), (33, 9, 2)])
def test_lattice_degenerate_shapes(shape):
    nx, ny, nz = shape
    uw = 0.05
    f0 = O.init_couette(nx, ny, nz, uw) + W.population_noise(shape, 1e-3, seed=2)
    from paper_1004_2416_gb300 import Sim

    s = Sim(nx, ny, nz, tau=1.3, precision="fp64", delta_points=2)
    s.set_shear_walls(uw)
    s.set_populations(f0)
    s.step(17)
    f = f0
    for _ in range(17):
        f = O.lbm_step(f, 1.3, uw)
    assert np.abs(s.get_populations() - f).max() < 1e-14


@pytest.mark.parametrize("shape", [(2, 3, 5), (6, 1, 3), (10, 2, 4)])
@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_lattice_short_even_rows(prec, shape):
    """Rows of 2, 6 and 10 cells in the two-cells-per-thread kernel: both
    periodic wraps in x fall on one thread's pair."""
    nx, ny, nz = shape
    uw = 0.05
    f0 = O.init_couette(nx, ny, nz, uw) + W.population_noise(shape, 1e-3, seed=3)
    from paper_1004_2416_gb300 import Sim

    s = Sim(nx, ny, nz, tau=1.3, precision=prec, delta_points=2)
    s.set_shear_walls(uw)
    s.set_populations(f0)
    s.step(17)
    f = f0
    for _ in range(17):
        f = O.lbm_step(f, 1.3, uw)
    _, w, _ = O.d3q19()
    wb = w[:, None, None, None]
    assert rel_inf(s.get_populations() - wb, f - wb) < {"fp32": 1e-5, "fp16": 3e-3}[prec]


# ---- one coupled step, every sub-step compared ------------------------------------------

@pytest.mark.parametrize("delta", [2, 3, 4])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
def test_one_step_all_substeps(prec, delta):
    case = _small_case(delta=delta, precision=prec)
    g = gpu_sim(case)
    o = oracle_sim(case)
    x0 = o.get_nodes() + W.jitter(o.n_nodes, 0.15, seed=3)
    f0 = o.get_f() + W.population_noise(case.shape, 1e-3, seed=4)
    g.set_nodes(x0)
    o.set_nodes(x0)
    g.set_populations(f0)
    o.set_f(f0)
    g.step(1)
    o.step(1)
    tol = ONE_STEP_TOL[prec]
    assert rel_inf(g.get_node_forces(), o.get_node_forces()) < (1e-12 if prec == "fp64" else 1e-5)
    assert rel_inf(g.get_force_field(), o.get_force_field()) < (1e-12 if prec == "fp64" else 1e-5)
    _, w, _ = O.d3q19()
    wb = w[:, None, None, None]
    assert rel_inf(g.get_populations() - wb, o.get_f() - wb) < tol
    assert rel_inf(g.get_velocity(), o.get_velocity()) < tol
    assert rel_inf(g.get_node_velocities(), o.get_node_velocities()) < tol
    assert np.abs(g.get_nodes() - o.get_nodes()).max() < tol * 1e-1


# ---- trajectories -----------------------------------------------------------------------

@pytest.mark.parametrize("delta", [2, 4])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_trajectory_small(prec, delta):
    case = _small_case(delta=delta, precision=prec, steps=300)
    g = gpu_sim(case)
    o = oracle_sim(case)
    g.step(case.steps)
    o.step(case.steps)
    tol = TRAJ_TOL[prec]
    r = case.capsules[0].radius
    assert np.abs(g.get_nodes() - o.get_nodes()).max() / r < tol
    assert rel_inf(g.get_velocity(), o.get_velocity()) < tol
    Tg, To = g.taylor(0), o.taylor(0)
    assert abs(Tg["D"] - To["D"]) / To["D"] < 10 * tol


def test_config1_fp64_full():
    """Config 1 as stated: 32^3, FP64, r = 4, 320 faces, G = 0.0125, phi3,
    1000 steps; fields, nodes and the Taylor deformation at 1e-10."""
    case = W.config1()
    g = gpu_sim(case)
    o = oracle_sim(case)
    g.step(case.steps)
    o.step(case.steps)
    assert np.abs(g.get_nodes() - o.get_nodes()).max() / case.capsules[0].radius < 1e-10
    assert rel_inf(g.get_velocity(), o.get_velocity()) < 1e-10
    assert rel_inf(g.get_density() - 1.0, o.get_density() - 1.0) < 1e-10
    Tg, To = g.taylor(0), o.taylor(0)
    for k in ("D", "theta", "V", "A", "r_a", "r_c"):
        assert abs(Tg[k] - To[k]) <= 1e-10 * abs(To[k]), k


def test_config2_full_size_one_step():
    """Config 2 at full size (128^3, 5120 faces, phi4, FP32): 200 GPU steps from
    the Couette start, then one more step on both sides from the GPU state,
    compared element by element over the whole lattice and mesh."""
    case = W.config2(G=0.0125, delta=4)
    g = gpu_sim(case)
    g.step(200)
    m0 = g.get_density().sum()
    f = g.get_populations()
    x = g.get_nodes()
    o = oracle_sim(case)
    o.set_f(f)
    o.set_nodes(x)
    g.step(1)
    o.step(1)
    _, w, _ = O.d3q19()
    wb = w[:, None, None, None]
    assert rel_inf(g.get_node_forces(), o.get_node_forces()) < 1e-5
    assert rel_inf(g.get_force_field(), o.get_force_field()) < 1e-5
    assert rel_inf(g.get_populations() - wb, o.get_f() - wb) < 1e-5
    assert rel_inf(g.get_velocity(), o.get_velocity()) < 1e-5
    assert rel_inf(g.get_node_velocities(), o.get_node_velocities()) < 1e-5
    assert np.abs(g.get_nodes() - o.get_nodes()).max() < 1e-6
    assert abs(g.get_density().sum() - m0) / m0 < 1e-9


# ---- Taylor deformation ------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_taylor_matches_oracle(prec):
    from paper_1004_2416_gb300 import Sim

    s = Sim(48, 48, 48, precision=prec)
    cid = s.add_capsule_icosphere((23.5, 24.0, 22.5), 8.0, 3)
    X0 = s.get_nodes(cid)
    _, tri = s.mesh(cid)
    a, b, c, th = 1.2, 1.0, 0.85, 0.5
    R = np.array([[np.cos(th), 0, -np.sin(th)], [0, 1, 0], [np.sin(th), 0, np.cos(th)]])
    x = ((X0 - X0.mean(0)) * np.array([a, b, c])) @ R.T + X0.mean(0) + W.jitter(len(X0), 0.05, 5)
    s.set_nodes(x, cid)
    xg = s.get_nodes(cid)
    Tg = s.taylor(cid)
    To = O.taylor(xg, tri)
    # FP64 build: double throughout; float builds: per-face terms in float,
    # sums in double (relative error of order 1e-7 in the sums)
    tol = 1e-11 if prec == "fp64" else 2e-6
    scale = {k: max(abs(v), 1.0) for k, v in To.items()}
    for k in ("I_xy", "I_xz", "I_yz"):
        scale[k] = max(scale[k], abs(To["I_xx"]))
    for k, v in To.items():
        assert abs(Tg[k] - v) <= tol * scale[k], (k, Tg[k], v)


# ---- edge cases ------------------------------------------------------------------------------

def test_stencil_beyond_wall_is_reported():
    from paper_1004_2416_gb300 import Sim, iblbm as B

    s = Sim(24, 24, 16, precision="fp32", delta_points=4)
    cid = s.add_capsule_icosphere((12.0, 12.0, 3.2), 3.0, 2)  # reaches z < 0 with phi4
    s.set_skalak(0.01, 1.0, cid)
    s.init_fluid(1)
    s.step(1)
    with pytest.raises(B.IblbmError) as e:
        s.sync()
    assert e.value.code == B.IBLBM_ERR_STENCIL
    s.sync()  # the status is cleared once returned


def test_no_capsules_and_capsule_added_later():
    case = _small_case(precision="fp64", steps=20)
    from paper_1004_2416_gb300 import Sim

    nx, ny, nz = case.shape
    s = Sim(nx, ny, nz, precision="fp64", delta_points=case.delta)
    s.set_shear_walls(case.u_wall)
    s.init_fluid(1)
    s.step(10)
    c = case.capsules[0]
    cid = s.add_capsule_icosphere(c.center, c.radius, c.subdivisions)
    s.set_skalak(c.k_s, 1.0, cid)
    s.step(10)
    o = oracle_sim(case)
    f = o.get_f()
    for _ in range(10):
        f = O.lbm_step(f, 1.0, case.u_wall)
    o.set_f(f)
    o.step(10)
    assert np.abs(s.get_nodes() - o.get_nodes()).max() < 1e-12
    assert rel_inf(s.get_velocity(), o.get_velocity()) < 1e-12


def test_setters_round_trip():
    from paper_1004_2416_gb300 import Sim

    s = Sim(20, 10, 12, precision="fp64")
    cid = s.add_capsule_icosphere((9.5, 4.5, 5.5), 2.5, 2)
    f = O.init_couette(20, 10, 12, 0.01) + W.population_noise((20, 10, 12), 1e-3, 6)
    s.set_populations(f)
    assert np.array_equal(s.get_populations(), f)
    x = s.get_nodes(cid) + W.jitter(162, 0.1, 7)
    s.set_nodes(x, cid)
    assert np.array_equal(s.get_nodes(cid), x)
    s32 = Sim(20, 10, 12, precision="fp32")
    cid = s32.add_capsule_icosphere((9.5, 4.5, 5.5), 2.5, 2)
    s32.set_nodes(x, cid)
    assert np.abs(s32.get_nodes(cid) - x).max() < 1e-12


@pytest.mark.parametrize("every", [1, 5])
def test_taylor_recording_ring(every):
    """Records taken inside the step sequence (direct launches and captured
    graphs, on the side stream) equal the immediate reduction of the same
    state, and the recorded history matches the oracle's trajectory."""
    case = _small_case(delta=3, precision="fp64", steps=0)
    g = gpu_sim(case)
    g.set_taylor_recording(every, ring=512)
    o = oracle_sim(case)
    hist = []
    for chunk in (7, 150, 3):  # 150 covers several graph replays
        g.step(chunk)
        for _ in range(chunk):
            o.step(1)
            hist.append(o.taylor(0)["D"])
    steps, rec = g.taylor_records(0)
    assert list(steps) == [k for k in range(every, 161, every)]
    now = g.taylor(0)
    assert np.array_equal(rec[-1], np.array([now[k] for k in now]))
    for st, r in zip(steps, rec):
        assert abs(r[0] - hist[st - 1]) <= 1e-10 * abs(hist[st - 1]) + 1e-13


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
def test_interp_modes_bit_identical(prec):
    """The interpolation gives the same bits whether every node forms u at its
    stencil cells or reads u formed once per cell of the flagged tiles.  One
    step from the reference shape (zero membrane force, so no atomic sums whose
    order could differ) over a perturbed flow."""
    case = _small_case(precision=prec, steps=1)
    o = oracle_sim(case)
    f0 = o.get_f() + W.population_noise(case.shape, 1e-3, seed=21)
    out = []
    for mode in (0, 1):
        g = gpu_sim(case)
        g.set_populations(f0)
        g.set_interp_mode(mode)
        g.step(1)
        out.append((g.get_nodes(), g.get_node_velocities()))
        g.close()
    assert np.abs(out[0][1]).max() > 0
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


def _dense_case(precision):
    """Eight capsules of 642 nodes (5 136 nodes: the membrane kernels take
    four nodes per warp) on a lattice whose rows take the vectorised kernels."""
    shape = (128, 64, 64)
    r, G = 6.0, 0.02
    centres = W.rsa_centres(shape, 8, r, seed=8, z_margin=r + 4.0)
    caps = [W.Capsule(c, r, 3, W.k_s_for(G, r)) for c in centres]
    return W.Case("dense", shape, 1.0, 3, precision, W.u_wall_for(shape[2]), caps, 1)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
def test_one_step_dense_suspension(prec):
    """Every sub-step of one coupled step with more than 152 x 32 nodes."""
    case = _dense_case(prec)
    g = gpu_sim(case)
    o = oracle_sim(case)
    assert o.n_nodes >= 152 * 32
    x0 = o.get_nodes() + W.jitter(o.n_nodes, 0.15, seed=31)
    f0 = o.get_f() + W.population_noise(case.shape, 1e-3, seed=32)
    g.set_nodes(x0)
    o.set_nodes(x0)
    g.set_populations(f0)
    o.set_f(f0)
    g.step(1)
    o.step(1)
    tol = ONE_STEP_TOL[prec]
    assert rel_inf(g.get_node_forces(), o.get_node_forces()) < (1e-12 if prec == "fp64" else 1e-5)
    assert rel_inf(g.get_force_field(), o.get_force_field()) < (1e-12 if prec == "fp64" else 1e-5)
    _, w, _ = O.d3q19()
    wb = w[:, None, None, None]
    assert rel_inf(g.get_populations() - wb, o.get_f() - wb) < tol
    assert rel_inf(g.get_velocity(), o.get_velocity()) < tol
    assert rel_inf(g.get_node_velocities(), o.get_node_velocities()) < tol
    assert np.abs(g.get_nodes() - o.get_nodes()).max() < tol * 1e-1


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_interp_modes_dense(prec):
    """Above 152 x 32 nodes the velocity-pass mode reduces four nodes per warp
    and the gather mode one: the same node velocities up to the rounding of
    the summation order."""
    case = _dense_case(prec)
    o = oracle_sim(case)
    f0 = o.get_f() + W.population_noise(case.shape, 1e-3, seed=33)
    out = []
    for mode in (0, 1):
        g = gpu_sim(case)
        g.set_populations(f0)
        g.set_interp_mode(mode)
        g.step(1)
        out.append((g.get_nodes(), g.get_node_velocities()))
        g.close()
    assert np.abs(out[0][1]).max() > 0
    assert rel_inf(out[1][1], out[0][1]) < 1e-6
    assert np.abs(out[1][0] - out[0][0]).max() < 1e-7


@pytest.mark.parametrize("dense", [False, True])
def test_launch_overlap_on_and_off(dense):
    """The step kernels launched to overlap their predecessor (programmatic
    dependent launch, the default) and launched one after the other give the
    oracle's trajectory; they differ only by the order of atomic additions."""
    case = _dense_case("fp32") if dense else _small_case(precision="fp32", steps=60)
    steps = 20 if dense else 60
    o = oracle_sim(case)
    f0 = o.get_f() + W.population_noise(case.shape, 1e-3, seed=41)
    x0 = o.get_nodes() + W.jitter(o.n_nodes, 0.1, seed=42)
    o.set_f(f0)
    o.set_nodes(x0)
    o.step(steps)
    out = {}
    for on in (True, False):
        g = gpu_sim(case)
        g.set_launch_overlap(on)
        g.set_populations(f0)
        g.set_nodes(x0)
        g.step(steps)
        out[on] = (g.get_nodes(), g.get_velocity())
        g.close()
    r = case.capsules[0].radius
    for on, (x, u) in out.items():
        assert np.abs(x - o.get_nodes()).max() / r < TRAJ_TOL["fp32"], on
        assert rel_inf(u, o.get_velocity()) < TRAJ_TOL["fp32"], on
    assert np.abs(out[True][0] - out[False][0]).max() / r < 1e-6


def test_kernel_launch_count():
    """The library counts the kernels it launches for time steps, graph
    replays included: three per step (spreading, collide, interpolation), one
    more with the per-cell velocity pass, and one per batch of records."""
    case = _small_case(precision="fp32", steps=0)
    g = gpu_sim(case)
    g.set_interp_mode(0)
    n0 = g.info().kernel_launches
    g.step(70)  # two 32-step graphs and six direct steps
    assert g.info().kernel_launches - n0 == 3 * 70
    g.set_interp_mode(1)
    n1 = g.info().kernel_launches
    g.step(40)
    assert g.info().kernel_launches - n1 == 4 * 40
    g.set_interp_mode(0)
    g.set_taylor_recording(1, ring=256)
    n2 = g.info().kernel_launches
    g.step(64)  # two graphs of 32 steps, each reducing its records in four batches of eight
    g.sync()
    assert g.info().kernel_launches - n2 == 3 * 64 + 8
    g.close()
