"""The FP64 oracle's coupled trajectory against the paper's printed results:
the smallest case of the coupled-convergence series of Sec. IV.C (H = 35,
1 280 faces, Re = 0.02, G = 0.01, tau = 1) with the 2-, 3- and 4-point
stencils, each run to kappa t = 120 (4 410 steps, about a minute and a half on
one core; the three run in parallel processes).  Their deviations from the
small-deformation theory (D_a = 25/4 G, theta_a^o / pi = 15/8 G) are compared
with Tab. convergence and their volume drifts with the ranges Sec. V gives,
with the bands the GPU series uses."""
import concurrent.futures as cf
import math
import multiprocessing as mp

import pytest

from conftest import read_golden

pytestmark = pytest.mark.slow

G, H = 0.01, 35


def _run(delta):
    """(dD, dtheta_o, dV/V0) of the oracle on the H = 35 case with `delta` points."""
    import oracle as O
    from paper_1004_2416_gb300 import workloads as W

    case = W.convergence_case(H, delta)
    cap = case.capsules[0]
    X0, tri = O.icosphere(cap.subdivisions, cap.radius, cap.center)
    V0 = O.taylor(X0, tri)["V"]
    o = O.Sim(*case.shape, case.tau, case.delta, case.u_wall)
    o.add_capsule(X0, tri, cap.k_s, cap.C * cap.k_s)
    o.step(case.steps)
    T = o.taylor(0)
    Da = 25.0 / 4.0 * G
    tho_a = 15.0 / 8.0 * G * math.pi
    return (T["D"] - Da) / Da, (math.pi / 4.0 - T["theta"] - tho_a) / tho_a, T["V"] / V0 - 1.0


def test_oracle_reproduces_table_convergence_h35(capsys):
    import oracle as O

    O.build()  # before the workers start, so that they only load the library
    dD_paper = {int(r[0]): [float(v) for v in r[2:5]] for r in read_golden("convergence_table.txt")}[H]
    rows = read_golden("convergence_theta_volume.txt")
    dth_paper = {int(r[0]): [float(v) for v in r[2:5]] for r in rows if r[0] != "volume"}[H]
    vol = {int(r[1]): (float(r[2]), float(r[3])) for r in rows if r[0] == "volume"}
    deltas = (2, 3, 4)
    with cf.ProcessPoolExecutor(max_workers=3, mp_context=mp.get_context("spawn")) as ex:
        res = dict(zip(deltas, ex.map(_run, deltas)))
    with capsys.disabled():
        for d, (dD, dth, dV) in res.items():
            print(f"\noracle H = 35, phi{d}: dD {dD:.4f} (paper {dD_paper[d - 2]}), dtheta_o {dth:.4f} "
                  f"(paper {dth_paper[d - 2]}), dV/V0 {dV:.2e} (paper {vol[d][0]:g}..{vol[d][1]:g} in magnitude)")
    for d, (dD, dth, dV) in res.items():
        assert abs(dD - dD_paper[d - 2]) < 0.012, d
        assert abs(dth - dth_paper[d - 2]) < 0.025, d
        lo, hi = vol[d]
        assert 0.5 * lo <= abs(dV) <= 1.5 * hi, d
