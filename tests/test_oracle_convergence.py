"""The FP64 oracle's coupled trajectory against the paper's printed results:
the smallest case of the coupled-convergence series of Sec. IV.C (H = 35,
1 280 faces, Re = 0.02, G = 0.01, tau = 1) with the 2-, 3- and 4-point
stencils, each run to kappa t = 120 (4 410 steps, about a minute and a half on
one core; the three run in parallel processes).

Bands.  The paper leaves open the initial fluid state and (through "H^3 fluid
nodes") only loosely fixes the wall placement.  tests/golden/
convergence_readings_h35.txt holds the oracle's deviations under the
alternatives (fluid at rest at t = 0; one fluid layer fewer or more between
the walls at the same shear rate), written by a script that calls only the
oracle.  The band of each printed deviation is the largest change any
alternative makes, plus half a unit of the table's last digit, and never more
than the fixed bands used before (1.2 points for dD, 2.5 for dtheta_o):

  stencil   dD band   (oracle, paper)        dtheta_o band  (oracle, paper)
  phi2      0.91 pp   (12.89 %, 13.2 %)      2.5 pp (capped) (14.07 %, 12.0 %)
  phi3      0.37 pp   (13.85 %, 13.5 %)      0.45 pp         (20.95 %, 20.9 %)
  phi4      0.43 pp   (17.17 %, 17.0 %)      0.45 pp         (31.13 %, 30.8 %)

Volume drift at kappa t = 120 (Sec. V gives the ranges over its runs): the
oracle's |dV/V0| is 1.01e-3 / 2.33e-4 / 3.89e-5 for phi2 / phi3 / phi4, 17 to
30 % above the upper ends of the printed ranges (8e-4, 2e-4, 3e-5).  Under the
alternative readings it moves to 9.1e-4 .. 1.0e-3 (phi2), 1.7e-4 .. 2.3e-4
(phi3) and 3e-6 .. 3.9e-5 (phi4): for phi3 and phi4 the readings' range
overlaps the printed one, for phi2 it stays 13 to 26 % above it.  Checked:
that ordering of the three stencils and the overlap for phi3 and phi4; the
phi2 excess is stated here, not hidden in a band."""
import concurrent.futures as cf
import math
import multiprocessing as mp

import pytest

from conftest import read_golden

pytestmark = pytest.mark.slow

G, H = 0.01, 35
OLD_BAND = {"dD": 0.012, "dth": 0.025}  # the fixed bands the derived ones may not exceed
PRINT_HALF_UNIT = 0.0005  # the table prints fractions to three decimals


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


def readings():
    """{stencil: {reading: (dD, dtheta_o, dV)}} of the oracle's readings study."""
    out = {}
    for r in read_golden("convergence_readings_h35.txt"):
        out.setdefault(int(r[0]), {})[r[1]] = tuple(float(v) for v in r[2:5])
    return out


def bands():
    """{stencil: (dD band, dtheta_o band)} derived from the readings study."""
    rd = readings()
    out = {}
    for d, rows in rd.items():
        base = rows["couette"]
        spread = [max(abs(v[k] - base[k]) for v in rows.values()) for k in (0, 1)]
        out[d] = (min(spread[0] + PRINT_HALF_UNIT, OLD_BAND["dD"]), min(spread[1] + PRINT_HALF_UNIT, OLD_BAND["dth"]))
    return out


def test_readings_study_is_the_oracle_run():
    """The study's 'couette' rows are the library's readings: the same run as
    below (checked there to the printed digits)."""
    rd = readings()
    assert set(rd) == {2, 3, 4} and all(set(v) == {"couette", "rest", "nz34", "nz36"} for v in rd.values())


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
    bd = bands()
    rd = readings()
    with capsys.disabled():
        for d, (dD, dth, dV) in res.items():
            print(f"\noracle H = 35, phi{d}: dD {dD:.4f} (paper {dD_paper[d - 2]}, band {bd[d][0]:.4f}), "
                  f"dtheta_o {dth:.4f} (paper {dth_paper[d - 2]}, band {bd[d][1]:.4f}), dV/V0 {dV:.2e} "
                  f"(paper {vol[d][0]:g}..{vol[d][1]:g} in magnitude)")
    for d, (dD, dth, dV) in res.items():
        # the run is the readings study's own (to the digits it stores)
        assert abs(dD - rd[d]["couette"][0]) < 2e-6 and abs(dth - rd[d]["couette"][1]) < 2e-6, d
        assert abs(dD - dD_paper[d - 2]) <= bd[d][0], d
        assert abs(dth - dth_paper[d - 2]) <= bd[d][1], d
    # wider stencils conserve volume better (Sec. V)
    assert abs(res[2][2]) > abs(res[3][2]) > abs(res[4][2])
    # for phi3 and phi4 the drifts under the readings overlap the printed range
    for d in (3, 4):
        lo, hi = min(abs(v[2]) for v in rd[d].values()), max(abs(v[2]) for v in rd[d].values())
        assert lo <= vol[d][1] and hi >= vol[d][0], d
