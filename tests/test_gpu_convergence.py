"""The coupled-convergence series of Sec. IV.C on the GPU library: nine runs
(H = 35, 70, 140 with 1 280, 5 120, 20 480 faces; 2-, 3- and 4-point
stencils) to kappa t = 120.  Their deviations from the small-deformation
theory are compared with the paper's Tab. convergence and its volume drifts
(tests/golden), and the short-time trajectory of the smallest case with the
FP64 oracle."""
import numpy as np
import pytest

from cases import gpu_sim, oracle_sim, rel_inf
from conftest import read_golden
from paper_1004_2416_gb300 import convergence as C
from paper_1004_2416_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _paper():
    dD = {int(r[0]): [float(v) for v in r[2:5]] for r in read_golden("convergence_table.txt")}
    rows = read_golden("convergence_theta_volume.txt")
    dth = {int(r[0]): [float(v) for v in r[2:5]] for r in rows if r[0] != "volume"}
    vol = {int(r[1]): (float(r[2]), float(r[3])) for r in rows if r[0] == "volume"}
    return dD, dth, vol


@pytest.fixture(scope="module")
def study():
    return {(H, d): C.run_case(W.convergence_case(H, d)) for H in (35, 70, 140) for d in (2, 3, 4)}


def test_against_table(study, capsys):
    dD, dth, vol = _paper()
    with capsys.disabled():
        print("\nH  phi  dD (paper)      dtheta_o (paper)   dV/V0")
        for (H, d), r in sorted(study.items()):
            print(f"{H:3d} {d}  {r['dD']:.4f} ({dD[H][d - 2]:.3f})  {r['dtheta_o']:.4f} ({dth[H][d - 2]:.3f})"
                  f"  {r['volume_drift']:.2e}")
    for (H, d), r in study.items():
        assert abs(r["dD"] - dD[H][d - 2]) < 0.012, (H, d)
        assert abs(r["dtheta_o"] - dth[H][d - 2]) < 0.025, (H, d)
        lo, hi = vol[d]
        assert 0.5 * lo <= abs(r["volume_drift"]) <= 1.5 * hi, (H, d)


def test_convergence_with_resolution(study):
    for d in (2, 3, 4):
        e = [abs(study[(H, d)]["dD"]) for H in (35, 70, 140)]
        assert e[0] > e[1] > e[2], d
    # fitted order of dD ~ N_r^-alpha between 1.2 and 2.5 for phi3 and phi4
    for d in (3, 4):
        e = np.array([study[(H, d)]["dD"] for H in (35, 70, 140)])
        alpha = -np.polyfit(np.log([3.5, 7.0, 14.0]), np.log(e), 1)[0]
        assert 1.2 < alpha < 2.5, (d, alpha)


def test_smallest_case_against_oracle():
    case = W.convergence_case(35, 3)
    case.steps = 300
    g = gpu_sim(case)
    o = oracle_sim(case)
    g.step(case.steps)
    o.step(case.steps)
    r = case.capsules[0].radius
    assert np.abs(g.get_nodes() - o.get_nodes()).max() / r < 1e-4
    assert rel_inf(g.get_velocity(), o.get_velocity()) < 1e-4
    g.close()
