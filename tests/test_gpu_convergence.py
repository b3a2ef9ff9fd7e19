"""The coupled-convergence series of Sec. IV.C on the GPU library: nine runs
(H = 35, 70, 140 with 1 280, 5 120, 20 480 faces; 2-, 3- and 4-point
stencils) to kappa t = 120.

Parity.  At H = 35 each stencil's full run (4 410 steps) is compared with the
FP64 oracle's own run of the same case (tests/golden/
convergence_readings_h35.txt, 'couette' rows, written by a script that calls
only the oracle): the deviations dD and dtheta_o to 1e-4 (FP32 trajectory
tolerance, relative to D and theta^o) and the volume drift to 2e-6 (5 % of
the smallest drift; node positions are double-float pairs).

Paper.  The H = 35 deviations are held to the paper's Tab. convergence with
the bands the oracle's readings study derives (largest change of any
alternative reading of the initial state or wall placement, plus half a
printed unit, never above 1.2 / 2.5 points; see tests/test_oracle_convergence.py).
At H = 70 and 140 no readings study exists (the oracle would need hours), so
the test holds what the paper claims about the trend: the error falls with
resolution, with a fitted order between 1.2 and 2.5 for the 3- and 4-point
stencils (paper 1.9 and 1.5), and wider stencils conserve volume better.  The
measured misses there (printed by the test) are, for dD: phi2 +0.4 / +1.0,
phi3 +0.4 / +0.4, phi4 +0.3 / +0.3 points at H = 70 / 140, i.e. the GPU sits
0.3 to 0.4 points above the table for phi3 and phi4 at every H, which is
larger than the H = 35 readings bands scaled to those resolutions."""
import numpy as np
import pytest

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


def _oracle_h35():
    """{stencil: (dD, dtheta_o, dV)} of the oracle's H = 35 runs (library readings)."""
    return {int(r[0]): tuple(float(v) for v in r[2:5])
            for r in read_golden("convergence_readings_h35.txt") if r[1] == "couette"}


def _bands_h35():
    import test_oracle_convergence as T

    return T.bands()


@pytest.fixture(scope="module")
def study():
    return {(H, d): C.run_case(W.convergence_case(H, d)) for H in (35, 70, 140) for d in (2, 3, 4)}


def test_h35_full_run_against_oracle(study):
    """GPU FP32 against the FP64 oracle after the full 4 410 steps."""
    orc = _oracle_h35()
    G = 0.01
    for d in (2, 3, 4):
        r = study[(35, d)]
        dD_o, dth_o, dV_o = orc[d]
        # deviations relative to D and theta^o themselves
        assert abs(r["dD"] - dD_o) * (25.0 / 4.0 * G) <= 1e-4 * (1 + dD_o) * (25.0 / 4.0 * G), d
        assert abs(r["dtheta_o"] - dth_o) <= 1e-4 * (1 + dth_o), d
        assert abs(r["volume_drift"] - dV_o) <= 2e-6, (d, r["volume_drift"], dV_o)


def test_h35_against_table(study):
    dD, dth, _ = _paper()
    bd = _bands_h35()
    for d in (2, 3, 4):
        r = study[(35, d)]
        assert abs(r["dD"] - dD[35][d - 2]) <= bd[d][0], d
        assert abs(r["dtheta_o"] - dth[35][d - 2]) <= bd[d][1], d


def test_series_trends(study, capsys):
    dD, dth, vol = _paper()
    with capsys.disabled():
        print("\nH  phi  dD (paper, miss pp)          dtheta_o (paper, miss pp)      dV/V0 (paper range)")
        for (H, d), r in sorted(study.items()):
            print(f"{H:3d} {d}  {r['dD']:.4f} ({dD[H][d - 2]:.3f}, {100 * (r['dD'] - dD[H][d - 2]):+.2f})"
                  f"   {r['dtheta_o']:.4f} ({dth[H][d - 2]:.3f}, {100 * (r['dtheta_o'] - dth[H][d - 2]):+.2f})"
                  f"   {r['volume_drift']:.2e} ({vol[d][0]:g}..{vol[d][1]:g})")
    for d in (2, 3, 4):
        e = [abs(study[(H, d)]["dD"]) for H in (35, 70, 140)]
        assert e[0] > e[1] > e[2], d
    # fitted order of dD ~ N_r^-alpha between 1.2 and 2.5 for phi3 and phi4
    for d in (3, 4):
        e = np.array([study[(H, d)]["dD"] for H in (35, 70, 140)])
        alpha = -np.polyfit(np.log([3.5, 7.0, 14.0]), np.log(e), 1)[0]
        assert 1.2 < alpha < 2.5, (d, alpha)
    # wider stencils conserve volume better, at every resolution (Sec. V)
    for H in (35, 70, 140):
        v = [abs(study[(H, d)]["volume_drift"]) for d in (2, 3, 4)]
        assert v[0] > v[1] > v[2], H


def test_smallest_case_against_oracle():
    """Element-wise: nodes and velocity field of the H = 35, 3-point case
    after 300 steps."""
    from cases import gpu_sim, oracle_sim, rel_inf

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
