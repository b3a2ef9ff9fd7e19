"""Mesh-degradation statistics of a simulated capsule through the C ABI against
the oracle's, evaluated on the same nodes; the ellipsoid fit and the inertia
tensor give close D for a capsule in shear (Sec. III)."""
import numpy as np
import pytest

import oracle as O
from cases import gpu_sim
from paper_1004_2416_gb300 import iblbm as B
from paper_1004_2416_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_mesh_quality_and_fit(prec):
    c = W.Capsule((19.2, 17.7, 13.6), 5.0, 3, W.k_s_for(0.1, 5.0))
    case = W.Case("diag", (40, 36, 28), 1.0, 3, prec, 0.04, [c], 400)
    g = gpu_sim(case)
    q0 = g.mesh_quality(0)
    # at the start the nodes are the reference (float builds keep ~48 bits of them)
    assert abs(q0["dA_mean"]) < 1e-12 and q0["dA_std"] < 1e-12 and abs(q0["dV"]) < 1e-12
    g.step(case.steps - 20)
    x_then = g.get_nodes()
    c_then = np.array([g.taylor(0)[k] for k in ("c_x", "c_y", "c_z")])
    g.step(20)
    x = g.get_nodes()
    X0, tri = O.icosphere(c.subdivisions, c.radius, c.center)
    q = g.mesh_quality(0)
    ref = O.face_area_stats(tri, X0, x)
    assert q["dA_mean"] == pytest.approx(ref["mean"], rel=1e-9, abs=1e-15)
    assert q["dA_std"] == pytest.approx(ref["std"], rel=1e-9, abs=1e-15)
    assert q["dA_max"] == pytest.approx(ref["max"], rel=1e-9)
    assert q["dA_std"] > 0
    T = g.taylor(0)
    V0 = O.taylor(X0, tri)["V"]
    assert q["dV"] == pytest.approx(O.taylor(x, tri)["V"] / V0 - 1, rel=1e-6, abs=1e-12)
    cen = np.array([T["c_x"], T["c_y"], T["c_z"]])
    fit = B.ellipsoid_fit(x, cen)
    # the library's fit of the GPU-run shape against the oracle's (QR and
    # Jacobi) on the same nodes, then the physics: the fitted ellipsoid and
    # the inertia tensor describe the same mildly deformed shape
    ofit = O.ellipsoid_fit(x, cen)
    for k in O.FIT_KEYS:
        assert fit[k] == pytest.approx(ofit[k], rel=1e-9, abs=1e-12), k
    assert fit["D"] == pytest.approx(T["D"], rel=0.1)
    # rotation rates over the last 20 steps (angles well below pi, so both
    # routes take the same branch), library against oracle on the nodes away
    # from the rotation axis, whose angles are well conditioned
    om, mean = B.tank_treading(x_then, x, c_then, cen, 20.0)
    om_o, mean_o = O.tank_treading(x_then, x, c_then, cen, 20.0)
    far = np.hypot(x[:, 0] - cen[0], x[:, 2] - cen[2]) > 0.3 * c.radius
    assert far.sum() > len(x) // 2
    assert np.abs(om - om_o)[far].max() <= 1e-9 * np.abs(om_o[far]).max()
    assert mean == pytest.approx(mean_o, rel=1e-6)
    # the membrane turns with the shear (shear rate 2 u_w / nz; a rigid
    # sphere would turn at half of it, a deforming one at no more than that)
    rate = 2 * case.u_wall / case.shape[2]
    assert 0.05 * rate < np.median(om[far]) < 0.6 * rate
