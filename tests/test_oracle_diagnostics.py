"""Pins of the oracle's shape and mesh diagnostics (Sec. III, Fig. degrade):
closed forms on rigid rotations, exact ellipsoids and uniform stretches."""
import numpy as np
import pytest

import oracle as O


def _roty(a):
    return np.array([[np.cos(a), 0, np.sin(a)], [0, 1, 0], [-np.sin(a), 0, np.cos(a)]])


def test_tank_treading_rigid_rotation():
    """Rotating every node by alpha about the y axis through the centroid in
    the shear sense (from +z toward +x) gives omega = alpha/dt at every node."""
    x0, _ = O.icosphere(2, 5.0, (0.0, 0.0, 0.0))
    c0 = np.array([10.0, 4.0, 7.0])
    alpha, dt = 0.03, 3.0
    R = _roty(alpha)  # x' = cos a x + sin a z: from +z toward +x
    x1 = x0 @ R.T
    # a centroid that also moves
    c1 = c0 + np.array([0.4, 0.0, -0.1])
    keep = np.abs(x0[:, 0]) + np.abs(x0[:, 2]) > 1e-9  # nodes on the y axis have no angle
    om, _ = O.tank_treading(x0[keep] + c0, x1[keep] + c1, c0, c1, dt)
    assert np.allclose(om, alpha / dt, rtol=0, atol=1e-12)
    # the shear flow's own rotation: u_x = g z moves a point at (x, z) to (x + g z dt, z)
    g = 1e-3
    pts = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 1.0], [-1.0, 0.0, 0.0], [0.0, 0.0, -1.0]]) * 3.0
    # a rigid rotation at rate g: u = (g z, 0, -g x)
    moved = pts + np.stack([g * pts[:, 2], 0 * pts[:, 2], -g * pts[:, 0]], 1)
    om2, mean2 = O.tank_treading(pts, moved, np.zeros(3), np.zeros(3), 1.0)
    assert mean2 == pytest.approx(g, rel=1e-5)
    assert np.all(om2 > 0)


@pytest.mark.parametrize("axes,theta", [((6.0, 5.0, 4.0), 0.3), ((5.0, 5.0, 5.0), 0.0), ((7.0, 4.0, 5.5), -0.4)])
def test_ellipsoid_fit_recovers_exact_ellipsoid(axes, theta):
    """Nodes of an icosphere mapped onto an ellipsoid with semiaxes (a, b, c)
    along (x, y, z), rotated about y by theta: the fit returns the semiaxes,
    D = (max - min)/(max + min) and the angle of the major axis."""
    u, _ = O.icosphere(3, 1.0, (0.0, 0.0, 0.0))
    a, b, c = axes
    p = u * np.array([a, b, c])
    R = _roty(-theta)  # rotates +x toward +z by theta
    q = p @ R.T
    cen = np.array([3.0, -2.0, 11.0])
    r = O.ellipsoid_fit(q + cen, cen)
    s = sorted(axes, reverse=True)
    assert [r["r_a"], r["r_b"], r["r_c"]] == pytest.approx(s, rel=1e-10)
    assert r["D"] == pytest.approx((s[0] - s[2]) / (s[0] + s[2]), abs=1e-10)
    if a > max(b, c):
        assert r["theta"] == pytest.approx(theta, abs=1e-9)
    # the fit parameters of Eq. (chisquare) themselves, for the unrotated ellipsoid
    r0 = O.ellipsoid_fit(p + cen, cen)
    assert [r0["zeta_x"], r0["zeta_y"], r0["zeta_z"]] == pytest.approx([1 / a**2, 1 / b**2, 1 / c**2], rel=1e-10)
    assert abs(r0["zeta_xz"]) < 1e-12


def test_face_area_stats_uniform_stretch_and_shear():
    X0, tri = O.icosphere(2, 4.0, (1.0, 2.0, 3.0))
    st = O.face_area_stats(tri, X0, X0)
    assert st["mean"] == 0.0 and st["std"] == 0.0 and st["max"] == 0.0
    s = 1.07
    x = (X0 - X0.mean(0)) * s + X0.mean(0) + np.array([5.0, 0.0, 0.0])
    st = O.face_area_stats(tri, X0, x)
    assert st["mean"] == pytest.approx(s * s - 1, rel=1e-12)
    assert st["std"] < 1e-12
    # an anisotropic stretch changes every face by its own factor: the three
    # statistics against a direct numpy evaluation of the same areas
    x2 = X0 * np.array([1.2, 1.0, 1.0 / 1.2])
    e1 = x2[tri[:, 1]] - x2[tri[:, 0]]
    e2 = x2[tri[:, 2]] - x2[tri[:, 0]]
    E1 = X0[tri[:, 1]] - X0[tri[:, 0]]
    E2 = X0[tri[:, 2]] - X0[tri[:, 0]]
    r = np.linalg.norm(np.cross(e1, e2), axis=1) / np.linalg.norm(np.cross(E1, E2), axis=1) - 1
    st = O.face_area_stats(tri, X0, x2)
    assert st["mean"] == pytest.approx(r.mean(), rel=1e-12)
    assert st["std"] == pytest.approx(r.std(), rel=1e-9)
    assert st["max"] == pytest.approx(np.abs(r).max(), rel=1e-12)
