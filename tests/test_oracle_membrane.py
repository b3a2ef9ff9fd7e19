"""Pins of the oracle's finite-element Skalak membrane (Sec. II.B) against
closed-form deformations, invariance and finite differences.  CPU only."""
import numpy as np
import pytest

import oracle as O


def _rot(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def _skalak(I1, I2, ks, ka):
    # Eq. (constitutivelaw)
    return ks / 12.0 * (I1 * I1 + 2.0 * I1 - 2.0 * I2) + ka / 12.0 * I2 * I2


def _planar_triangle(rng):
    p = np.array([[0.0, 0.0], [1.0 + rng.random(), 0.2 * rng.standard_normal()],
                  [0.3 * rng.standard_normal(), 0.8 + rng.random()]])
    return p


@pytest.mark.parametrize("seed", range(6))
def test_anisotropic_stretch_closed_form(seed):
    """In-plane deformation gradient R diag(l1, l2) R^T of a triangle: the
    principal stretches are l1, l2, so I1 = l1^2 + l2^2 - 2 and
    I2 = l1^2 l2^2 - 1 whatever the orientation of triangle and frame."""
    rng = np.random.default_rng(seed)
    p = _planar_triangle(rng)
    l1, l2 = 0.7 + 0.6 * rng.random(2)
    a = rng.uniform(0, np.pi)
    R2 = np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]])
    Fd = R2 @ np.diag([l1, l2]) @ R2.T
    q = p @ Fd.T
    X0 = np.c_[p, np.zeros(3)] @ _rot(rng).T + rng.standard_normal(3)
    x = np.c_[q, np.zeros(3)] @ _rot(rng).T + rng.standard_normal(3)
    I1, I2 = O.face_invariants(X0, x)
    assert I1 == pytest.approx(l1 ** 2 + l2 ** 2 - 2.0, abs=1e-13)
    assert I2 == pytest.approx(l1 ** 2 * l2 ** 2 - 1.0, abs=1e-13)
    ks, ka = 0.3, 0.7
    e1, e2 = p[1] - p[0], p[2] - p[0]
    A0 = 0.5 * abs(e1[0] * e2[1] - e1[1] * e2[0])
    assert O.face_energy(X0, x, ks, ka) == pytest.approx(A0 * _skalak(I1, I2, ks, ka), rel=1e-12)


def test_simple_shear_invariants():
    """Simple shear [[1, g], [0, 1]]: lambda1^2 + lambda2^2 = 2 + g^2,
    lambda1 lambda2 = 1."""
    rng = np.random.default_rng(1)
    p = _planar_triangle(rng)
    for g in (0.05, 0.3, 1.1):
        q = p @ np.array([[1.0, g], [0.0, 1.0]]).T
        I1, I2 = O.face_invariants(np.c_[p, np.zeros(3)], np.c_[q, np.zeros(3)])
        assert I1 == pytest.approx(g * g, abs=1e-13)
        assert I2 == pytest.approx(0.0, abs=1e-13)


@pytest.mark.parametrize("lam", [0.9, 1.0, 1.05, 1.3])
def test_uniform_stretch_closed_form(lam):
    X0, tri = O.icosphere(2, 3.0)
    ks, ka = 0.05, 0.05
    W, F = O.membrane_forces(X0, lam * X0, tri, ks, ka)
    I1 = 2 * lam ** 2 - 2
    I2 = lam ** 4 - 1
    A0 = sum(0.5 * np.linalg.norm(np.cross(X0[t[1]] - X0[t[0]], X0[t[2]] - X0[t[0]])) for t in tri)
    assert W == pytest.approx(A0 * _skalak(I1, I2, ks, ka), rel=1e-12, abs=1e-15)
    if lam == 1.0:
        assert np.abs(F).max() < 1e-14


def test_rigid_motion_gives_no_force():
    rng = np.random.default_rng(2)
    X0, tri = O.icosphere(3, 5.0, (10.0, 11.0, 12.0))
    R = _rot(rng)
    x = (X0 - X0.mean(0)) @ R.T + X0.mean(0) + rng.standard_normal(3)
    W, F = O.membrane_forces(X0, x, tri, 0.1, 0.1)
    assert abs(W) < 1e-15
    assert np.abs(F).max() < 1e-13


def test_finite_differences_of_energy():
    rng = np.random.default_rng(4)
    for _ in range(5):
        X0 = rng.standard_normal((3, 3))
        x = X0 @ (np.eye(3) + 0.2 * rng.standard_normal((3, 3))).T
        ks, ka = 0.4, 0.9
        _, F = O.face_forces(X0, x, ks, ka)
        h = 1e-6
        g = np.zeros(9)
        for k in range(9):
            xp = x.ravel().copy()
            xm = x.ravel().copy()
            xp[k] += h
            xm[k] -= h
            g[k] = (O.face_energy(X0, xp, ks, ka) - O.face_energy(X0, xm, ks, ka)) / (2 * h)
        assert np.allclose(-g, F.ravel(), rtol=1e-6, atol=1e-9 * np.abs(F).max())


def test_net_force_and_torque_vanish():
    rng = np.random.default_rng(9)
    X0, tri = O.icosphere(3, 6.0, (20.0, 20.0, 20.0))
    x = X0 + 0.3 * rng.standard_normal(X0.shape)
    W, F = O.membrane_forces(X0, x, tri, 0.05, 0.05)
    assert W > 0
    scale = np.abs(F).max()
    assert np.abs(F.sum(axis=0)).max() < 1e-12 * scale * len(F)
    torque = np.cross(x, F).sum(axis=0)
    assert np.abs(torque).max() < 1e-11 * scale * len(F) * 20.0


def test_node_forces_assemble_face_forces():
    """The membrane routine sums per-face corner forces over adjacent faces."""
    rng = np.random.default_rng(12)
    X0, tri = O.icosphere(1, 2.0)
    x = X0 + 0.05 * rng.standard_normal(X0.shape)
    _, F = O.membrane_forces(X0, x, tri, 0.2, 0.3)
    G = np.zeros_like(F)
    for t in tri:
        _, Ff = O.face_forces(X0[t], x[t], 0.2, 0.3)
        G[t] += Ff
    assert np.allclose(F, G, atol=1e-15)
