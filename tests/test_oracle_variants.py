"""Pins of the two method variants the paper describes beside the main
scheme: the linearised equilibrium of Sec. IV.A and the Adams-Bashforth node
advection of Sec. II.C (oracle only, no GPU)."""
import numpy as np
import pytest

import oracle as O


def _c():
    c, w, _ = O.d3q19()
    return c.astype(float), w


@pytest.mark.parametrize("u", [(0.0, 0.0, 0.0), (0.03, -0.02, 0.01), (0.1, 0.05, -0.07)])
@pytest.mark.parametrize("rho", [1.0, 0.93])
def test_linear_equilibrium_moments(u, rho):
    """Zeroth and first moments as the full equilibrium, second moment
    rho/3 I without the rho u u of Eq. (equilibrium)."""
    c, _ = _c()
    f = np.array([O.feq_linear(i, rho, u) for i in range(19)])
    ff = np.array([O.feq(i, rho, u) for i in range(19)])
    u = np.array(u)
    assert f.sum() == pytest.approx(rho, abs=1e-15)
    assert np.allclose(c.T @ f, rho * u, atol=1e-15)
    assert np.allclose(np.einsum("ia,ib,i->ab", c, c, f), rho / 3 * np.eye(3), atol=1e-15)
    assert np.allclose(np.einsum("ia,ib,i->ab", c, c, ff), rho * (np.eye(3) / 3 + np.outer(u, u)), atol=1e-15)


def test_linear_equilibrium_couette_stationary_and_mass():
    """The linear Couette velocity profile, started from the linearised
    equilibrium, stays stationary at tau = 1 (u.grad u = 0 for it, and the
    half-way moving walls hold a linear profile), and a random state keeps its
    mass."""
    nx, ny, nz, uw = 4, 3, 12, 0.03
    gamma = 2 * uw / nz
    f = np.zeros((19, nz, ny, nx))
    for z in range(nz):
        u = (gamma * (z - 0.5 * (nz - 1)), 0.0, 0.0)
        for i in range(19):
            f[i, z] = O.feq_linear(i, 1.0, u)
    c, _ = _c()
    g = f
    for _ in range(20):
        g = O.lbm_step(g, 1.0, uw, order=1)
    rho = g.sum(axis=0)
    ux = np.einsum("i,izyx->zyx", c[:, 0], g) / rho
    prof = gamma * (np.arange(nz) - 0.5 * (nz - 1))
    assert np.abs(ux - prof[:, None, None]).max() < 1e-15
    assert np.abs(rho - 1.0).max() < 1e-15
    rng = np.random.default_rng(5)
    f2 = f + 1e-3 * rng.standard_normal(f.shape)
    g2 = O.lbm_step(f2, 0.8, uw, order=1)
    assert g2.sum() == pytest.approx(f2.sum(), rel=1e-14)
    # the two equilibria agree at rest
    f0 = np.broadcast_to(_c()[1][:, None, None, None], f.shape).copy()
    assert np.array_equal(O.lbm_step(f0, 0.8, 0.0, order=1), O.lbm_step(f0, 0.8, 0.0, order=2))


def _drifting_nodes(mode, n):
    """Force-free nodes in a shear flow developing from rest: the velocity at
    a node depends on its height and time only, and heights do not change."""
    nx, ny, nz, uw = 8, 6, 16, 0.04
    s = O.Sim(nx, ny, nz, 1.0, 3, uw)
    _, w = _c()
    s.set_f(np.broadcast_to(w[:, None, None, None], (19, nz, ny, nx)).copy())
    X0, tri = O.icosphere(1, 2.5, (3.5, 2.5, 9.3))
    s.add_capsule(X0, tri, 0.0, 0.0)
    s.set_integrator(mode)
    x0 = s.get_nodes()
    us = []
    for _ in range(n):
        s.step(1)
        us.append(s.get_node_velocities())
    return x0, s.get_nodes(), us


def test_adams_bashforth_telescopes_against_euler():
    """With the same velocity history u_1 .. u_n (Euler first step), the
    Adams-Bashforth positions differ from Euler's by 1/2 (u_n - u_1)."""
    n = 25
    x0, xe, ue = _drifting_nodes(0, n)
    _, xa, ua = _drifting_nodes(1, n)
    for a, b in zip(ue, ua):
        assert np.allclose(a, b, rtol=0, atol=1e-16)
    assert np.abs(ue[-1] - ue[0]).max() > 1e-4  # the velocity does change
    assert np.allclose(xa - xe, 0.5 * (ue[-1] - ue[0]), rtol=0, atol=1e-13)


def test_adams_bashforth_is_euler_for_steady_velocity():
    """In the stationary Couette flow (the oracle's start), node velocities are
    constant and both rules move the nodes alike."""
    s = {}
    for mode in (0, 1):
        o = O.Sim(8, 6, 16, 1.0, 3, 0.04)
        X0, tri = O.icosphere(1, 2.5, (3.5, 2.5, 9.3))
        o.add_capsule(X0, tri, 0.0, 0.0)
        o.set_integrator(mode)
        o.step(12)
        s[mode] = o.get_nodes()
    assert np.allclose(s[0], s[1], rtol=0, atol=1e-13)
