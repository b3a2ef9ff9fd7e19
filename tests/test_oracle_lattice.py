"""Pins of the oracle's lattice Boltzmann part (Sec. II.A) against closed forms,
the printed velocity set and exact special cases.  CPU only."""
import numpy as np
import pytest

import oracle as O
from conftest import read_golden


def test_velocity_set_matches_figure():
    c, _, _ = O.d3q19()
    gold = np.array([[int(v) for v in row[1:]] for row in read_golden("d3q19_figure.txt")])
    assert np.array_equal(c, gold)


def test_opposites():
    c, w, opp = O.d3q19()
    for i in range(19):
        assert np.array_equal(c[opp[i]], -c[i])
        assert w[opp[i]] == w[i]
    assert sorted(opp.tolist()) == list(range(19))


def test_weight_isotropy():
    c, w, _ = O.d3q19()
    c = c.astype(float)
    d = np.eye(3)
    assert np.isclose(w.sum(), 1.0, rtol=0, atol=1e-15)
    assert np.allclose(np.einsum("i,ia->a", w, c), 0.0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), d / 3.0, atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0.0, atol=1e-16)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9.0
    assert np.allclose(m4, iso, atol=1e-15)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_equilibrium_moments(seed):
    rng = np.random.default_rng(seed)
    c, _, _ = O.d3q19()
    rho = 1.0 + 0.1 * rng.standard_normal()
    u = 0.05 * rng.standard_normal(3)
    f = np.array([O.feq(i, rho, u) for i in range(19)])
    assert np.isclose(f.sum(), rho, rtol=1e-14)
    assert np.allclose(c.T @ f, rho * u, atol=1e-15)
    P = np.einsum("i,ia,ib->ab", f, c, c)
    assert np.allclose(P, rho * (np.eye(3) / 3.0 + np.outer(u, u)), atol=1e-15)


@pytest.mark.parametrize("tau", [0.6, 1.0, 1.7])
def test_guo_moments(tau):
    rng = np.random.default_rng(7)
    c, _, _ = O.d3q19()
    u = 0.05 * rng.standard_normal(3)
    f = 1e-3 * rng.standard_normal(3)
    F = np.array([O.guo(i, tau, u, f) for i in range(19)])
    k = 1.0 - 1.0 / (2.0 * tau)
    assert abs(F.sum()) < 1e-18
    assert np.allclose(c.T @ F, k * f, atol=1e-18)
    P = np.einsum("i,ia,ib->ab", F, c, c)
    assert np.allclose(P, k * (np.outer(u, f) + np.outer(f, u)), atol=1e-18)


def test_moments_recover_equilibrium_velocity():
    rng = np.random.default_rng(3)
    rho = 1.02
    u = np.array([0.03, -0.01, 0.02])
    force = 1e-3 * rng.standard_normal(3)
    f = np.array([O.feq(i, rho, u) for i in range(19)])
    r, uu = O.moments(f, force)
    assert np.isclose(r, rho, rtol=1e-15)
    assert np.allclose(uu, u + 0.5 * force / rho, atol=1e-16)


def _stream_expected(rho, u_wall):
    """Exact result of one step at tau = 1 from f_i = w_i rho(x) (u = 0): the
    post-collision state is the rest equilibrium w_i rho(x), which moves to
    x + c_i; populations leaving through a wall plane come back reversed with
    Ladd's moving-wall term 2 w_i (c_i . u_w) / c_s^2 for the outgoing c_i."""
    c, w, opp = O.d3q19()
    nz, ny, nx = rho.shape
    out = np.zeros((19, nz, ny, nx))
    for i in range(19):
        post = w[i] * rho
        cx, cy, cz = c[i]
        moved = np.roll(np.roll(post, cx, axis=2), cy, axis=1)
        if cz == 0:
            out[i] = moved
        elif cz == 1:
            out[i, 1:] = moved[:-1]
        else:
            out[i, :-1] = moved[1:]
    for i in range(19):
        cx, cy, cz = c[i]
        if cz == 0:
            continue
        j = opp[i]  # outgoing direction after reflection
        if cz == 1:  # hits the top plane (wall velocity +u_wall)
            out[j, -1] = w[i] * rho[-1] + 2.0 * w[j] * (c[j][0] * u_wall) * 3.0
        else:  # hits the bottom plane (wall velocity -u_wall)
            out[j, 0] = w[i] * rho[0] + 2.0 * w[j] * (c[j][0] * -u_wall) * 3.0
    return out


@pytest.mark.parametrize("u_wall", [0.0, 0.04])
def test_streaming_and_moving_wall_exact(u_wall):
    rng = np.random.default_rng(11)
    nx, ny, nz = 5, 4, 6
    rho = 1.0 + 0.01 * rng.standard_normal((nz, ny, nx))
    _, w, _ = O.d3q19()
    f = w[:, None, None, None] * rho[None]
    out = O.lbm_step(f, 1.0, u_wall)
    exp = _stream_expected(rho, u_wall)
    assert np.allclose(out, exp, rtol=0, atol=1e-15)


@pytest.mark.parametrize("tau", [0.7, 1.0, 1.5])
def test_mass_conservation(tau):
    rng = np.random.default_rng(5)
    nx, ny, nz = 6, 5, 7
    _, w, _ = O.d3q19()
    f = w[:, None, None, None] * (1.0 + 0.02 * rng.random((19, nz, ny, nx)))
    force = 1e-3 * rng.standard_normal((3, nz, ny, nx))
    m0 = f.sum()
    for _ in range(30):
        f = O.lbm_step(f, tau, 0.03, force)
    assert abs(f.sum() - m0) / m0 < 1e-13


def test_couette_is_stationary_at_tau_one():
    nx, ny, nz = 3, 2, 16
    u_wall = 0.05
    f = O.init_couette(nx, ny, nz, u_wall)
    for _ in range(200):
        f = O.lbm_step(f, 1.0, u_wall)
    c, _, _ = O.d3q19()
    rho = f.sum(axis=0)
    ux = np.einsum("i,izyx->zyx", c[:, 0].astype(float), f) / rho
    z = np.arange(nz)
    exact = 2.0 * u_wall / nz * (z - 0.5 * (nz - 1))
    assert np.allclose(rho, 1.0, atol=1e-14)
    assert np.allclose(ux, exact[:, None, None], atol=1e-15)
    uz = np.einsum("i,izyx->zyx", c[:, 2].astype(float), f) / rho
    assert np.allclose(uz, 0.0, atol=1e-15)


def test_couette_linear_profile_other_tau():
    """Half-way bounce-back carries the linear Couette profile exactly in BGK;
    away from tau = 1 the start from equilibrium relaxes to it."""
    nx, ny, nz = 2, 2, 10
    u_wall = 0.03
    f = O.init_couette(nx, ny, nz, u_wall)
    for _ in range(600):
        f = O.lbm_step(f, 0.8, u_wall)
    c, _, _ = O.d3q19()
    rho = f.sum(axis=0)
    ux = np.einsum("i,izyx->zyx", c[:, 0].astype(float), f) / rho
    z = np.arange(nz)
    exact = 2.0 * u_wall / nz * (z - 0.5 * (nz - 1))
    assert np.allclose(ux, exact[:, None, None], atol=1e-12)


@pytest.mark.parametrize("tau", [0.6, 1.0, 1.9])
def test_momentum_gain_equals_force(tau):
    """Collision with the half-force velocity of Eq. (lbmmomenta1) plus the Guo
    term of Eq. (latticeforce) adds exactly f(X) to the momentum of each cell;
    with the fluid at rest near the walls the walls exchange nothing in one
    step, so the lattice gains sum_X f(X)."""
    rng = np.random.default_rng(17)
    nx, ny, nz = 6, 5, 9
    c, w, _ = O.d3q19()
    f = w[:, None, None, None] * np.ones((19, nz, ny, nx))
    force = np.zeros((3, nz, ny, nx))
    force[:, 2:nz - 2] = 1e-3 * rng.standard_normal((3, nz - 4, ny, nx))
    out = O.lbm_step(f, tau, 0.0, force)
    j0 = np.einsum("ia,izyx->a", c.astype(float), f)
    j1 = np.einsum("ia,izyx->a", c.astype(float), out)
    assert np.allclose(j1 - j0, force.reshape(3, -1).sum(axis=1), atol=1e-15)
