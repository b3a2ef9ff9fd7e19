"""Pins of the oracle's immersed-boundary coupling (Sec. II.C): the discrete
delta kernels of Eqs. (2point)-(4point) against their defining moment
identities, spreading and interpolation against conservation laws, exactness
on linear fields, and their mutual adjointness.  CPU only."""
import numpy as np
import pytest

import oracle as O

OFFSETS = np.linspace(0.0, 1.0, 41, endpoint=False)


def _sums(n, r, power=1, moment=0, parity=None):
    s = 0.0
    for j in range(-4, 5):
        if parity is not None and (j % 2) != parity:
            continue
        d = r - j
        s += (d ** moment) * O.phi(n, d) ** power
    return s


@pytest.mark.parametrize("n", [2, 3, 4])
def test_partition_of_unity_and_first_moment(n):
    for r in OFFSETS:
        assert abs(_sums(n, r) - 1.0) < 1e-14
        assert abs(_sums(n, r, moment=1)) < 1e-14


def test_sum_of_squares_phi3_phi4():
    for r in OFFSETS:
        assert abs(_sums(3, r, power=2) - 0.5) < 1e-14
        assert abs(_sums(4, r, power=2) - 3.0 / 8.0) < 1e-14


def test_even_odd_sums_phi4():
    for r in OFFSETS:
        assert abs(_sums(4, r, parity=0) - 0.5) < 1e-14
        assert abs(_sums(4, r, parity=1) - 0.5) < 1e-14


def test_branch_joins_and_support():
    assert O.phi(3, 0.5) == pytest.approx(0.5, abs=1e-15)
    assert O.phi(3, 0.5 + 1e-12) == pytest.approx(0.5, abs=1e-9)
    assert O.phi(4, 1.0) == pytest.approx(0.25, abs=1e-15)
    assert O.phi(4, 1.0 + 1e-12) == pytest.approx(0.25, abs=1e-9)
    assert O.phi(2, 0.0) == 1.0
    assert O.phi(3, 1.5) == pytest.approx(0.0, abs=1e-15)
    assert O.phi(4, 2.0) == pytest.approx(0.0, abs=1e-15)
    for n, edge in ((2, 1.0), (3, 1.5), (4, 2.0)):
        for r in (edge + 1e-9, edge + 0.3, 7.0):
            assert O.phi(n, r) == 0.0 and O.phi(n, -r) == 0.0
        for r in np.linspace(0, edge, 50):
            assert O.phi(n, r) == O.phi(n, -r)
            assert O.phi(n, r) >= 0.0


@pytest.mark.parametrize("n", [2, 3, 4])
def test_stencil_covers_support(n):
    rng = np.random.default_rng(n)
    xs = np.concatenate([rng.uniform(-5, 5, 300), np.arange(-3, 4) * 0.5])
    for x in xs:
        b = O.stencil_base(n, x)
        for X in range(int(np.floor(x)) - 5, int(np.floor(x)) + 6):
            if O.phi(n, X - x) != 0.0:
                assert b <= X < b + n


def _nodes(rng, k, shape, margin):
    nx, ny, nz = shape
    lo = np.array([margin, margin, margin])
    hi = np.array([nx, ny, nz]) - 1 - margin
    return lo + (hi - lo) * rng.random((k, 3))


@pytest.mark.parametrize("n", [2, 3, 4])
def test_spread_conserves_force_and_torque(n):
    rng = np.random.default_rng(10 + n)
    shape = (12, 11, 10)
    x = _nodes(rng, 25, shape, 2.5)
    F = rng.standard_normal((25, 3))
    f = O.spread(shape, n, x, F)
    nx, ny, nz = shape
    assert np.allclose(f.reshape(3, -1).sum(axis=1), F.sum(axis=0), atol=1e-13)
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pos = np.stack([X, Y, Z]).reshape(3, -1)
    torque_lat = np.cross(pos.T, f.reshape(3, -1).T).sum(axis=0)
    torque_nodes = np.cross(x, F).sum(axis=0)
    assert np.allclose(torque_lat, torque_nodes, atol=1e-11)


@pytest.mark.parametrize("n", [2, 3, 4])
def test_interpolation_exact_on_linear_fields(n):
    rng = np.random.default_rng(20 + n)
    shape = (10, 9, 11)
    nx, ny, nz = shape
    x = _nodes(rng, 30, shape, 2.5)
    a = rng.standard_normal(3)
    B = rng.standard_normal((3, 3))
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pos = np.stack([X, Y, Z]).astype(float)
    u = a[:, None, None, None] + np.einsum("ab,bzyx->azyx", B, pos)
    ui = O.interpolate(n, x, u)
    assert np.allclose(ui, a + x @ B.T, atol=1e-12)


@pytest.mark.parametrize("n", [2, 3, 4])
def test_spread_interpolate_adjoint(n):
    """sum_i F_i . (I u)_i = sum_X (S F)(X) . u(X), including periodic wrap."""
    rng = np.random.default_rng(30 + n)
    shape = (8, 7, 12)
    nx, ny, nz = shape
    x = rng.random((40, 3)) * np.array([nx, ny, 1.0]) + np.array([-3.0, -2.0, 4.0])
    x[:, 0] += rng.integers(-2, 3, 40) * nx  # unwrapped coordinates
    F = rng.standard_normal((40, 3))
    u = rng.standard_normal((3, nz, ny, nx))
    lhs = np.sum(F * O.interpolate(n, x, u))
    rhs = np.sum(O.spread(shape, n, x, F) * u)
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))


def test_stencil_outside_walls_is_an_error():
    with pytest.raises(ValueError):
        O.spread((8, 8, 8), 3, np.array([[4.0, 4.0, 0.2]]), np.ones((1, 3)))
    with pytest.raises(ValueError):
        O.interpolate(4, np.array([[4.0, 4.0, 6.5]]), np.zeros((3, 8, 8, 8)))
    O.spread((8, 8, 8), 2, np.array([[4.0, 4.0, 0.2]]), np.ones((1, 3)))
