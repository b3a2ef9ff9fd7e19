"""Pins of the oracle's icosphere (Sec. II.D, Tab. mesh_quality) and of its
shape measures (Sec. III).  CPU only."""
import numpy as np
import pytest

import oracle as O
from conftest import read_golden


def _golden():
    return {row[0]: (float(row[1]), int(row[2])) for row in read_golden("mesh_quality.txt")}


def _edges(tri):
    e = {}
    for t in tri:
        for k in range(3):
            a, b = int(t[k]), int(t[(k + 1) % 3])
            e.setdefault((min(a, b), max(a, b)), []).append((a, b))
    return e


@pytest.mark.parametrize("m", [0, 1, 2, 3, 4])
def test_counts_closed_oriented(m):
    x, tri = O.icosphere(m, 2.5, (1.0, 2.0, 3.0))
    nf = 20 * 4 ** m
    assert len(tri) == nf
    assert 2 * len(x) == nf + 4  # Sec. II.D
    e = _edges(tri)
    assert len(x) - len(e) + nf == 2  # Euler characteristic of a sphere
    for uses in e.values():  # every edge in two faces, opposite directions
        assert len(uses) == 2 and uses[0] == (uses[1][1], uses[1][0])
    assert np.allclose(np.linalg.norm(x - np.array([1.0, 2.0, 3.0]), axis=1), 2.5, rtol=1e-15)
    c = x[tri].mean(axis=1) - np.array([1.0, 2.0, 3.0])
    n = np.cross(x[tri[:, 1]] - x[tri[:, 0]], x[tri[:, 2]] - x[tri[:, 0]])
    assert np.all(np.einsum("ij,ij->i", c, n) > 0)  # outward
    assert len(np.unique(tri, axis=0)) == nf


def _stats(x, tri):
    A = 0.5 * np.linalg.norm(np.cross(x[tri[:, 1]] - x[tri[:, 0]], x[tri[:, 2]] - x[tri[:, 0]]), axis=1)
    nrm = np.cross(x[tri[:, 1]] - x[tri[:, 0]], x[tri[:, 2]] - x[tri[:, 0]])
    nrm /= np.linalg.norm(nrm, axis=1)[:, None]
    e = {}
    for fi, t in enumerate(tri):
        for k in range(3):
            a, b = int(t[k]), int(t[(k + 1) % 3])
            e.setdefault((min(a, b), max(a, b)), []).append(fi)
    lengths = np.array([np.linalg.norm(x[a] - x[b]) for a, b in e])
    phin = np.array([np.arccos(np.clip(nrm[f[0]] @ nrm[f[1]], -1, 1)) for f in e.values()])
    ang = []
    for t in tri:
        p = x[t]
        for k in range(3):
            u, v = p[(k + 1) % 3] - p[k], p[(k + 2) % 3] - p[k]
            ang.append(np.arccos(u @ v / np.linalg.norm(u) / np.linalg.norm(v)))
    ang = np.array(ang)
    deg = np.bincount(np.array(list(e.keys())).ravel())
    return dict(sigma_A_over_A=A.std() / A.mean(), sigma_l_over_l=lengths.std() / lengths.mean(),
                sigma_phin_over_phin=phin.std() / phin.mean(),
                sigma_phie_over_phie=ang.std() / ang.mean(), nn_min=deg.min(), nn_max=deg.max(),
                lbar=lengths.mean())


def test_mesh_quality_table():
    """Tab. mesh_quality, column 'subdivision', N_f = 1280, to the printed digit."""
    g = _golden()
    x, tri = O.icosphere(3, 5.0)
    s = _stats(x, tri)
    assert len(tri) == g["n_faces"][0]
    assert s["nn_min"] == g["nn_min"][0] and s["nn_max"] == g["nn_max"][0]
    for key in ("sigma_A_over_A", "sigma_l_over_l", "sigma_phin_over_phin", "sigma_phie_over_phie"):
        val, digits = g[key]
        assert abs(s[key] - val) <= 0.5 * 10.0 ** (-digits) + 1e-12, key


@pytest.mark.parametrize("m,key", [(2, "lbar_r5_nf320"), (3, "lbar_r5_nf1280"), (4, "lbar_r5_nf5120")])
def test_mean_edge_length_at_r5(m, key):
    """Sec. IV.B: mean edge 1.50, 0.75, 0.38 for N_f = 320, 1280, 5120 at r = 5."""
    val, digits = _golden()[key]
    x, tri = O.icosphere(m, 5.0)
    assert abs(_stats(x, tri)["lbar"] - val) <= 0.5 * 10.0 ** (-digits) + 1e-12


# ---- Sec. III shape measures ----------------------------------------------------

def _rot(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    return q * np.sign(np.diag(r))


def test_eig3_recovers_rotated_spectrum():
    rng = np.random.default_rng(0)
    for _ in range(20):
        Q = _rot(rng)
        lam = np.sort(rng.uniform(-3, 5, 3))
        A = Q @ np.diag(lam) @ Q.T
        ev, vec = O.eig3(A)
        assert np.allclose(ev, lam, atol=1e-13)
        for k in range(3):
            assert np.allclose(A @ vec[:, k], lam[k] * vec[:, k], atol=1e-12)
        assert np.allclose(vec.T @ vec, np.eye(3), atol=1e-13)


def test_regular_icosahedron_volume_and_area():
    r = 3.0
    x, tri = O.icosphere(0, r)
    a = 4.0 * r / np.sqrt(10.0 + 2.0 * np.sqrt(5.0))  # edge of the inscribed icosahedron
    T = O.taylor(x, tri)
    assert T["V"] == pytest.approx(5.0 * (3.0 + np.sqrt(5.0)) / 12.0 * a ** 3, rel=1e-13)
    assert T["A"] == pytest.approx(5.0 * np.sqrt(3.0) * a ** 2, rel=1e-13)
    assert T["D"] < 1e-13


def test_sphere_limit():
    r = 4.0
    err_v = []
    for m in (2, 3, 4, 5):
        x, tri = O.icosphere(m, r, (7.0, -2.0, 1.5))
        T = O.taylor(x, tri)
        assert T["D"] < 1e-12
        assert np.allclose([T["c_x"], T["c_y"], T["c_z"]], [7.0, -2.0, 1.5], atol=1e-12)
        err_v.append(abs(T["V"] / (4.0 / 3.0 * np.pi * r ** 3) - 1.0))
        assert T["A"] < 4.0 * np.pi * r * r
    assert all(b < 0.3 * a for a, b in zip(err_v, err_v[1:]))  # second order
    assert err_v[-1] < 1e-3


@pytest.mark.parametrize("m", [1, 3, 4])
def test_affine_ellipsoid_exact(m):
    """An icosphere stretched to semi-axes (a, b, c) and turned by theta0 about
    y: the inertia formula is covariant under linear maps and isotropic on the
    icosahedral mesh, so D = (a - c)/(a + c) and theta = theta0 exactly."""
    a, b, c, th = 1.3, 1.0, 0.75, 0.55
    x, tri = O.icosphere(m, 5.0)
    x = x * np.array([a, b, c])
    R = np.array([[np.cos(th), 0, -np.sin(th)], [0, 1, 0], [np.sin(th), 0, np.cos(th)]])
    x = x @ R.T + np.array([30.0, 20.0, 10.0])
    T = O.taylor(x, tri)
    assert T["D"] == pytest.approx((a - c) / (a + c), abs=1e-13)
    assert T["theta"] == pytest.approx(th, abs=1e-13)
    assert T["r_a"] / T["r_c"] == pytest.approx(a / c, rel=1e-13)
    assert T["r_b"] / T["r_c"] == pytest.approx(b / c, rel=1e-13)
