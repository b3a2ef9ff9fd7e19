"""Host-side checks of the C ABI library that need no GPU: every function the
header declares is exported, the host-only icosphere matches the oracle's bit
for bit, and creating a simulation without a device fails cleanly."""
import ctypes
import os
import re

import numpy as np
import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "iblbm.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(iblbm_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = _declared()
    for must in ("iblbm_create", "iblbm_destroy", "iblbm_step", "iblbm_set_shear_walls",
                 "iblbm_set_skalak", "iblbm_add_capsule_icosphere", "iblbm_get_velocity",
                 "iblbm_get_nodes", "iblbm_get_taylor"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1004_2416_gb300 import LIB_PATH

    lib = ctypes.CDLL(LIB_PATH)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert lib.iblbm_bounds_checked() == 0


def test_checked_build_exports_every_declared_symbol():
    """The bounds-checked build of the same sources (loaded by the binding
    when IBLBM_LIBRARY=checked) has the same entry points and says so."""
    path = os.path.join(ROOT, "paper_1004_2416_gb300", "lib", "libiblbm_checked.so")
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert lib.iblbm_bounds_checked() == 1


@pytest.mark.parametrize("m", range(0, 6))
def test_icosphere_bit_exact_with_oracle(m):
    import oracle as O
    from paper_1004_2416_gb300 import iblbm as B

    c = (15.5, 63.5 - m, -2.25)
    n1, t1 = B.icosphere(m, 4.0 + 3 * m, c)
    n2, t2 = O.icosphere(m, 4.0 + 3 * m, c)
    assert np.array_equal(t1, t2)
    assert np.array_equal(n1.view(np.int64), n2.view(np.int64))


def test_icosphere_rejects_bad_arguments():
    from paper_1004_2416_gb300 import iblbm as B

    with pytest.raises(B.IblbmError):
        B.icosphere(8, 1.0)
    with pytest.raises(B.IblbmError):
        B.icosphere(2, -1.0)


def test_status_strings():
    from paper_1004_2416_gb300 import iblbm as B

    assert B.iblbm_status_string(B.IBLBM_ERR_STENCIL) == b"IBLBM_ERR_STENCIL"
    assert B.iblbm_status_string(0) == b"IBLBM_OK"


def test_create_without_device_or_with_bad_args_fails_cleanly():
    from paper_1004_2416_gb300 import iblbm as B

    with pytest.raises(B.IblbmError) as e:
        B.Sim(8, 8, 8, tau=0.4)
    assert e.value.code == B.IBLBM_ERR_ARG
    with pytest.raises(B.IblbmError) as e:
        B.Sim(8, 8, 8, delta_points=5)
    assert e.value.code == B.IBLBM_ERR_ARG
    with pytest.raises(B.IblbmError) as e:
        B.Sim(0, 8, 8)
    assert e.value.code == B.IBLBM_ERR_ARG


def test_taylor_gradient_against_oracle_finite_differences():
    """The host reverse pass through the Taylor deformation against central
    differences of the oracle's D (and its D itself)."""
    import oracle as O
    from paper_1004_2416_gb300 import iblbm as B

    rng = np.random.default_rng(3)
    x0, tri = O.icosphere(2, 4.0, (10.0, 11.0, 9.0))
    th = 0.4
    R = np.array([[np.cos(th), 0, -np.sin(th)], [0, 1, 0], [np.sin(th), 0, np.cos(th)]])
    x = ((x0 - x0.mean(0)) * np.array([1.2, 1.0, 0.85])) @ R.T + x0.mean(0) + 0.05 * rng.standard_normal(x0.shape)
    D, g = B.taylor_gradient(x, tri)
    assert D == pytest.approx(O.taylor(x, tri)["D"], rel=1e-12)
    h = 1e-6
    for _ in range(6):
        d = rng.standard_normal(x.shape)
        d /= np.linalg.norm(d)
        fd = (O.taylor(x + h * d, tri)["D"] - O.taylor(x - h * d, tri)["D"]) / (2 * h)
        assert np.sum(g * d) == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_diagnostics_against_oracle():
    """The library's host diagnostics (normal equations and a closed-form 2 x 2
    eigen-solution for the fit; cross/dot angles for the rotation) against the
    oracle's (QR and Jacobi; atan2 differences) on a deformed, rotated and
    jittered icosphere."""
    import oracle as O
    from paper_1004_2416_gb300 import iblbm as B

    rng = np.random.default_rng(8)
    X0, tri = O.icosphere(3, 6.0, (0.0, 0.0, 0.0))
    th = 0.37
    R = np.array([[np.cos(th), 0, -np.sin(th)], [0, 1, 0], [np.sin(th), 0, np.cos(th)]])
    x = (X0 * np.array([1.25, 0.95, 0.8])) @ R.T + 0.02 * rng.standard_normal(X0.shape)
    c = np.array([20.0, 30.0, 15.0])
    x = x + c
    a = B.ellipsoid_fit(x, c)
    b = O.ellipsoid_fit(x, c)
    for k in O.FIT_KEYS:
        assert a[k] == pytest.approx(b[k], rel=1e-10, abs=1e-12), k
    # tank-treading between two snapshots
    y = (x - c) @ np.array([[np.cos(0.02), 0, np.sin(0.02)], [0, 1, 0], [-np.sin(0.02), 0, np.cos(0.02)]]).T + c + 0.3
    om_a, m_a = B.tank_treading(x, y, c, c + 0.3, 2.0)
    om_b, m_b = O.tank_treading(x, y, c, c + 0.3, 2.0)
    assert np.allclose(om_a, om_b, rtol=1e-12, atol=1e-14)
    assert m_a == pytest.approx(m_b, rel=1e-12)
    assert m_a == pytest.approx(0.01, rel=1e-9)
    with pytest.raises(B.IblbmError):
        B.ellipsoid_fit(x[:3], c)


def test_taylor_from_sums_against_oracle():
    """The library's host conversion of a capsule's reduced sums (V, A, c, I)
    into D, theta and the semi-axes (its own 3 x 3 eigen-solver) against the
    oracle's values from its Jacobi route, on a stretched, tilted and jittered
    icosphere."""
    import oracle as O
    from paper_1004_2416_gb300 import iblbm as B

    rng = np.random.default_rng(5)
    x0, tri = O.icosphere(3, 5.0, (12.0, 9.0, 10.0))
    th = -0.3
    R = np.array([[np.cos(th), 0, -np.sin(th)], [0, 1, 0], [np.sin(th), 0, np.cos(th)]])
    x = ((x0 - x0.mean(0)) * np.array([1.3, 0.95, 0.8])) @ R.T + x0.mean(0) + 0.02 * rng.standard_normal(x0.shape)
    ref = O.taylor(x, tri)
    sums = [ref[k] for k in ("V", "A", "c_x", "c_y", "c_z", "I_xx", "I_yy", "I_zz", "I_xy", "I_xz", "I_yz")] + [0.0]
    got = B.taylor_from_sums(np.array(sums))
    for k in ("D", "r_a", "r_b", "r_c"):
        assert got[k] == pytest.approx(ref[k], rel=1e-12), k
    assert got["theta"] == pytest.approx(ref["theta"], abs=1e-12)
    assert got["D"] > 0.1
    with pytest.raises(B.IblbmError):
        B._check(B.iblbm_taylor_from_sums(None, None))


def test_entry_points_reject_a_null_object():
    """Calls on no object return IBLBM_ERR_ARG without touching a device."""
    from paper_1004_2416_gb300 import iblbm as B

    assert B.iblbm_set_launch_overlap(None, 1) == B.IBLBM_ERR_ARG
    assert B.iblbm_set_interp_mode(None, 0) == B.IBLBM_ERR_ARG
    assert B.iblbm_read_async(None, None, None) == B.IBLBM_ERR_ARG
    assert B.iblbm_step(None, 1) == B.IBLBM_ERR_ARG
    assert B.iblbm_sync(None) == B.IBLBM_ERR_ARG
