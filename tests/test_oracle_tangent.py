"""The oracle's tangent-linear derivative (complex-step build of the whole
coupled step, oracle.tangent_taylor_D) pinned to things other than itself:

- its real part is the double oracle's D bit for bit (the complex build runs
  the same arithmetic);
- it matches the central finite differences of the double oracle
  (tests/golden/adjoint_fd_small.json) for dD/dk_s, dD/du_wall and three
  directions of dD/dX0 to 1e-6 relative (the differences' own error: O(h^2)
  truncation with h = 1e-5 relative, rounding of D over 2h);
- it is linear in the direction: the derivative along d1 + 2 d2 is the
  derivative along d1 plus twice that along d2 to rounding;
- it vanishes along a change of k_s when the capsule is never deformed
  (walls at rest).
"""
import importlib.util
import json
import os

import pytest

import oracle as O
from conftest import GOLDEN

_spec = importlib.util.spec_from_file_location("make_adjoint_fd", os.path.join(GOLDEN, "make_adjoint_fd.py"))
FD = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(FD)


def _small():
    c, ndir, _ = FD.case("small")
    cap = c.capsules[0]
    X0, tri = O.icosphere(cap.subdivisions, cap.radius, cap.center)
    return c, cap, X0, tri, ndir


def _tangent(c, cap, X0, tri, steps=None, **kw):
    return O.tangent_taylor_D(c.shape, c.tau, c.delta, c.u_wall, X0, tri, cap.k_s, cap.C,
                              c.steps if steps is None else steps, **kw)


def test_real_part_is_the_double_oracle():
    c, cap, X0, tri, _ = _small()
    D, _ = _tangent(c, cap, X0, tri, steps=40, dks=1.0)
    o = O.Sim(*c.shape, c.tau, c.delta, c.u_wall)
    o.add_capsule(X0, tri, cap.k_s, cap.C * cap.k_s)
    o.step(40)
    assert D == o.taylor(0)["D"]
    o.close()


def test_against_finite_differences():
    c, cap, X0, tri, ndir = _small()
    with open(os.path.join(GOLDEN, "adjoint_fd_small.json")) as fh:
        fd = json.load(fh)
    _, dks = _tangent(c, cap, X0, tri, dks=1.0)
    _, duw = _tangent(c, cap, X0, tri, du_wall=1.0)
    assert dks == pytest.approx(fd["dD_dks"], rel=1e-6)
    assert duw == pytest.approx(fd["dD_duw"], rel=1e-6)
    dirs = FD.directions(len(X0), ndir, fd["directions_seed"])
    for d, ref in zip(dirs, fd["dD_dX0_along"]):
        _, dx = _tangent(c, cap, X0, tri, dX0=d)
        assert abs(dx - ref) <= 1e-6 * abs(ref) + 1e-12, (dx, ref)


def test_linear_in_the_direction():
    c, cap, X0, tri, _ = _small()
    d1, d2 = FD.directions(len(X0), 2, seed=7)
    a = _tangent(c, cap, X0, tri, steps=30, dX0=d1)[1]
    b = _tangent(c, cap, X0, tri, steps=30, dX0=d2)[1]
    ab = _tangent(c, cap, X0, tri, steps=30, dX0=d1 + 2.0 * d2)[1]
    assert abs(ab - (a + 2.0 * b)) <= 1e-11 * (abs(a) + 2.0 * abs(b))


def test_no_deformation_no_derivative():
    """Walls at rest: the fluid stays at rest, the capsule is never deformed,
    so D (zero up to the icosphere's rounding) has no derivative with respect
    to k_s."""
    c, cap, X0, tri, _ = _small()
    D, dks0 = O.tangent_taylor_D(c.shape, c.tau, c.delta, 0.0, X0, tri, cap.k_s, cap.C, 30, dks=1.0)
    assert abs(D) < 1e-12 and abs(dks0) < 1e-9


@pytest.mark.parametrize("name", ["small", "config5"])
def test_stored_tangents_agree_with_stored_differences(name):
    """The committed reference gradients (complex step) and the committed
    central differences, both from the oracle, agree to the differences' error
    (1e-6 relative; 1e-6 of the largest for the X0 directions)."""
    with open(os.path.join(GOLDEN, f"adjoint_fd_{name}.json")) as fh:
        fd = json.load(fh)
    with open(os.path.join(GOLDEN, f"adjoint_tangent_{name}.json")) as fh:
        tg = json.load(fh)
    assert tg["D"] == pytest.approx(fd["D"], rel=1e-12)
    assert tg["dD_dks"] == pytest.approx(fd["dD_dks"], rel=1e-6)
    assert tg["dD_duw"] == pytest.approx(fd["dD_duw"], rel=1e-6)
    scale = max(abs(v) for v in fd["dD_dX0_along"])
    for a, b in zip(tg["dD_dX0_along"], fd["dD_dX0_along"]):
        assert abs(a - b) <= 1e-6 * scale
