"""Adjoint extension: the gradient of the final Taylor deformation with respect
to the shear modulus, the wall speed (capillary number) and the reference node
positions, from the hand-written reverse sweep, against central finite
differences of the FP64 oracle (tests/golden/adjoint_fd_*.json, written by
tests/golden/make_adjoint_fd.py) and against the oracle's own reference
gradient, its complex-step tangent (tests/golden/adjoint_tangent_*.json,
written by tests/golden/make_adjoint_tangent.py); both scripts call only the
oracle.  The tangent carries no truncation error, so the FP64 build is held to
it at 1e-8 (the rounding of two different evaluation orders over the run)."""
import importlib.util
import json
import os

import numpy as np
import pytest

from cases import gpu_sim
from conftest import GOLDEN

pytestmark = pytest.mark.gpu

_spec = importlib.util.spec_from_file_location("make_adjoint_fd", os.path.join(GOLDEN, "make_adjoint_fd.py"))
FDMOD = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(FDMOD)


def _fd(name):
    with open(os.path.join(GOLDEN, f"adjoint_fd_{name}.json")) as fh:
        return json.load(fh)


def _tangent(name):
    path = os.path.join(GOLDEN, f"adjoint_tangent_{name}.json")
    if not os.path.exists(path):
        pytest.skip(f"{path} not written")
    with open(path) as fh:
        return json.load(fh)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-8), ("fp32", 1e-3)])
def test_adjoint_small_against_oracle_tangent(prec, tol, capsys):
    case, _, _ = FDMOD.case("small")
    t = _tangent("small")
    g = gpu_sim(case, precision=prec)
    g.adjoint_forward(case.steps, 50)
    n = len(g.get_nodes())
    r = g.adjoint_backward(0)
    assert r["D"] == pytest.approx(t["D"], rel=1e-9 if prec == "fp64" else 1e-4)
    _check(r, t, n, tol, capsys, f"adjoint {prec} vs tangent")
    g.close()


def _check(r, fd, n_nodes, tol, capsys, label):
    dirs = FDMOD.directions(n_nodes, fd["n_directions"], fd["directions_seed"])
    gtot = r["dD_dX0"] + r["dD_dx0"]
    along = [float(np.sum(gtot * d)) for d in dirs]
    gnorm = float(np.linalg.norm(gtot))
    with capsys.disabled():
        print(f"\n{label}: D {r['D']:.8g} (fd {fd['D']:.8g}); dD/dks {r['dD_dks']:.8g} (fd {fd['dD_dks']:.8g}); "
              f"dD/duw {r['dD_duw']:.8g} (fd {fd['dD_duw']:.8g}); dD/dX0 along "
              f"{np.round(along, 8).tolist()} (fd {np.round(fd['dD_dX0_along'], 8).tolist()}), |grad| {gnorm:.4g}")
    assert r["dD_dks"] == pytest.approx(fd["dD_dks"], rel=tol)
    assert r["dD_duw"] == pytest.approx(fd["dD_duw"], rel=tol)
    for a, b in zip(along, fd["dD_dX0_along"]):
        assert abs(a - b) <= tol * gnorm


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_adjoint_small_against_oracle_fd(prec, capsys):
    case, _, _ = FDMOD.case("small")
    fd = _fd("small")
    g = gpu_sim(case, precision=prec)
    g.adjoint_forward(case.steps, 50)
    x_end = g.get_nodes()
    f_end = g.get_populations()
    r = g.adjoint_backward(0)
    assert r["D"] == pytest.approx(fd["D"], rel=1e-9 if prec == "fp64" else 1e-4)
    _check(r, fd, len(x_end), 1e-6 if prec == "fp64" else 1e-3, capsys, f"adjoint {prec}")
    # the simulation is left in its final state
    assert np.array_equal(g.get_nodes(), x_end)
    assert np.array_equal(g.get_populations(), f_end)
    # a second backward pass gives the same gradient
    r2 = g.adjoint_backward(0)
    assert r2["dD_dks"] == pytest.approx(r["dD_dks"], rel=1e-5)


def test_adjoint_requires_forward_run():
    from paper_1004_2416_gb300 import iblbm as B

    case, _, _ = FDMOD.case("small")
    g = gpu_sim(case, precision="fp32")
    with pytest.raises(B.IblbmError) as e:
        g.adjoint_backward(0)
    assert e.value.code == B.IBLBM_ERR_STATE
    g.adjoint_forward(10, 5)
    g.step(1)
    with pytest.raises(B.IblbmError) as e:
        g.adjoint_backward(0)
    assert e.value.code == B.IBLBM_ERR_STATE


def test_autograd_function_against_oracle_fd():
    """torch.autograd through TaylorDeformation: D.backward() gives the
    oracle's finite-difference gradients."""
    torch = pytest.importorskip("torch")
    import oracle as O
    from paper_1004_2416_gb300.autograd import ShearSetup, taylor_deformation

    case, _, _ = FDMOD.case("small")
    fd = _fd("small")
    cap = case.capsules[0]
    X0np, tri = O.icosphere(cap.subdivisions, cap.radius, cap.center)
    setup = ShearSetup(shape=case.shape, tri=tri, steps=case.steps, checkpoint_every=50,
                       precision="fp64", delta_points=case.delta)
    ks = torch.tensor(cap.k_s, dtype=torch.float64, requires_grad=True)
    uw = torch.tensor(case.u_wall, dtype=torch.float64, requires_grad=True)
    X0 = torch.tensor(X0np, dtype=torch.float64, requires_grad=True)
    D = taylor_deformation(ks, uw, X0, setup)
    D.backward()
    assert float(D.detach()) == pytest.approx(fd["D"], rel=1e-9)
    assert float(ks.grad) == pytest.approx(fd["dD_dks"], rel=1e-6)
    assert float(uw.grad) == pytest.approx(fd["dD_duw"], rel=1e-6)
    dirs = FDMOD.directions(len(X0np), fd["n_directions"], fd["directions_seed"])
    g = X0.grad.numpy()
    for d, b in zip(dirs, fd["dD_dX0_along"]):
        assert float(np.sum(g * d)) == pytest.approx(b, abs=1e-6 * np.linalg.norm(g))


def test_adjoint_config5_against_oracle_fd(capsys):
    """Config 5 as stated: 64^3, FP32, one 1280-face capsule of radius 8,
    G = 0.0125, phi3, 2000 steps, checkpoints every 100 steps; the gradient of
    the final D against FP64 central differences within 1e-3."""
    case, _, _ = FDMOD.case("config5")
    fd = _fd("config5")
    g = gpu_sim(case, precision="fp32")
    g.adjoint_forward(case.steps, 100)
    r = g.adjoint_backward(0)
    assert r["D"] == pytest.approx(fd["D"], rel=1e-4)
    _check(r, fd, len(r["dD_dX0"]), 1e-3, capsys, "adjoint config5 fp32")
    # and against the oracle's complex-step tangent along the same directions
    t = _tangent("config5")
    _check(r, t, len(r["dD_dX0"]), 1e-3, capsys, "adjoint config5 fp32 vs tangent")
    g.close()


def test_adjoint_taylor_one_call(capsys):
    """The one-call entry point: dD/dCa is dD/du_wall scaled by du_wall/dG at
    fixed k_s (G = (2 u_wall / nz) eta r / k_s), and dD/dX0 moves the reference
    and the initial shape together, as the finite differences do."""
    case, _, _ = FDMOD.case("small")
    fd = _fd("small")
    cap = case.capsules[0]
    g = gpu_sim(case, precision="fp64")
    r = g.adjoint_taylor(case.steps, 50)
    eta = (case.tau - 0.5) / 3.0
    fd_dCa = fd["dD_duw"] * case.shape[2] * cap.k_s / (2.0 * eta * cap.radius)
    with capsys.disabled():
        print(f"\nadjoint one call: dD/dCa {r['dD_dCa']:.8g} (fd {fd_dCa:.8g})")
    assert r["D"] == pytest.approx(fd["D"], rel=1e-9)
    assert r["dD_dks"] == pytest.approx(fd["dD_dks"], rel=1e-6)
    assert r["dD_dCa"] == pytest.approx(fd_dCa, rel=1e-6)
    dirs = FDMOD.directions(len(r["dD_dX0"]), fd["n_directions"], fd["directions_seed"])
    gnorm = float(np.linalg.norm(r["dD_dX0"]))
    for d, b in zip(dirs, fd["dD_dX0_along"]):
        assert abs(float(np.sum(r["dD_dX0"] * d)) - b) <= 1e-6 * gnorm
