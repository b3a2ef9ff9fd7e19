"""Precision extension: populations stored as FP16 (scaled) or FP32 deviations
from the rest equilibrium, arithmetic in FP32, against the FP64 oracle, on a
dense-suspension set-up shaped like config 4 (capsules of radius 6 on the
1280-face mesh, G = 0.02, 3-point delta, shear walls) but on a smaller
lattice so that the oracle finishes in seconds.  The measured errors are
printed; the asserted bounds are the stated ones."""
import numpy as np
import pytest

from cases import gpu_sim, oracle_sim, rel_inf
from paper_1004_2416_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# stated error bounds after 120 steps (relative, infinity norm)
BOUND = {"fp32": {"u": 1e-5, "x": 1e-6, "D": 1e-4}, "fp16": {"u": 2e-2, "x": 5e-4, "D": 5e-2}}


def _suspension_case(precision):
    shape = (128, 64, 64)
    r, G = 6.0, 0.02
    centres = W.rsa_centres(shape, 6, r, seed=4, z_margin=r + 4.0)
    caps = [W.Capsule(c, r, 3, W.k_s_for(G, r)) for c in centres]
    return W.Case("suspension-small", shape, 1.0, 3, precision, W.u_wall_for(shape[2]), caps, 120)


def test_storage_precision_errors_against_oracle(capsys):
    ref = _suspension_case("fp32")
    o = oracle_sim(ref)
    o.step(ref.steps)
    u_o, x_o = o.get_velocity(), o.get_nodes()
    D_o = np.array([o.taylor(k)["D"] for k in range(len(ref.capsules))])
    errs = {}
    for prec in ("fp32", "fp16"):
        case = _suspension_case(prec)
        g = gpu_sim(case)
        g.step(case.steps)
        D_g = np.array([g.taylor(k)["D"] for k in range(len(case.capsules))])
        errs[prec] = {"u": rel_inf(g.get_velocity(), u_o),
                      "x": float(np.abs(g.get_nodes() - x_o).max() / 6.0),
                      "D": float(np.abs(D_g - D_o).max() / np.abs(D_o).max())}
    with capsys.disabled():
        print(f"\nstorage precision errors vs FP64 oracle after {ref.steps} steps: {errs}")
    for prec, e in errs.items():
        for k, v in e.items():
            assert v < BOUND[prec][k], (prec, k, v)
    assert errs["fp16"]["u"] > errs["fp32"]["u"]  # the half storage is the coarser one
