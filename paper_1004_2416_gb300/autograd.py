"""Differentiable Taylor deformation: a ``torch.autograd.Function`` over the
library's adjoint.

``taylor_deformation(k_s, u_wall, X0, setup)`` runs ``setup.steps`` time steps
of one capsule in simple shear (through the C ABI) and returns the Taylor
deformation D of its final shape (Sec. III).  ``backward`` calls the
library's reverse sweep (checkpoints every ``setup.checkpoint_every`` steps,
recomputation in between) and returns dD/dk_s at fixed C = k_alpha/k_s,
dD/du_wall and dD/dX0, where X0 is the capsule's reference shape, which is
also its initial shape.  All arithmetic runs in the CUDA library; this module
only moves arguments.

The reduced shear rate (capillary number) of Sec. III is
G = gdot eta r / k_s with gdot = 2 u_wall / nz, so at fixed k_s
dD/dG = dD/du_wall * k_s nz / (2 eta r): see :func:`dD_dG`.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from .iblbm import Sim


@dataclasses.dataclass
class ShearSetup:
    shape: tuple          # (nx, ny, nz)
    tri: np.ndarray       # faces [m, 3] of the capsule mesh
    steps: int
    checkpoint_every: int
    tau: float = 1.0
    C: float = 1.0        # k_alpha / k_s
    delta_points: int = 3
    precision: str = "fp32"


class TaylorDeformation(torch.autograd.Function):
    @staticmethod
    def forward(ctx, k_s, u_wall, X0, setup: ShearSetup):
        nx, ny, nz = setup.shape
        sim = Sim(nx, ny, nz, tau=setup.tau, precision=setup.precision, delta_points=setup.delta_points)
        sim.set_shear_walls(float(u_wall))
        cid = sim.add_capsule_mesh(X0.detach().cpu().double().numpy(), setup.tri)
        sim.set_skalak(float(k_s), setup.C, cid)
        sim.init_fluid(1)
        sim.adjoint_forward(setup.steps, setup.checkpoint_every)
        ctx.sim = sim
        ctx.dtypes = (k_s.dtype, u_wall.dtype, X0.dtype, X0.device)
        return torch.tensor(sim.taylor(cid)["D"], dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_D):
        r = ctx.sim.adjoint_backward(0)
        tk, tu, tx, dev = ctx.dtypes
        g = float(grad_D)
        gks = torch.tensor(g * r["dD_dks"], dtype=tk)
        guw = torch.tensor(g * r["dD_duw"], dtype=tu)
        gX0 = torch.from_numpy(g * (r["dD_dX0"] + r["dD_dx0"])).to(dtype=tx, device=dev)
        return gks, guw, gX0, None


def taylor_deformation(k_s, u_wall, X0, setup: ShearSetup):
    return TaylorDeformation.apply(k_s, u_wall, X0, setup)


def dD_dG(dD_duw: float, k_s: float, nz: int, radius: float, tau: float = 1.0) -> float:
    """dD/dG at fixed k_s from dD/du_wall (G = 2 u_wall eta r / (nz k_s))."""
    eta = (tau - 0.5) / 3.0
    return dD_duw * k_s * nz / (2.0 * eta * radius)
