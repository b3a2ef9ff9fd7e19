"""The coupled-convergence study of Sec. IV.C (Tab. convergence) on the GPU
library: for H = 35, 70, 140 and the 2-, 3- and 4-point stencils, one capsule
in simple shear run to kappa t = 120, and the relative deviations of the
Taylor deformation and of the opposite inclination angle from the
small-deformation results D_a = 25/4 G and theta_a^o / pi = 15/8 G (Sec. III).

    python -m paper_1004_2416_gb300.convergence [--H 35 70 140] [--delta 2 3 4] [--precision fp32]

prints one JSON line per case.
"""
from __future__ import annotations

import argparse
import json
import math
import time

from . import workloads as W
from .iblbm import Sim


def run_case(case: W.Case, stream=None) -> dict:
    nx, ny, nz = case.shape
    c = case.capsules[0]
    G = 0.01
    sim = Sim(nx, ny, nz, tau=case.tau, precision=case.precision, delta_points=case.delta, stream=stream)
    try:
        sim.set_shear_walls(case.u_wall)
        cid = sim.add_capsule_icosphere(c.center, c.radius, c.subdivisions)
        sim.set_skalak(c.k_s, c.C, cid)
        sim.init_fluid(1)
        t0 = time.perf_counter()
        sim.step(case.steps)
        sim.sync()
        dt = time.perf_counter() - t0
        T = sim.taylor(cid)
        q = sim.mesh_quality(cid)
    finally:
        sim.close()
    D_a = 25.0 / 4.0 * G
    th_o_a = 15.0 / 8.0 * G * math.pi
    th_o = math.pi / 4.0 - T["theta"]
    return {"case": case.name, "H": nx, "faces": 20 * 4 ** c.subdivisions, "delta_points": case.delta,
            "steps": case.steps, "D": T["D"], "dD": (T["D"] - D_a) / D_a, "theta": T["theta"],
            "dtheta_o": (th_o - th_o_a) / th_o_a, "volume_drift": q["dV"], "face_area_dev_std": q["dA_std"],
            "seconds": dt, "MLUPS": nx * ny * nz * case.steps / dt / 1e6}


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--H", type=int, nargs="+", default=[35, 70, 140])
    p.add_argument("--delta", type=int, nargs="+", default=[2, 3, 4])
    p.add_argument("--precision", default="fp32")
    a = p.parse_args(argv)
    for H in a.H:
        for d in a.delta:
            print(json.dumps(run_case(W.convergence_case(H, d, a.precision))), flush=True)


if __name__ == "__main__":
    main()
