"""Builds the GPU simulation (through the C ABI) and the FP64 oracle from the
same workload description and seeded inputs."""
import numpy as np

import oracle as O
from paper_1004_2416_gb300 import workloads as W


def gpu_sim(case: W.Case, precision=None):
    from paper_1004_2416_gb300 import Sim

    nx, ny, nz = case.shape
    s = Sim(nx, ny, nz, tau=case.tau, precision=precision or case.precision, delta_points=case.delta)
    s.set_shear_walls(case.u_wall)
    for c in case.capsules:
        cid = s.add_capsule_icosphere(c.center, c.radius, c.subdivisions)
        s.set_skalak(c.k_s, c.C, cid)
    s.init_fluid(1)
    return s


def oracle_sim(case: W.Case):
    nx, ny, nz = case.shape
    o = O.Sim(nx, ny, nz, case.tau, case.delta, case.u_wall)
    for c in case.capsules:
        X0, tri = O.icosphere(c.subdivisions, c.radius, c.center)
        o.add_capsule(X0, tri, c.k_s, c.C * c.k_s)
    return o


def rel_inf(a, b):
    """||a - b||_inf / ||b||_inf."""
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
