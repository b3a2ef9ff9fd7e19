"""Tiny cases run on the bounds-checked build of the library (the process is
started with IBLBM_LIBRARY=checked, so the binding loads
lib/libiblbm_checked.so): every kernel path of a time step on lattices of
4..16 cells per side, each compared with the FP64 oracle and its fault count
read.  Run by tests/test_gpu_bounds_checked.py as
``python bounds_cases.py`` from the tests folder; prints one JSON line per case
({"case", "faults", "err", "tol"}) and exits 0."""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import oracle as O  # noqa: E402
from cases import gpu_sim, oracle_sim, rel_inf  # noqa: E402
from paper_1004_2416_gb300 import Sim  # noqa: E402
from paper_1004_2416_gb300 import iblbm as B  # noqa: E402
from paper_1004_2416_gb300 import workloads as W  # noqa: E402

TOL = {"fp64": 1e-10, "fp32": 1e-4, "fp16": 5e-3}


def emit(name, faults, err, tol):
    print(json.dumps({"case": name, "faults": int(faults), "err": float(err), "tol": tol}), flush=True)


def lattice_only():
    for shape in ((4, 4, 4), (8, 6, 5), (6, 5, 4), (5, 7, 6), (16, 4, 4)):
        for prec in ("fp64", "fp32", "fp16"):
            nx, ny, nz = shape
            uw = 0.02
            f0 = O.init_couette(nx, ny, nz, uw) + W.population_noise(shape, 2e-3, seed=5)
            s = Sim(nx, ny, nz, tau=0.9, precision=prec, delta_points=3)
            s.set_shear_walls(uw)
            s.set_populations(f0)
            s.step(10)
            f = f0
            for _ in range(10):
                f = O.lbm_step(f, 0.9, uw)
            _, w, _ = O.d3q19()
            wb = w[:, None, None, None]
            err = rel_inf(s.get_populations() - wb, f - wb)
            emit(f"lattice {shape} {prec}", s.bounds_faults(), err, TOL[prec])
            s.close()


def capsule(shape, caps, prec, delta, steps, name, det=False, staging=None, record=False):
    case = W.Case(name, shape, 1.0, delta, prec, 0.01, caps, steps)
    g = gpu_sim(case)
    if det:
        g.set_deterministic_spreading(True)
    if staging is not None:
        g.set_collide_staging(staging)
    if record:
        g.set_taylor_recording(1, 16)
    o = oracle_sim(case)
    g.step(steps)
    o.step(steps)
    r = min(c.radius for c in caps)
    err = max(np.abs(g.get_nodes() - o.get_nodes()).max() / r, rel_inf(g.get_velocity(), o.get_velocity()))
    emit(f"{name} {prec} phi{delta}", g.bounds_faults(), err, TOL[prec])
    g.close()
    o.close()


def batch():
    runs = [((8, 8, 8), (3.6, 3.4, 3.7)), ((6, 4, 6), (2.6, 1.7, 2.4))]
    b = Sim.batch([(*sh, 1.0, 0.01) for sh, _ in runs], precision="fp32", delta_points=2)
    cases = []
    for k, (sh, c) in enumerate(runs):
        cap = W.Capsule(c, 1.2, 1, 0.05)
        cid = b.add_capsule_icosphere_in_run(k, cap.center, cap.radius, cap.subdivisions)
        b.set_skalak(cap.k_s, cap.C, cid)
        cases.append(W.Case(f"run{k}", sh, 1.0, 2, "fp32", 0.01, [cap], 5))
    b.init_fluid(1)
    b.step(5)
    err = 0.0
    for k, c in enumerate(cases):
        o = oracle_sim(c)
        o.step(5)
        err = max(err, rel_inf(b.get_run_velocity(k), o.get_velocity()),
                  np.abs(b.get_nodes(k) - o.get_nodes()).max() / 1.2)
        o.close()
    emit("batch fp32", b.bounds_faults(), err, TOL["fp32"])
    b.close()


def slabs():
    cap = W.Capsule((7.7, 4.1, 4.2), 1.5, 1, 0.05)
    case = W.Case("slabs", (16, 8, 9), 1.0, 3, "fp64", 0.01, [cap], 6)
    g = Sim.slabs(16, 8, 9, 2, tau=1.0, precision="fp64", delta_points=3)
    g.set_shear_walls(case.u_wall)
    cid = g.add_capsule_icosphere(cap.center, cap.radius, cap.subdivisions)
    g.set_skalak(cap.k_s, cap.C, cid)
    g.init_fluid(1)
    g.step(6)
    o = oracle_sim(case)
    o.step(6)
    err = max(np.abs(g.get_nodes() - o.get_nodes()).max() / 1.5, rel_inf(g.get_velocity(), o.get_velocity()))
    emit("slabs fp64", g.bounds_faults(), err, TOL["fp64"])
    g.close()
    o.close()


def main():
    assert B.iblbm_bounds_checked() == 1, "not the bounds-checked build"
    lattice_only()
    small = [W.Capsule((3.6, 3.4, 3.7), 1.5, 1, 0.05)]
    for prec in ("fp64", "fp32"):
        for delta in (2, 3, 4):
            capsule((8, 8, 8), small, prec, delta, 5, "capsule8", record=True)
    capsule((8, 8, 8), small, "fp16", 3, 5, "capsule8")
    capsule((8, 8, 8), small, "fp32", 3, 5, "capsule8-deterministic", det=True)
    capsule((8, 8, 8), small, "fp32", 3, 5, "capsule8-staged", staging=1)
    capsule((7, 6, 8), small, "fp32", 3, 5, "capsule-odd")
    # two overlapping 2 562-node capsules on 16^3: the four-nodes-per-warp
    # membrane kernels and the per-cell velocity pass
    dense = [W.Capsule((7.7, 8.2, 8.1), 4.0, 4, 0.05), W.Capsule((8.3, 7.9, 8.4), 4.0, 4, 0.05)]
    capsule((16, 16, 16), dense, "fp32", 3, 3, "dense16")
    batch()
    slabs()


if __name__ == "__main__":
    main()
