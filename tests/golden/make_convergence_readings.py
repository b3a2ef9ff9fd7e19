"""Writes tests/golden/convergence_readings_h35.txt: the FP64 oracle on the
smallest case of the coupled-convergence series of Sec. IV.C (H = 35, 1 280
faces, Re = 0.02, G = 0.01, tau = 1; Tab. convergence), under the readings of
the paper that its text leaves open, at kappa t = 120:

  couette   the library's readings (linear Couette start, walls half-way
            outside the nz = H fluid layers)
  rest      the fluid starts at rest (the paper gives no initial state)
  nz34/36   one fluid layer fewer / more between the walls at the same shear
            rate (the paper's "H^3 fluid nodes" fixes H = nz; the other wall
            placements are the nearest alternatives)

Columns: stencil reading dD dtheta_o dV/V0 (deviations from D_a = 25/4 G and
theta_a^o / pi = 15/8 G as fractions, relative volume change).  The spread of
the first two over the readings bounds how closely the oracle can be expected
to reproduce the paper's printed deviations.  Calls only the oracle (and the
seeded workload description).  About four minutes on 8 cores:
    python tests/golden/make_convergence_readings.py
"""
import concurrent.futures as cf
import math
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

G, H = 0.01, 35
READINGS = ("couette", "rest", "nz34", "nz36")


def run(arg):
    """(dD, dtheta_o, dV/V0) of one stencil under one reading."""
    delta, reading = arg
    import numpy as np

    import oracle as O
    from paper_1004_2416_gb300 import workloads as W

    O.set_threads(2)
    case = W.convergence_case(H, delta)
    cap = case.capsules[0]
    gdot = 2.0 * case.u_wall / H
    nz = {"nz34": 34, "nz36": 36}.get(reading, H)
    center = (cap.center[0], cap.center[1], (nz - 1) / 2.0)
    X0, tri = O.icosphere(cap.subdivisions, cap.radius, center)
    V0 = O.taylor(X0, tri)["V"]
    o = O.Sim(H, H, nz, case.tau, case.delta, gdot * nz / 2.0)
    o.add_capsule(X0, tri, cap.k_s, cap.C * cap.k_s)
    if reading == "rest":
        _, w, _ = O.d3q19()
        o.set_f(np.ascontiguousarray(np.broadcast_to(w[:, None, None, None], (19, nz, H, H))))
    o.step(case.steps)
    T = o.taylor(0)
    o.close()
    Da = 25.0 / 4.0 * G
    tho_a = 15.0 / 8.0 * G * math.pi
    return delta, reading, (T["D"] - Da) / Da, (math.pi / 4.0 - T["theta"] - tho_a) / tho_a, T["V"] / V0 - 1.0


def main():
    import oracle as O

    O.build()
    args = [(d, r) for r in READINGS for d in (2, 3, 4)]
    workers = max(1, min(len(args), (os.cpu_count() or 2) // 2))
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(run, args))
    out = os.path.join(HERE, "convergence_readings_h35.txt")
    with open(out, "w") as fh:
        fh.write("# FP64 oracle, smallest case of Tab. convergence (H = 35, 1 280 faces, Re = 0.02,\n"
                 "# G = 0.01, tau = 1) at kappa t = 120 under the readings the paper leaves open:\n"
                 "# couette (the library's), rest (fluid starts at rest), nz34 / nz36 (one fluid\n"
                 "# layer fewer / more between the walls, same shear rate).\n"
                 "# Written by tests/golden/make_convergence_readings.py (calls only the oracle).\n"
                 "# Columns: stencil reading dD dtheta_o dV/V0\n")
        for d, r, dD, dth, dV in sorted(res, key=lambda t: (t[0], READINGS.index(t[1]))):
            fh.write(f"{d} {r} {dD:.6f} {dth:.6f} {dV:.6e}\n")
    print("wrote", out)


if __name__ == "__main__":
    main()
