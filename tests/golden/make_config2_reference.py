"""Writes tests/golden/config2_oracle_2000.npz (and, with --steps 20000
--every 500 --out tests/golden/config2_oracle_20000.npz, the workload's full
20 000 steps): the FP64 oracle's state after that many full-size steps of the
128^3 single-capsule shear flow (r = 16, 5 120 faces, 4-point delta, reduced
shear rate G = 0.0125, shear rate 1e-3, tau = 1, Couette start), the sub-step
list of Sec. II.C run on the host.

Calls only the oracle (and the seeded workload description, which holds none
of the method's arithmetic).  Stored:
  nodes      [2562, 3]   node positions after the last step
  u_slice    [3, 64, 64] lattice velocity u(X, t) of Eq. (lbmmomenta1) on the
                         plane y = 64, every second cell in z and x
                         ([3][z/2][x/2])
  D_steps    [n]         steps after which D was taken (every 100, or --every)
  D, theta   [n]         Taylor deformation and inclination of Sec. III
  steps, G, delta        the run's parameters

The oracle's whole-lattice loops run on all host cores (results do not depend
on the thread count).  About 12 minutes on 8 cores for 2 000 steps, 80 for
20 000.
    python tests/golden/make_config2_reference.py [--steps 2000] [--threads N]
"""
import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1004_2416_gb300 import workloads as W  # noqa: E402

Y_PLANE = 64


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--every", type=int, default=100)
    ap.add_argument("--threads", type=int, default=os.cpu_count())
    ap.add_argument("--out", default=os.path.join(HERE, "config2_oracle_2000.npz"))
    a = ap.parse_args()
    case = W.config2(G=0.0125, delta=4)
    O.set_threads(a.threads)
    o = O.Sim(*case.shape, case.tau, case.delta, case.u_wall)
    for c in case.capsules:
        X0, tri = O.icosphere(c.subdivisions, c.radius, c.center)
        o.add_capsule(X0, tri, c.k_s, c.C * c.k_s)
    D_steps, D, theta = [], [], []
    t0 = time.time()
    done = 0
    while done < a.steps:
        n = min(a.every, a.steps - done)
        o.step(n)
        done += n
        T = o.taylor(0)
        D_steps.append(done)
        D.append(T["D"])
        theta.append(T["theta"])
        print(f"step {done}: D {T['D']:.9f} theta {T['theta']:.6f} ({time.time() - t0:.0f} s)", flush=True)
    u = o.get_velocity()  # [3][nz][ny][nx]
    np.savez(a.out, nodes=o.get_nodes(), u_slice=np.ascontiguousarray(u[:, ::2, Y_PLANE, ::2]),
             D_steps=np.array(D_steps), D=np.array(D), theta=np.array(theta),
             steps=a.steps, G=0.0125, delta=case.delta)
    o.close()
    print("wrote", a.out)


if __name__ == "__main__":
    main()
