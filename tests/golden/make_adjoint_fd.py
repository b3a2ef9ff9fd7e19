"""Writes tests/golden/adjoint_fd_<case>.json: central finite differences of the
final Taylor deformation D of the FP64 oracle with respect to the shear
modulus k_s (at fixed C = k_alpha/k_s), the wall speed u_wall and the capsule's
reference (= initial) node positions along a few seeded unit directions.

Only the oracle and the seeded workload description are used.  Each
perturbed run is independent; they run in parallel processes.

    python tests/golden/make_adjoint_fd.py small     # seconds
    python tests/golden/make_adjoint_fd.py config5   # minutes (64^3, 2000 steps)
"""
import json
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def case(name):
    from paper_1004_2416_gb300 import workloads as W

    if name == "config5":
        return W.config5(), 4, 1e-5
    c = W.Capsule((11.3, 9.6, 10.4), 3.0, 2, W.k_s_for(0.05, 3.0))
    return W.Case("adjoint-small-24x20x22-r3-320f-phi3", (24, 20, 22), 1.0, 3, "fp64",
                  W.u_wall_for(22), [c], 150), 3, 1e-5


def directions(n_nodes, k, seed=51):
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((k, n_nodes, 3))
    return d / np.linalg.norm(d.reshape(k, -1), axis=1)[:, None, None]


def run_D(args):
    name, ks, uw, dX = args
    import oracle as O

    c, _, _ = case(name)
    cap = c.capsules[0]
    nx, ny, nz = c.shape
    o = O.Sim(nx, ny, nz, c.tau, c.delta, uw)
    X0, tri = O.icosphere(cap.subdivisions, cap.radius, cap.center)
    if dX is not None:
        X0 = X0 + dX
    o.add_capsule(X0, tri, ks, cap.C * ks)
    o.step(c.steps)
    return o.taylor(0)["D"]


def main(name):
    c, ndir, rel = case(name)
    cap = c.capsules[0]
    n_nodes = 10 * 4 ** cap.subdivisions + 2
    ks, uw = cap.k_s, c.u_wall
    hk, hu, hx = rel * ks, rel * uw, 1e-5
    dirs = directions(n_nodes, ndir)
    jobs = [(name, ks, uw, None), (name, ks + hk, uw, None), (name, ks - hk, uw, None),
            (name, ks, uw + hu, None), (name, ks, uw - hu, None)]
    for d in dirs:
        jobs += [(name, ks, uw, hx * d), (name, ks, uw, -hx * d)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
        D = pool.map(run_D, jobs)
    out = {
        "case": c.name, "steps": c.steps, "k_s": ks, "u_wall": uw, "D": D[0],
        "dD_dks": (D[1] - D[2]) / (2 * hk), "dD_duw": (D[3] - D[4]) / (2 * hu),
        "directions_seed": 51, "n_directions": ndir, "h_x": hx,
        "dD_dX0_along": [(D[5 + 2 * k] - D[6 + 2 * k]) / (2 * hx) for k in range(ndir)],
        "method": "central differences of the FP64 oracle; X0 moves both the reference and the "
                  "initial shape of the capsule",
    }
    path = os.path.join(HERE, f"adjoint_fd_{name}.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(path, out)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "small")
