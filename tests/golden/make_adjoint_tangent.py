"""Writes tests/golden/adjoint_tangent_<case>.json: directional derivatives of
the final Taylor deformation D of the oracle by the complex-step method
(oracle.tangent_taylor_D: the whole coupled step evaluated in complex
arithmetic, derivative = Im D / h with h = 1e-30), with respect to the shear
modulus k_s (at fixed C = k_alpha/k_s), the wall speed u_wall (including the
Couette start's dependence on it) and the capsule's reference (= initial) node
positions along the seeded unit directions of make_adjoint_fd.py.

Unlike the central differences of make_adjoint_fd.py these carry no
truncation error and no cancellation: they are the oracle's own reference
gradient.  Only the oracle and the seeded workload description are used; the
runs are independent and go to parallel processes.

    python tests/golden/make_adjoint_tangent.py small     # seconds
    python tests/golden/make_adjoint_tangent.py config5   # about ten minutes on 8 cores
"""
import json
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)

import make_adjoint_fd as FD  # noqa: E402  (the cases and the seeded directions)


def run(args):
    name, kind, k, threads = args
    import oracle as O

    c, ndir, _ = FD.case(name)
    cap = c.capsules[0]
    X0, tri = O.icosphere(cap.subdivisions, cap.radius, cap.center)
    kw = {}
    if kind == "ks":
        kw["dks"] = 1.0
    elif kind == "uw":
        kw["du_wall"] = 1.0
    else:
        kw["dX0"] = FD.directions(len(X0), ndir)[k]
    return kind, k, O.tangent_taylor_D(c.shape, c.tau, c.delta, c.u_wall, X0, tri, cap.k_s, cap.C, c.steps,
                                       threads=threads, **kw)


def main(name):
    import oracle as O

    O.build()
    c, ndir, _ = FD.case(name)
    jobs = [("ks", 0), ("uw", 0)] + [("x", k) for k in range(ndir)]
    procs = min(len(jobs), os.cpu_count() or 1)
    threads = max(1, (os.cpu_count() or 1) // procs)
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(run, [(name, kind, k, threads) for kind, k in jobs])
    D = res[0][2][0]
    assert all(r[2][0] == D for r in res)  # every run is the same real trajectory
    out = {"case": c.name, "steps": c.steps, "k_s": c.capsules[0].k_s, "u_wall": c.u_wall, "D": D,
           "dD_dks": res[0][2][1], "dD_duw": res[1][2][1], "directions_seed": 51, "n_directions": ndir,
           "dD_dX0_along": [r[2][1] for r in res[2:]], "h": 1e-30,
           "method": "complex-step derivative of the FP64 oracle (every sub-step of Sec. II.C and the "
                     "reductions of Sec. III in complex arithmetic); X0 moves both the reference and the "
                     "initial shape of the capsule"}
    path = os.path.join(HERE, f"adjoint_tangent_{name}.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(path, out)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "small")
