"""x-slab decomposition across processes: each of two (or three) processes
holds one slab of the lattice on the GPU and advances it with the slab phases
of the C ABI, exchanging the boundary columns and the partial node
velocities over the host (gloo; paper_1004_2416_gb300.slabs).  The slabs'
populations, assembled along x, and the nodes equal those of the
single-process slab group (iblbm_create_slabs) to the rounding of the
spreading's atomic additions (whose order varies between runs: 1e-12 in the
FP64 build, 1e-5 in FP32), and match the oracle of the undivided lattice
(1e-10, 1e-4).  The processes share the one GPU; no kernel waits on another
process (every exchange is on the host)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

from conftest import ROOT

pytestmark = pytest.mark.gpu

STEPS = 30


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case(prec):
    sys.path.insert(0, ROOT)
    from paper_1004_2416_gb300 import workloads as W

    c = W.Capsule((17.7, 17.7, 13.6), 5.0, 3, W.k_s_for(0.05, 5.0))
    return W.Case("slab-ranks", (36, 36, 28), 1.0, 3, prec, 0.02, [c], STEPS)


def _rank_main(rank, ws, port, prec, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    from paper_1004_2416_gb300 import Sim
    from paper_1004_2416_gb300 import slabs as SL

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        torch.cuda.set_device(0)
        case = _case(prec)
        nx, ny, nz = case.shape
        x0, w = SL.slab_bounds(nx, ws, rank)
        s = Sim(w, ny, nz, tau=case.tau, precision=prec, delta_points=case.delta)
        s.slab_configure(x0, nx)
        s.set_shear_walls(case.u_wall)
        for c in case.capsules:
            cid = s.add_capsule_icosphere(c.center, c.radius, c.subdivisions)
            s.set_skalak(c.k_s, c.C, cid)
        s.init_fluid(1)
        SL.step(s, dist, STEPS)
        s.sync()
        q.put((rank, x0, s.get_populations(), s.get_nodes()))
        s.close()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("ws", [2, 3])
def test_ranks_equal_single_process_group(prec, ws):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, prec, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=600) for _ in range(ws)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    from paper_1004_2416_gb300 import Sim

    case = _case(prec)
    nx, ny, nz = case.shape
    g = Sim.slabs(nx, ny, nz, ws, tau=case.tau, precision=prec, delta_points=case.delta)
    g.set_shear_walls(case.u_wall)
    for c in case.capsules:
        cid = g.add_capsule_icosphere(c.center, c.radius, c.subdivisions)
        g.set_skalak(c.k_s, c.C, cid)
    g.init_fluid(1)
    g.step(STEPS)
    f = g.get_populations()
    import oracle as O
    from cases import oracle_sim, rel_inf

    o = oracle_sim(case)
    o.step(STEPS)
    fo = o.get_f()
    _, w, _ = O.d3q19()
    wb = w[:, None, None, None]
    tol_g = 1e-12 if prec == "fp64" else 1e-5
    tol_o = 1e-10 if prec == "fp64" else 1e-4
    r = case.capsules[0].radius
    for rank, x0, fr, xr in res:
        sl = (..., slice(x0, x0 + fr.shape[-1]))
        assert rel_inf(fr - wb, f[sl] - wb) < tol_g, rank
        assert rel_inf(fr - wb, fo[sl] - wb) < tol_o, rank
        assert np.abs(xr - g.get_nodes()).max() / r < tol_g, rank
        assert np.abs(xr - o.get_nodes()).max() / r < tol_o, rank
    # every rank holds the same copy of the nodes, bit for bit (the partials
    # are summed in rank order on every rank)
    assert all(np.array_equal(res[0][3], xr) for _, _, _, xr in res)
    g.close()
