"""The host-staged exchange of an x-slab decomposition across processes
(paper_1004_2416_gb300.slabs), on gloo ranks on the CPU: every rank receives
exactly its left ring neighbour's boundary columns (for its c_x = +1
populations) and its right neighbour's (for c_x = -1), and the partial node
velocities of all ranks in rank order, whatever the number of ranks; the slab
bounds are those of iblbm_create_slabs."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

from conftest import ROOT


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _cols(rank):
    return np.random.default_rng(100 + rank).integers(0, 256, 10 * 7 * 5 * 4, dtype=np.uint8)


def _part(rank):
    return np.random.default_rng(200 + rank).integers(0, 256, 33 * 16, dtype=np.uint8)


def _rank_main(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    from paper_1004_2416_gb300 import slabs as SL

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        left, right = SL.exchange_columns(_cols(rank), dist)
        parts = SL.gather_partials(_part(rank), dist)
        q.put((rank, np.array_equal(left, _cols((rank - 1) % ws)), np.array_equal(right, _cols((rank + 1) % ws)),
               np.array_equal(parts, np.concatenate([_part(r) for r in range(ws)]))))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2, 3])
def test_exchange_between_gloo_ranks(ws):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == list(range(ws))
    assert all(r[1] and r[2] and r[3] for r in res), res


def test_slab_bounds_cover_the_lattice():
    sys.path.insert(0, ROOT)
    from paper_1004_2416_gb300 import slabs as SL

    for nx, p in ((36, 2), (41, 3), (128, 5)):
        b = [SL.slab_bounds(nx, p, k) for k in range(p)]
        assert sum(w for _, w in b) == nx
        assert [x0 for x0, _ in b] == list(np.cumsum([0] + [w for _, w in b[:-1]]))
        assert max(w for _, w in b) - min(w for _, w in b) <= 1
