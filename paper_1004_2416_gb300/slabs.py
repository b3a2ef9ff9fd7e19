"""x-slab decomposition across processes, exchanging over the host.

Each process holds one slab of a periodic lattice (a :class:`Sim` of the
slab's width, ``slab_configure(x0, nx)``) and advances it with the slab phases
of the C ABI; between them the processes exchange, through a
``torch.distributed`` process group (gloo for host memory):

- the ten boundary columns of the populations with each ring neighbour: a
  slab's c_x = +1 columns come from its left neighbour, its c_x = -1 columns
  from its right one (10 ny nz populations per boundary and step, Eq.
  lbequation's streaming across the slab boundary);
- the partial node velocities of every slab, gathered in rank order and
  summed on every process in that order (Eq. velocityinterpolation over the
  whole lattice), so every copy of the replicated membranes moves alike.

With ranks in slab order this computes what ``Sim.slabs`` computes in one
process, bit for bit.
"""
from __future__ import annotations

import numpy as np


def slab_bounds(nx: int, n_slabs: int, k: int):
    """(first global column, width) of slab k: nx / n_slabs columns, one more
    for the first nx mod n_slabs slabs (as iblbm_create_slabs)."""
    w = [nx // n_slabs + (j < nx % n_slabs) for j in range(n_slabs)]
    return int(sum(w[:k])), int(w[k])


def exchange_columns(cols: np.ndarray, dist):
    """(left, right): the packed boundary columns of the left and right ring
    neighbours of this rank (its own for a single rank)."""
    import torch

    ws, rank = dist.get_world_size(), dist.get_rank()
    if ws == 1:
        return cols.copy(), cols.copy()
    left_rank, right_rank = (rank - 1) % ws, (rank + 1) % ws
    mine = torch.from_numpy(np.ascontiguousarray(cols))
    from_left = torch.empty_like(mine)
    from_right = torch.empty_like(mine)
    ops = [dist.P2POp(dist.isend, mine, right_rank), dist.P2POp(dist.isend, mine, left_rank),
           dist.P2POp(dist.irecv, from_left, left_rank), dist.P2POp(dist.irecv, from_right, right_rank)]
    if ws == 2:  # both neighbours are the same rank: one message each way carries both
        ops = [dist.P2POp(dist.isend, mine, right_rank), dist.P2POp(dist.irecv, from_left, left_rank)]
    for r in dist.batch_isend_irecv(ops):
        r.wait()
    if ws == 2:
        from_right = from_left
    return from_left.numpy(), from_right.numpy()


def gather_partials(part: np.ndarray, dist) -> np.ndarray:
    """Every rank's partial node velocities, concatenated in rank order."""
    import torch

    ws = dist.get_world_size()
    if ws == 1:
        return part.copy()
    mine = torch.from_numpy(np.ascontiguousarray(part))
    out = [torch.empty_like(mine) for _ in range(ws)]
    dist.all_gather(out, mine)
    return np.concatenate([t.numpy() for t in out])


def step(sim, dist, n_steps: int = 1):
    """n_steps of the slab held by this rank, exchanging with the others."""
    ws = dist.get_world_size()
    for _ in range(n_steps):
        sim.slab_step_begin()
        left, right = exchange_columns(sim.slab_columns(), dist)
        sim.slab_set_columns(left, right)
        sim.slab_step_end(gather_partials(sim.slab_partials(), dist), ws)
