"""Device memory from the caller's allocator (iblbm_allocator of
iblbm_create): PyTorch's caching allocator gives the library's own results
and gets every block back at destruction; an allocator that refuses after a
given number of blocks makes the failing call return IBLBM_ERR_OOM, with no
block leaked or freed twice, and the same calls repeated once memory is
available again continue the run as if nothing had failed (node positions
kept across a failed rebuild of the membrane tables)."""
import ctypes

import numpy as np
import pytest

from cases import gpu_sim, rel_inf
from paper_1004_2416_gb300 import iblbm as B
from paper_1004_2416_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CAPS = [W.Capsule((17.3, 17.6, 13.4), 5.0, 3, W.k_s_for(0.05, 5.0)),
        W.Capsule((30.1, 18.2, 14.9), 4.0, 2, W.k_s_for(0.02, 4.0))]
SHAPE = (48, 36, 28)


class CountingAllocator:
    """Blocks from PyTorch, at most `budget` of them (None: unlimited);
    counts what it hands out and what comes back."""

    def __init__(self, budget=None):
        import torch

        self.torch = torch
        self.budget = budget
        self.live = {}
        self.given = 0
        self.returned = 0
        self.double_frees = 0
        self.refused = 0
        self.c = B.iblbm_allocator(B.ALLOC_FN(self._alloc), B.FREE_FN(self._free), None)

    def _alloc(self, nbytes, stream, ctx):
        if self.budget is not None and self.given >= self.budget:
            self.refused += 1
            return None
        t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device="cuda")
        self.live[t.data_ptr()] = t
        self.given += 1
        return t.data_ptr()

    def _free(self, ptr, stream, ctx):
        if ptr not in self.live:
            self.double_frees += 1
            return
        del self.live[ptr]
        self.returned += 1


def _scenario(sim_factory, alloc):
    """create; a capsule; 7 steps with records; a second capsule (the membrane
    tables are rebuilt around the moved nodes of the first); 9 more steps;
    read-back.  A call that fails with OOM is repeated once the allocator
    gives blocks again."""
    failures = []
    box = {}

    def run(call):
        try:
            return call()
        except B.IblbmError as e:
            assert e.code == B.IBLBM_ERR_OOM, str(e)
            failures.append(str(e))
            alloc.budget = None
            return call()

    box["s"] = run(sim_factory)
    s = box["s"]
    for k, cap in enumerate(CAPS):
        cid = run(lambda: s.add_capsule_icosphere(cap.center, cap.radius, cap.subdivisions))
        run(lambda: s.set_skalak(cap.k_s, cap.C, cid))
        if k == 0:
            run(lambda: s.set_shear_walls(0.02))
            run(lambda: s.init_fluid(1))
            run(lambda: s.set_taylor_recording(1, 32))
        run(lambda: s.step(7 if k == 0 else 9))
    out = (run(s.get_nodes), run(s.get_velocity), run(lambda: s.taylor(0))["D"])
    s.close()
    return out, failures


def _factory(alloc):
    from paper_1004_2416_gb300 import Sim

    return lambda: Sim(*SHAPE, tau=1.0, precision="fp32", delta_points=3, allocator=alloc.c)


def test_torch_allocator_same_results():
    from paper_1004_2416_gb300 import Sim

    case = W.Case("alloc", SHAPE, 1.0, 3, "fp32", 0.02, CAPS[:1], 30)
    ref = gpu_sim(case)
    ref.step(30)
    s = Sim(*SHAPE, tau=1.0, precision="fp32", delta_points=3, allocator="torch")
    cid = s.add_capsule_icosphere(CAPS[0].center, CAPS[0].radius, CAPS[0].subdivisions)
    s.set_skalak(CAPS[0].k_s, CAPS[0].C, cid)
    s.set_shear_walls(case.u_wall)
    s.init_fluid(1)
    s.step(30)
    live = s._keep[1]
    assert len(live) > 0  # the library's buffers are PyTorch tensors
    assert np.abs(s.get_nodes() - ref.get_nodes()).max() < 1e-5
    assert rel_inf(s.get_velocity(), ref.get_velocity()) < 1e-5
    s.close()
    assert len(live) == 0  # every block came back
    ref.close()


def test_refusing_allocator_every_point_of_failure():
    full = CountingAllocator()
    ref, failures = _scenario(_factory(full), full)
    assert not failures and full.double_frees == 0 and full.given == full.returned
    total = full.given
    assert total >= 10
    for budget in range(total):
        a = CountingAllocator(budget)
        out, failures = _scenario(_factory(a), a)
        assert a.refused > 0 and failures, budget
        assert a.double_frees == 0, budget
        assert a.given == a.returned and not a.live, budget  # nothing leaked
        assert np.abs(out[0] - ref[0]).max() < 1e-5, budget
        assert rel_inf(out[1], ref[1]) < 1e-5, budget
        assert abs(out[2] - ref[2]) <= 1e-5 * abs(ref[2]) + 1e-9, budget
