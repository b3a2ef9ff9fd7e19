"""The oracle's thread count changes no result, and oracle-side processes never
map the product library.

The oracle runs its whole-lattice loops (collide-and-stream of Eq. lbequation
and the velocity field of Eq. lbmmomenta1) on several threads when asked;
each output element is written by exactly one cell, and the spreading, the
membrane forces and every reduction stay serial in their fixed order, so a
coupled run is bit-identical for every thread count.  The input generators
(``workloads``), the golden-value writers and the CPU arm of the bench import
without loading ``libiblbm.so``.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle as O
from paper_1004_2416_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(threads, integrator=0, order=2):
    O.set_threads(threads)
    try:
        c = W.Capsule((19.2, 17.7, 13.6), 5.0, 3, W.k_s_for(0.05, 5.0))
        o = O.Sim(40, 36, 28, 1.0, 3, 0.02)
        X0, tri = O.icosphere(3, 5.0, c.center)
        o.add_capsule(X0, tri, c.k_s, c.k_s)
        o.set_integrator(integrator)
        o.set_equilibrium(order)
        o.step(6)
        out = (o.get_f(), o.get_nodes(), o.get_velocity(), o.get_force_field(), o.get_density())
        o.close()
        return out
    finally:
        O.set_threads(1)


@pytest.mark.parametrize("integrator,order", [(0, 2), (1, 1)])
def test_thread_count_bit_identical(integrator, order):
    ref = _run(1, integrator, order)
    for th in (3, 8):
        got = _run(th, integrator, order)
        for a, b in zip(ref, got):
            assert np.array_equal(a, b)
    assert O.get_threads() == 1


def test_lbm_step_threads_bit_identical():
    f0 = O.init_couette(23, 9, 11, 0.03) + W.population_noise((23, 9, 11), 2e-3, seed=3)
    force = W.population_noise((23, 9, 11), 1e-4, seed=4)[:3]
    O.set_threads(1)
    a = O.lbm_step(f0, 0.8, 0.03, force)
    O.set_threads(5)
    try:
        b = O.lbm_step(f0, 0.8, 0.03, force)
    finally:
        O.set_threads(1)
    assert np.array_equal(a, b)


_PROBE = r"""
import sys, runpy
sys.path.insert(0, {root!r})
sys.argv = ["x"]
import oracle
oracle.build()
from paper_1004_2416_gb300 import workloads
import importlib.util
for name in ("make_adjoint_fd", "make_config2_reference"):
    spec = importlib.util.spec_from_file_location(name, {root!r} + "/tests/golden/" + name + ".py")
    spec.loader.exec_module(importlib.util.module_from_spec(spec))
spec = importlib.util.spec_from_file_location("bench", {root!r} + "/bench.py")
bench = importlib.util.module_from_spec(spec)
spec.loader.exec_module(bench)
class A: pass
a = A(); a.workload = "config1"; a.delta = 3; a.G = 0.0125; a.precision = None
case = bench._workload(a)
bench._oracle_run(case, 0.05, 1, None, threads=1)
maps = open("/proc/self/maps").read()
print("LIBIBLBM" if "libiblbm" in maps else "CLEAN", "LIBORACLE" if "liboracle" in maps else "")
"""


@pytest.mark.skipif(not os.path.exists("/proc/self/maps"), reason="needs /proc/self/maps")
def test_oracle_side_imports_do_not_map_the_product_library():
    out = subprocess.run([sys.executable, "-c", _PROBE.format(root=ROOT)], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    assert "CLEAN LIBORACLE" in out.stdout, out.stdout
