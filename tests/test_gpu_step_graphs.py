"""Step dispatch through captured graphs of any length (the sub-step list of
Sec. II.C, steps 1-6, replayed as CUDA graphs): one call of n steps, n calls
of one step, calls split at odd lengths after a prepare, and Taylor records
at every phase of their period all follow the oracle element by element
(FP64 build 1e-10, FP32 1e-4, as every trajectory test), and record the
reductions after the same steps as the oracle."""
import numpy as np
import pytest

from cases import gpu_sim, oracle_sim, rel_inf
from paper_1004_2416_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-4}
D_TOL = {"fp64": 1e-11, "fp32": 2e-6}  # absolute: D starts at round-off on the sphere
STEPS = 20


def _case(prec):
    c = W.Capsule((19.2, 17.7, 13.6), 5.0, 3, W.k_s_for(0.05, 5.0))
    return W.Case("graphs", (40, 36, 28), 1.0, 3, prec, 0.02, [c], STEPS)


@pytest.fixture(scope="module")
def oracle_run():
    """Oracle nodes, velocity and D after each of the STEPS steps."""
    case = _case("fp64")
    o = oracle_sim(case)
    D, xs = [], []
    for _ in range(STEPS):
        o.step(1)
        D.append(o.taylor(0)["D"])
        xs.append(o.get_nodes())
    out = {"D": np.array(D), "x": xs, "u": o.get_velocity()}
    o.close()
    return out


def _check(s, ref, prec, r=5.0):
    tol = TOL[prec]
    assert s.info().step == STEPS
    assert np.abs(s.get_nodes() - ref["x"][-1]).max() / r < tol
    assert rel_inf(s.get_velocity(), ref["u"]) < tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("split", [[20], [1] * 20, [5, 15], [3, 7, 1, 9], [13, 2, 5]])
def test_any_split_matches_oracle(prec, split, oracle_run):
    """Records every step; graphs of lengths 20, 1, 5, 15, 3, 7, 9, 13, 2 at
    both buffer parities.  A prepare before every call captures what the call
    replays."""
    s = gpu_sim(_case(prec))
    s.set_taylor_recording(1, ring=64)
    for n in split:
        s.prepare_steps(n)
        s.step(n)
    _check(s, oracle_run, prec)
    steps, rec = s.taylor_records(0)
    assert list(steps) == list(range(1, STEPS + 1))
    D = np.array([r[0] for r in rec])
    assert np.abs(D - oracle_run["D"]).max() < D_TOL[prec]
    s.close()


@pytest.mark.parametrize("every", [3, 7])
def test_record_phases(every, oracle_run):
    """A recording period that does not divide the call lengths: records after
    steps every, 2 every, ... whatever the split."""
    s = gpu_sim(_case("fp64"))
    s.set_taylor_recording(every, ring=64)
    for n in (2, 9, 4, 5):
        s.step(n)
    _check(s, oracle_run, "fp64")
    steps, rec = s.taylor_records(0)
    want = list(range(every, STEPS + 1, every))
    assert list(steps) == want
    D = np.array([r[0] for r in rec])
    assert np.abs(D - oracle_run["D"][np.array(want) - 1]).max() < D_TOL["fp64"]
    s.close()


def test_many_lengths_evict_graphs(oracle_run):
    """More distinct call lengths than graphs kept (16): preparing 20 lengths
    drops the least recently used; the calls then replay some graphs kept and
    recapture the others, with unchanged results."""
    s = gpu_sim(_case("fp64"))
    s.set_taylor_recording(1, ring=64)
    for n in range(1, STEPS + 1):
        s.prepare_steps(n)
    for n in (1, 2, 3, 4, 10):
        s.step(n)
    _check(s, oracle_run, "fp64")
    steps, _ = s.taylor_records(0)
    assert list(steps) == list(range(1, STEPS + 1))
    s.close()


def test_kernel_timing_graphs(oracle_run):
    """Event nodes around the kernel groups change no result; the times cover
    the steps of the last replay of each graph."""
    s = gpu_sim(_case("fp32"))
    s.set_taylor_recording(1, ring=64)
    s.set_kernel_timing(True)
    s.step(5)
    s.prepare_steps(15)
    t0 = s.kernel_times()
    assert t0["steps"] == 5
    s.step(15)
    t = s.kernel_times()
    assert t["steps"] == 15
    for k in ("force_spread", "collide_stream", "interp_advect"):
        assert 0.0 < t[k] < 50.0
    assert s.kernel_times()["steps"] == 0  # read once
    _check(s, oracle_run, "fp32")
    assert s.collide_kernel().startswith("k_collide_pair<float>")
    s.close()
