"""Checkpoint and restart through the C ABI: a run continued from a restored
checkpoint matches the uninterrupted run (bit for bit without membranes,
where nothing depends on the order of atomic additions; to rounding of the
spreading's atomics with them), in every storage precision, with host and
device buffers, into the same object and into a fresh one; mismatched,
truncated or corrupt checkpoints (a byte flipped in a section fails that
section's checksum) are rejected before anything is written."""
import numpy as np
import pytest

from cases import gpu_sim, rel_inf
from paper_1004_2416_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _case(with_capsule: bool, precision: str):
    caps = [W.Capsule((17.3, 9.6, 8.4), 3.0, 2, W.k_s_for(0.05, 3.0))] if with_capsule else []
    return W.Case("checkpoint-36x20x18", (36, 20, 18), 1.0, 3, precision, W.u_wall_for(18), caps, 60)


def _state(g, with_capsule):
    out = {"u": g.get_velocity(), "f": g.get_populations()}
    if with_capsule:
        out["x"] = g.get_nodes()
        out["D"] = g.taylor(0)["D"]
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
@pytest.mark.parametrize("with_capsule", [False, True])
def test_restart_matches_uninterrupted_run(prec, with_capsule):
    import torch

    case = _case(with_capsule, prec)
    g = gpu_sim(case)
    g.step(37)
    host = g.checkpoint_save()
    dev = torch.empty(g.checkpoint_size(), dtype=torch.uint8, device="cuda")
    g.checkpoint_save(dev)
    assert np.array_equal(dev.cpu().numpy(), host)
    g.step(41)
    ref = _state(g, with_capsule)
    assert g.info().step == 78

    for buf in (host, dev):
        g.checkpoint_restore(buf)
        assert g.info().step == 37
        g.step(41)
        got = _state(g, with_capsule)
        for k in ref:
            if with_capsule:
                tol = {"fp64": 1e-12, "fp32": 1e-5, "fp16": 1e-3}[prec]
                assert rel_inf(np.asarray(got[k]), np.asarray(ref[k])) <= tol, k
            else:
                assert np.array_equal(got[k], ref[k]), k

    # into a fresh object of the same configuration
    g2 = gpu_sim(case)
    g2.checkpoint_restore(host)
    g2.step(41)
    got = _state(g2, with_capsule)
    for k in ref:
        if with_capsule:
            tol = {"fp64": 1e-12, "fp32": 1e-5, "fp16": 1e-3}[prec]
            assert rel_inf(np.asarray(got[k]), np.asarray(ref[k])) <= tol, k
        else:
            assert np.array_equal(got[k], ref[k]), k
    g.close()
    g2.close()


def test_checkpoint_rejects_mismatch_and_corruption():
    from paper_1004_2416_gb300 import iblbm as B

    g = gpu_sim(_case(True, "fp32"))
    g.step(5)
    buf = g.checkpoint_save()
    before = g.get_populations()
    # other precision, other lattice, no capsule
    for other in (gpu_sim(_case(True, "fp64")), gpu_sim(_case(False, "fp32")),
                  gpu_sim(W.Case("c", (36, 20, 20), 1.0, 3, "fp32", W.u_wall_for(20),
                                 [W.Capsule((17.3, 9.6, 8.4), 3.0, 2, 0.01)], 1))):
        with pytest.raises(B.IblbmError) as e:
            other.checkpoint_restore(np.resize(buf, max(buf.size, other.checkpoint_size())))
        assert e.value.code == B.IBLBM_ERR_ARG
        other.close()
    bad = buf.copy()
    bad[0] ^= 0xFF
    with pytest.raises(B.IblbmError) as e:
        g.checkpoint_restore(bad)
    assert e.value.code == B.IBLBM_ERR_ARG
    assert np.array_equal(g.get_populations(), before)  # nothing was written
    # one byte flipped inside a section: the section's checksum no longer
    # matches, in a host buffer and in a device buffer; a truncated buffer is
    # refused by its length
    import torch

    size = g.checkpoint_size()
    for off, section in ((256 + 1234, "populations"), (size - 300, "node velocities")):
        bad = buf.copy()
        bad[off] ^= 0x04
        for b in (bad, torch.from_numpy(bad).cuda()):
            with pytest.raises(B.IblbmError) as e:
                g.checkpoint_restore(b)
            assert e.value.code == B.IBLBM_ERR_ARG and "checksum" in str(e.value), str(e.value)
            assert section in str(e.value)
    for n in (100, size - 1):
        with pytest.raises(B.IblbmError) as e:
            g.checkpoint_restore(buf[:n].copy())
        assert e.value.code == B.IBLBM_ERR_ARG
    assert np.array_equal(g.get_populations(), before)
    g.checkpoint_restore(torch.from_numpy(buf).cuda())  # the intact copy on the device
    assert np.array_equal(g.get_populations(), before)
    # a host buffer declared as device memory is refused
    ptr = B.ctypes.c_void_p(buf.ctypes.data)
    assert B.iblbm_checkpoint_save(g._h, ptr, 1) == B.IBLBM_ERR_ARG
    with pytest.raises(ValueError):
        g.checkpoint_save(np.empty(16, np.uint8))
    g.close()


def test_restore_discards_a_pending_adjoint_run():
    from paper_1004_2416_gb300 import iblbm as B

    g = gpu_sim(_case(True, "fp32"))
    buf = g.checkpoint_save()
    g.adjoint_forward(20, 10)
    g.checkpoint_restore(buf)
    with pytest.raises(B.IblbmError) as e:
        g.adjoint_backward(0)
    assert e.value.code == B.IBLBM_ERR_STATE
    g.close()
