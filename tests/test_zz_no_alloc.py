"""The allocation-free capsule reductions (iblbm_taylor_sums_noalloc) against the
regular entry point (iblbm_get_taylor) and the FP64 oracle, through the C ABI.

The allocation-free call serves callers that cannot allocate device memory
when they need the reductions: code whose device memory is all owned by
another allocator (a framework's caching allocator or a fixed arena),
plug-ins called back from such a framework, or loops where an allocation
would synchronise.  Its inputs and output are device buffers owned by the
caller (here PyTorch tensors); its scratch is one fixed device array shared
by every call, so a call on a small mesh right after one on a large mesh must
not pick up the large mesh's leftover partial sums.  This file is collected
last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

KEYS = ("V", "A", "c_x", "c_y", "c_z", "I_xx", "I_yy", "I_zz", "I_xy", "I_xz", "I_yz")


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _deformed(X0, a, c, th, rng):
    R = np.array([[np.cos(th), 0, -np.sin(th)], [0, 1, 0], [np.sin(th), 0, np.cos(th)]])
    x = ((X0 - X0.mean(0)) * np.array([a, 1.0, c])) @ R.T + X0.mean(0)
    return x + rng.uniform(-0.05, 0.05, x.shape)


def _close(got, ref, what):
    for k, v in zip(KEYS, got[:11]):
        tol = 1e-11 * max(abs(ref[k]), 1.0 if k.startswith("c_") else 0.0, 1e-300)
        if k in ("I_xy", "I_yz"):
            tol = 1e-11 * abs(ref["I_xx"])  # off-diagonals vanish up to rounding here
        assert abs(v - ref[k]) <= tol, (what, k, v, ref[k])


def test_no_alloc_matches_regular_entry_point_two_calls():
    """Two calls in a row: first a 20 480-face mesh (160 blocks of partial
    sums), then a 1 280-face mesh (10 blocks) whose reductions must use only
    the blocks it wrote."""
    torch = pytest.importorskip("torch")
    import oracle as O
    from paper_1004_2416_gb300 import Sim, iblbm as B

    torch.cuda.init()
    stream = torch.cuda.current_stream()
    out = torch.full((12,), float("nan"), dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(21)
    s = Sim(64, 64, 64, precision="fp64")
    for call, (sub, (a, c, th)) in enumerate(((5, (1.25, 0.8, 0.4)), (3, (1.1, 0.93, -0.7)))):
        cid = s.add_capsule_icosphere((31.5, 32.0, 30.5), 12.0, sub)
        X0 = s.get_nodes(cid)
        _, tri = s.mesh(cid)
        x = _deformed(X0, a, c, th, rng)
        s.set_nodes(x, cid)
        ref = s.taylor(cid)
        orc = O.taylor(x, tri)
        x_d = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        tri_d = torch.from_numpy(np.ascontiguousarray(tri, np.int32)).cuda()
        origin = np.ascontiguousarray(X0.mean(axis=0))
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        rc = B.iblbm_taylor_sums_noalloc(_ptr(x_d), len(x), _ptr(tri_d), len(tri),
                                         origin.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         _ptr(out), ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, B.iblbm_last_error(None)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert got[11] == 0.0  # no face skipped
        _close(got, ref, f"call {call} vs iblbm_get_taylor")
        # the oracle's face sums of Sec. III, with its own eigen-solver for D
        assert abs(got[0] - orc["V"]) <= 1e-11 * orc["V"]
        assert abs(got[1] - orc["A"]) <= 1e-11 * orc["A"]
        D = B.taylor_from_sums(got)["D"]
        assert abs(D - orc["D"]) <= 1e-9 * abs(orc["D"]), (call, D, orc["D"])


def test_no_alloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    from paper_1004_2416_gb300 import iblbm as B

    x_d = torch.zeros((8, 3), dtype=torch.float64, device="cuda")
    t_d = torch.zeros((8, 3), dtype=torch.int32, device="cuda")
    out = torch.zeros(12, dtype=torch.float64, device="cuda")
    org = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    rc = B.iblbm_taylor_sums_noalloc(_ptr(x_d), 8, _ptr(t_d), 131073, org, _ptr(out), None)
    assert rc == B.IBLBM_ERR_ARG
    assert b"131072" in B.iblbm_last_error(None)
    rc = B.iblbm_taylor_sums_noalloc(None, 8, _ptr(t_d), 8, org, _ptr(out), None)
    assert rc == B.IBLBM_ERR_ARG
