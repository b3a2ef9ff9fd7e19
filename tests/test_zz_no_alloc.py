"""The allocation-free capsule reductions (iblbm_taylor_sums_noalloc) against the
regular entry point (iblbm_get_taylor), through the C ABI.

The allocation-free call serves callers that cannot allocate device memory
when they need the reductions (inside a framework's graph capture, with all
device memory owned by another allocator, or in loops where an allocation
would synchronise).  Its inputs and output are device buffers owned by the
caller (here PyTorch tensors); its scratch is a fixed device array, so two
calls in a row must not see each other's data.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

KEYS = ("V", "A", "c_x", "c_y", "c_z", "I_xx", "I_yy", "I_zz", "I_xy", "I_xz", "I_yz")


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_no_alloc_matches_regular_entry_point_two_calls():
    torch = pytest.importorskip("torch")
    from paper_1004_2416_gb300 import Sim, iblbm as B

    torch.cuda.init()
    s = Sim(64, 64, 64, precision="fp64")
    cid = s.add_capsule_icosphere((31.5, 32.0, 30.5), 12.0, 4)  # 2562 nodes, 5120 faces
    X0 = s.get_nodes(cid)
    _, tri = s.mesh(cid)
    tri_d = torch.from_numpy(np.ascontiguousarray(tri, np.int32)).cuda()
    out = torch.full((12,), float("nan"), dtype=torch.float64, device="cuda")
    origin = np.ascontiguousarray(X0.mean(axis=0))
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(21)
    for call, (a, c, th) in enumerate(((1.25, 0.8, 0.4), (1.1, 0.93, -0.7))):
        R = np.array([[np.cos(th), 0, -np.sin(th)], [0, 1, 0], [np.sin(th), 0, np.cos(th)]])
        x = ((X0 - X0.mean(0)) * np.array([a, 1.0, c])) @ R.T + X0.mean(0)
        x = x + rng.uniform(-0.05, 0.05, x.shape)
        s.set_nodes(x, cid)
        ref = s.taylor(cid)
        x_d = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        torch.cuda.synchronize()
        rc = B.iblbm_taylor_sums_noalloc(_ptr(x_d), len(x), _ptr(tri_d), len(tri),
                                         origin.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         _ptr(out), ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, B.iblbm_last_error(None)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert got[11] == 0.0  # no face skipped
        scale = {"c_x": 1.0, "c_y": 1.0, "c_z": 1.0}
        for k, v in zip(KEYS, got[:11]):
            tol = 1e-11 * max(abs(ref[k]), scale.get(k, 0.0), 1e-300)
            if k in ("I_xy", "I_yz"):
                tol = 1e-11 * abs(ref["I_xx"])  # off-diagonals vanish up to rounding here
            assert abs(v - ref[k]) <= tol, (call, k, v, ref[k])


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
