"""ctypes binding of ``include/iblbm.h`` (the IB-LBM-FEM library for GB300).

Argument marshalling only: every computation runs in ``lib/libiblbm.so``.
The module raises ``ImportError`` at import time when the library is not
built (there is no fallback path).  Functions keep the C names
(``iblbm_create`` ...); :class:`Sim` wraps them with numpy arrays.

Streams and device memory can come from PyTorch: pass
``stream=torch.cuda.current_stream()`` to :class:`Sim`, or
``allocator="torch"`` to let the library allocate through PyTorch's caching
allocator (or an ``iblbm_allocator`` of one's own, kept alive by the caller).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# IBLBM_LIBRARY=checked selects the bounds-checked build of the same sources
LIB_PATH = os.path.join(_HERE, "lib", "libiblbm_checked.so" if os.environ.get("IBLBM_LIBRARY") == "checked"
                        else "libiblbm.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'` "
        "(nvcc, sm_103a); there is no non-CUDA fallback")

_lib = ctypes.CDLL(LIB_PATH)

IBLBM_OK = 0
IBLBM_ERR_ARG = -1
IBLBM_ERR_OOM = -2
IBLBM_ERR_CUDA = -3
IBLBM_ERR_UNSTABLE = -4
IBLBM_ERR_STENCIL = -5
IBLBM_ERR_TIMEOUT = -6
IBLBM_ERR_STATE = -7

IBLBM_FP64 = 0
IBLBM_FP32 = 1
IBLBM_FP16 = 2
PRECISIONS = {"fp64": IBLBM_FP64, "fp32": IBLBM_FP32, "fp16": IBLBM_FP16}

_vp = ctypes.c_void_p
_int = ctypes.c_int
_dbl = ctypes.c_double
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_i32p = ctypes.POINTER(ctypes.c_int32)

ALLOC_FN = ctypes.CFUNCTYPE(_vp, ctypes.c_size_t, _vp, _vp)
FREE_FN = ctypes.CFUNCTYPE(None, _vp, _vp, _vp)


class iblbm_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", _vp)]


class iblbm_info(ctypes.Structure):
    _fields_ = [("nx", _int), ("ny", _int), ("nz", _int), ("precision", _int),
                ("delta_points", _int), ("n_capsules", _int), ("n_nodes", _int),
                ("n_faces", _int), ("step", ctypes.c_int64), ("tau", _dbl), ("u_wall", _dbl),
                ("n_runs", _int), ("kernel_launches", ctypes.c_int64)]


class iblbm_run_spec(ctypes.Structure):
    _fields_ = [("nx", _int), ("ny", _int), ("nz", _int), ("tau", _dbl), ("u_wall", _dbl)]


_SIGS = {
    "iblbm_create": (_int, [ctypes.POINTER(_vp), _int, _int, _int, _dbl, _int, _int, _vp,
                            ctypes.POINTER(iblbm_allocator)]),
    "iblbm_destroy": (_int, [_vp]),
    "iblbm_last_error": (ctypes.c_char_p, [_vp]),
    "iblbm_status_string": (ctypes.c_char_p, [_int]),
    "iblbm_get_info": (_int, [_vp, ctypes.POINTER(iblbm_info)]),
    "iblbm_set_shear_walls": (_int, [_vp, _dbl]),
    "iblbm_add_capsule_icosphere": (_int, [_vp, _dbl, _dbl, _dbl, _dbl, _int, _ip]),
    "iblbm_add_capsule_mesh": (_int, [_vp, _dp, _int, _i32p, _int, _ip]),
    "iblbm_set_skalak": (_int, [_vp, _int, _dbl, _dbl]),
    "iblbm_init_fluid": (_int, [_vp, _int]),
    "iblbm_step": (_int, [_vp, ctypes.c_int64]),
    "iblbm_prepare_steps": (_int, [_vp, ctypes.c_int64]),
    "iblbm_set_kernel_timing": (_int, [_vp, _int]),
    "iblbm_get_kernel_times": (_int, [_vp, _dp, ctypes.POINTER(ctypes.c_int64)]),
    "iblbm_collide_kernel": (ctypes.c_char_p, [_vp]),
    "iblbm_set_collide_staging": (_int, [_vp, _int]),
    "iblbm_set_device_wait_limit": (_int, [_vp, ctypes.c_int64]),
    "iblbm_sync": (_int, [_vp]),
    "iblbm_get_velocity": (_int, [_vp, _dp]),
    "iblbm_get_density": (_int, [_vp, _dp]),
    "iblbm_get_populations": (_int, [_vp, _dp]),
    "iblbm_set_populations": (_int, [_vp, _dp]),
    "iblbm_get_force_field": (_int, [_vp, _dp]),
    "iblbm_get_nodes": (_int, [_vp, _int, _dp]),
    "iblbm_set_nodes": (_int, [_vp, _int, _dp]),
    "iblbm_get_node_forces": (_int, [_vp, _int, _dp]),
    "iblbm_get_node_velocities": (_int, [_vp, _int, _dp]),
    "iblbm_get_mesh": (_int, [_vp, _int, _ip, _ip, _i32p]),
    "iblbm_get_taylor": (_int, [_vp, _int, _dp]),
    "iblbm_icosphere": (_int, [_int, _dbl, _dp, _dp, _i32p]),
    "iblbm_set_taylor_recording": (_int, [_vp, _int, _int]),
    "iblbm_get_taylor_records": (_int, [_vp, _int, _int, _dp, ctypes.POINTER(ctypes.c_int64), _ip]),
    "iblbm_profile_kernels": (_int, [_vp, _int, _dp]),
    "iblbm_taylor_sums_noalloc": (_int, [_vp, _int, _vp, _int, _dp, _vp, _vp]),
    "iblbm_taylor_gradient": (_int, [_dp, _int, _i32p, _int, _dp, _dp]),
    "iblbm_adjoint_forward": (_int, [_vp, ctypes.c_int64, _int]),
    "iblbm_adjoint_backward": (_int, [_vp, _int, _dp, _dp, _dp, _dp, _dp]),
    "iblbm_adjoint_taylor": (_int, [_vp, _int, ctypes.c_int64, _int, _dp, _dp, _dp, _dp]),
    "iblbm_checkpoint_size": (_int, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "iblbm_set_interp_mode": (_int, [_vp, _int]),
    "iblbm_set_launch_overlap": (_int, [_vp, _int]),
    "iblbm_set_deterministic_spreading": (_int, [_vp, _int]),
    "iblbm_bounds_checked": (_int, []),
    "iblbm_bounds_faults": (_int, [_vp, ctypes.POINTER(ctypes.c_ulonglong)]),
    "iblbm_read_async": (_int, [_vp, _vp, _vp]),
    "iblbm_taylor_from_sums": (_int, [_vp, _vp]),
    "iblbm_set_integrator": (_int, [_vp, _int]),
    "iblbm_tank_treading": (_int, [_dp, _dp, _int, _dp, _dp, _dbl, _dp, _dp]),
    "iblbm_ellipsoid_fit": (_int, [_dp, _int, _dp, _dp]),
    "iblbm_mesh_quality": (_int, [_vp, _int, _dp]),
    "iblbm_set_equilibrium": (_int, [_vp, _int]),
    "iblbm_checkpoint_save": (_int, [_vp, _vp, _int]),
    "iblbm_checkpoint_restore": (_int, [_vp, _vp, ctypes.c_size_t, _int]),
    "iblbm_batch_create": (_int, [ctypes.POINTER(_vp), ctypes.POINTER(iblbm_run_spec), _int, _int, _int,
                                  _vp, ctypes.POINTER(iblbm_allocator)]),
    "iblbm_create_slabs": (_int, [ctypes.POINTER(_vp), _int, _int, _int, _dbl, _int, _int, _int, _vp,
                                  ctypes.POINTER(iblbm_allocator)]),
    "iblbm_get_slab": (_int, [_vp, _int, _ip, _ip]),
    "iblbm_slab_configure": (_int, [_vp, _int, _int]),
    "iblbm_slab_step_begin": (_int, [_vp]),
    "iblbm_slab_columns_size": (_int, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "iblbm_slab_get_columns": (_int, [_vp, _vp, _int]),
    "iblbm_slab_set_columns": (_int, [_vp, _vp, _vp, _int]),
    "iblbm_slab_partials_size": (_int, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "iblbm_slab_get_partials": (_int, [_vp, _vp, _int]),
    "iblbm_slab_step_end": (_int, [_vp, _vp, _int, _int]),
    "iblbm_add_capsule_icosphere_in_run": (_int, [_vp, _int, _dbl, _dbl, _dbl, _dbl, _int, _ip]),
    "iblbm_autotune_tiles": (_int, [_vp, _int]),
    "iblbm_get_run_tile": (_int, [_vp, _int, _ip, _ip]),
    "iblbm_get_run_velocity": (_int, [_vp, _int, _dp]),
    "iblbm_get_run_populations": (_int, [_vp, _int, _dp]),
    "iblbm_set_run_populations": (_int, [_vp, _int, _dp]),
}

for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    globals()[_name] = _f


class IblbmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{iblbm_status_string(code).decode()} ({code}): {msg}")
        self.code = code


def _check(rc: int, handle=None):
    if rc != IBLBM_OK:
        msg = iblbm_last_error(handle).decode(errors="replace")
        raise IblbmError(rc, msg)


def _d(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _buffer(buf, need: int):
    """(pointer, on_device) of a contiguous byte buffer: a numpy array or a torch
    tensor on the host or the device, of at least `need` bytes."""
    if isinstance(buf, np.ndarray):
        if not buf.flags["C_CONTIGUOUS"] or buf.nbytes < need:
            raise ValueError(f"need a C-contiguous buffer of at least {need} bytes")
        return ctypes.c_void_p(buf.ctypes.data), 0
    if hasattr(buf, "data_ptr") and hasattr(buf, "is_cuda"):
        nbytes = buf.numel() * buf.element_size()
        if not buf.is_contiguous() or nbytes < need:
            raise ValueError(f"need a contiguous buffer of at least {need} bytes")
        return ctypes.c_void_p(buf.data_ptr()), 1 if buf.is_cuda else 0
    raise TypeError("checkpoint buffers are numpy arrays or torch tensors")


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


def _torch_allocator():
    import torch

    live = {}

    def _alloc(nbytes, stream, ctx):
        t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
        live[t.data_ptr()] = t
        return t.data_ptr()

    def _free(ptr, stream, ctx):
        live.pop(ptr, None)

    a = iblbm_allocator(ALLOC_FN(_alloc), FREE_FN(_free), None)
    return a, live


def icosphere(subdivisions: int, radius: float, center=(0.0, 0.0, 0.0)):
    """The library's canonical icosphere (host only): nodes [n, 3], faces [f, 3]."""
    nf = 20 * 4 ** subdivisions
    nodes = np.empty((nf // 2 + 2, 3), np.float64)
    tri = np.empty((nf, 3), np.int32)
    c = np.ascontiguousarray(center, np.float64)
    _check(iblbm_icosphere(subdivisions, radius, _d(c), _d(nodes), tri.ctypes.data_as(_i32p)))
    return nodes, tri


def taylor_gradient(nodes, tri):
    """(D, dD/dx [n, 3]) of one closed membrane (host, FP64)."""
    x = np.ascontiguousarray(nodes, np.float64)
    t = np.ascontiguousarray(tri, np.int32)
    D = ctypes.c_double()
    g = np.empty_like(x)
    _check(iblbm_taylor_gradient(_d(x), len(x), t.ctypes.data_as(_i32p), len(t), ctypes.byref(D), _d(g)))
    return D.value, g


TAYLOR_KEYS = ("D", "theta", "r_a", "r_b", "r_c", "V", "A", "c_x", "c_y", "c_z",
               "I_xx", "I_yy", "I_zz", "I_xy", "I_xz", "I_yz")


class Sim:
    """One lattice with its capsules (owns an ``iblbm_sim``)."""

    def __init__(self, nx: int, ny: int, nz: int, tau: float = 1.0, precision="fp32",
                 delta_points: int = 3, stream=None, allocator=None):
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self._keep = None
        alloc_p = None
        if allocator == "torch":
            a, live = _torch_allocator()
            self._keep = (a, live)
            alloc_p = ctypes.pointer(a)
        elif isinstance(allocator, iblbm_allocator):  # the caller keeps its callbacks alive
            self._keep = allocator
            alloc_p = ctypes.pointer(allocator)
        h = _vp()
        rc = iblbm_create(ctypes.byref(h), nx, ny, nz, tau, prec, delta_points,
                          _stream_handle(stream), alloc_p)
        if rc != IBLBM_OK:
            raise IblbmError(rc, iblbm_last_error(None).decode(errors="replace"))
        self._h = h
        self.shape = (nx, ny, nz)
        self.ncell = nx * ny * nz
        self._ncaps = 0

    @classmethod
    def batch(cls, runs, precision="fp32", delta_points: int = 3, stream=None):
        """Batch of independent lattices; runs = [(nx, ny, nz, tau, u_wall), ...]."""
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        arr = (iblbm_run_spec * len(runs))(*[iblbm_run_spec(int(a), int(b), int(c), float(t), float(u))
                                             for a, b, c, t, u in runs])
        h = _vp()
        rc = iblbm_batch_create(ctypes.byref(h), arr, len(runs), prec, delta_points,
                                _stream_handle(stream), None)
        if rc != IBLBM_OK:
            raise IblbmError(rc, iblbm_last_error(None).decode(errors="replace"))
        self = cls.__new__(cls)
        self._keep = None
        self._h = h
        self.runs = [tuple(r[:3]) for r in runs]
        self.shape = self.runs[0]
        self.ncell = sum(a * b * c for a, b, c in self.runs)
        self._ncaps = 0
        return self

    @classmethod
    def slabs(cls, nx: int, ny: int, nz: int, n_slabs: int, tau: float = 1.0, precision="fp32",
              delta_points: int = 3, stream=None):
        """One nx*ny*nz lattice decomposed into n_slabs x-slabs (iblbm_create_slabs)."""
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        h = _vp()
        rc = iblbm_create_slabs(ctypes.byref(h), nx, ny, nz, tau, prec, delta_points, n_slabs,
                                _stream_handle(stream), None)
        if rc != IBLBM_OK:
            raise IblbmError(rc, iblbm_last_error(None).decode(errors="replace"))
        self = cls.__new__(cls)
        self._keep = None
        self._h = h
        self.shape = (nx, ny, nz)
        self.ncell = nx * ny * nz
        self.runs = [self.shape]
        self._ncaps = 0
        return self

    # x-slab phases of one slab held by this process (iblbm_slab_*); buffers are
    # host numpy arrays of bytes
    def slab_configure(self, x0: int, nx_global: int):
        _check(iblbm_slab_configure(self._h, int(x0), int(nx_global)), self._h)

    def slab_step_begin(self):
        _check(iblbm_slab_step_begin(self._h), self._h)

    def slab_columns(self) -> np.ndarray:
        n = ctypes.c_size_t()
        _check(iblbm_slab_columns_size(self._h, ctypes.byref(n)), self._h)
        out = np.empty(n.value, np.uint8)
        _check(iblbm_slab_get_columns(self._h, out.ctypes.data_as(_vp), 0), self._h)
        return out

    def slab_set_columns(self, left: np.ndarray, right: np.ndarray):
        left, right = np.ascontiguousarray(left, np.uint8), np.ascontiguousarray(right, np.uint8)
        _check(iblbm_slab_set_columns(self._h, left.ctypes.data_as(_vp), right.ctypes.data_as(_vp), 0), self._h)

    def slab_partials(self) -> np.ndarray:
        n = ctypes.c_size_t()
        _check(iblbm_slab_partials_size(self._h, ctypes.byref(n)), self._h)
        out = np.empty(max(n.value, 1), np.uint8)
        _check(iblbm_slab_get_partials(self._h, out.ctypes.data_as(_vp), 0), self._h)
        return out[:n.value]

    def slab_step_end(self, parts: np.ndarray, n_parts: int):
        parts = np.ascontiguousarray(parts, np.uint8)
        _check(iblbm_slab_step_end(self._h, parts.ctypes.data_as(_vp), int(n_parts), 0), self._h)

    def slab(self, k: int):
        """(first global column, width) of slab k of a slab group."""
        x0, w = _int(), _int()
        _check(iblbm_get_slab(self._h, k, ctypes.byref(x0), ctypes.byref(w)), self._h)
        return x0.value, w.value

    def add_capsule_icosphere_in_run(self, run: int, center, radius: float, subdivisions: int) -> int:
        cid = _int()
        _check(iblbm_add_capsule_icosphere_in_run(self._h, run, *map(float, center), float(radius),
                                                  int(subdivisions), ctypes.byref(cid)), self._h)
        self._ncaps += 1
        return cid.value

    def autotune_tiles(self, repeats: int = 5):
        _check(iblbm_autotune_tiles(self._h, repeats), self._h)

    def run_tile(self, run: int):
        tx, ty = _int(), _int()
        _check(iblbm_get_run_tile(self._h, run, ctypes.byref(tx), ctypes.byref(ty)), self._h)
        return tx.value, ty.value

    def get_run_velocity(self, run: int):
        nx, ny, nz = self.runs[run]
        out = np.empty((3, nz, ny, nx), np.float64)
        _check(iblbm_get_run_velocity(self._h, run, _d(out)), self._h)
        return out

    def get_run_populations(self, run: int):
        nx, ny, nz = self.runs[run]
        out = np.empty((19, nz, ny, nx), np.float64)
        _check(iblbm_get_run_populations(self._h, run, _d(out)), self._h)
        return out

    def set_run_populations(self, run: int, f):
        nx, ny, nz = self.runs[run]
        f = np.ascontiguousarray(f, np.float64)
        assert f.shape == (19, nz, ny, nx)
        _check(iblbm_set_run_populations(self._h, run, _d(f)), self._h)

    def close(self):
        if getattr(self, "_h", None):
            iblbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    def info(self) -> iblbm_info:
        out = iblbm_info()
        _check(iblbm_get_info(self._h, ctypes.byref(out)), self._h)
        return out

    def set_shear_walls(self, u_wall: float):
        _check(iblbm_set_shear_walls(self._h, u_wall), self._h)

    def add_capsule_icosphere(self, center, radius: float, subdivisions: int) -> int:
        cid = _int()
        _check(iblbm_add_capsule_icosphere(self._h, *map(float, center), float(radius),
                                           int(subdivisions), ctypes.byref(cid)), self._h)
        self._ncaps += 1
        return cid.value

    def add_capsule_mesh(self, nodes, tri) -> int:
        x = np.ascontiguousarray(nodes, np.float64)
        t = np.ascontiguousarray(tri, np.int32)
        cid = _int()
        _check(iblbm_add_capsule_mesh(self._h, _d(x), x.shape[0], t.ctypes.data_as(_i32p),
                                      t.shape[0], ctypes.byref(cid)), self._h)
        self._ncaps += 1
        return cid.value

    def set_skalak(self, k_s: float, C: float = 1.0, capsule_id: int = -1):
        _check(iblbm_set_skalak(self._h, capsule_id, k_s, C), self._h)

    def init_fluid(self, mode: int = 1):
        _check(iblbm_init_fluid(self._h, mode), self._h)

    def step(self, n: int = 1):
        _check(iblbm_step(self._h, int(n)), self._h)

    def sync(self):
        _check(iblbm_sync(self._h), self._h)

    def _field(self, fn, shape):
        out = np.empty(shape, np.float64)
        _check(fn(self._h, _d(out)), self._h)
        return out

    def get_velocity(self):
        nx, ny, nz = self.shape
        return self._field(iblbm_get_velocity, (3, nz, ny, nx))

    def get_density(self):
        nx, ny, nz = self.shape
        return self._field(iblbm_get_density, (nz, ny, nx))

    def get_populations(self):
        nx, ny, nz = self.shape
        return self._field(iblbm_get_populations, (19, nz, ny, nx))

    def set_populations(self, f):
        nx, ny, nz = self.shape
        f = np.ascontiguousarray(f, np.float64)
        assert f.shape == (19, nz, ny, nx)
        _check(iblbm_set_populations(self._h, _d(f)), self._h)

    def get_force_field(self):
        nx, ny, nz = self.shape
        return self._field(iblbm_get_force_field, (3, nz, ny, nx))

    def n_nodes(self, capsule_id: int = -1) -> int:
        if capsule_id == -1:
            return self.info().n_nodes
        return self.mesh(capsule_id)[0]

    def mesh(self, capsule_id: int):
        nn, nt = _int(), _int()
        _check(iblbm_get_mesh(self._h, capsule_id, ctypes.byref(nn), ctypes.byref(nt), None), self._h)
        tri = np.empty((nt.value, 3), np.int32)
        _check(iblbm_get_mesh(self._h, capsule_id, ctypes.byref(nn), ctypes.byref(nt),
                              tri.ctypes.data_as(_i32p)), self._h)
        return nn.value, tri

    def _nodes(self, fn, capsule_id):
        out = np.empty((self.n_nodes(capsule_id), 3), np.float64)
        _check(fn(self._h, capsule_id, _d(out)), self._h)
        return out

    def get_nodes(self, capsule_id: int = -1):
        return self._nodes(iblbm_get_nodes, capsule_id)

    def set_nodes(self, x, capsule_id: int = -1):
        x = np.ascontiguousarray(x, np.float64)
        assert x.shape == (self.n_nodes(capsule_id), 3)
        _check(iblbm_set_nodes(self._h, capsule_id, _d(x)), self._h)

    def get_node_forces(self, capsule_id: int = -1):
        return self._nodes(iblbm_get_node_forces, capsule_id)

    def get_node_velocities(self, capsule_id: int = -1):
        return self._nodes(iblbm_get_node_velocities, capsule_id)

    def set_taylor_recording(self, every: int, ring: int = 1024):
        _check(iblbm_set_taylor_recording(self._h, every, ring), self._h)

    def taylor_records(self, capsule_id: int = 0, max_records: int = 1 << 20):
        """(steps [n], records [n, 16]) of the recorded shape measures."""
        n = _int()
        _check(iblbm_get_taylor_records(self._h, capsule_id, 0, None, None, ctypes.byref(n)), self._h)
        out = np.empty((max(1, min(max_records, 1 << 24)), 16), np.float64)
        steps = np.empty(out.shape[0], np.int64)
        _check(iblbm_get_taylor_records(self._h, capsule_id, out.shape[0], _d(out),
                                        steps.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                        ctypes.byref(n)), self._h)
        return steps[:n.value], out[:n.value]

    def profile_kernels(self, n_steps: int) -> dict:
        ms = np.zeros(4, np.float64)
        _check(iblbm_profile_kernels(self._h, int(n_steps), _d(ms)), self._h)
        return dict(zip(("force_spread", "collide_stream", "interp_advect", "taylor"), ms.tolist()))

    def prepare_steps(self, n: int):
        """Captures the graphs a following step(n) replays (runs nothing)."""
        _check(iblbm_prepare_steps(self._h, int(n)), self._h)

    def set_kernel_timing(self, on: bool = True):
        _check(iblbm_set_kernel_timing(self._h, 1 if on else 0), self._h)

    def kernel_times(self) -> dict:
        """Mean device ms per step of the kernel groups of the last replay of
        every step graph replayed since the previous call (kernel timing on)."""
        ms = np.zeros(3)
        n = ctypes.c_int64(0)
        _check(iblbm_get_kernel_times(self._h, _d(ms), ctypes.byref(n)), self._h)
        return {"force_spread": ms[0], "collide_stream": ms[1], "interp_advect": ms[2], "steps": int(n.value)}

    def collide_kernel(self) -> str:
        return iblbm_collide_kernel(self._h).decode()

    def set_collide_staging(self, mode: int):
        """-1 automatic, 0 direct loads, 1 populations staged by bulk copies."""
        _check(iblbm_set_collide_staging(self._h, int(mode)), self._h)

    def set_device_wait_limit(self, ns: int):
        _check(iblbm_set_device_wait_limit(self._h, int(ns)), self._h)

    def adjoint_forward(self, n_steps: int, checkpoint_every: int):
        _check(iblbm_adjoint_forward(self._h, int(n_steps), int(checkpoint_every)), self._h)

    def adjoint_backward(self, capsule_id: int = 0) -> dict:
        n = self.n_nodes(capsule_id)
        D, dks, duw = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        gX0 = np.empty((n, 3), np.float64)
        gx0 = np.empty((n, 3), np.float64)
        _check(iblbm_adjoint_backward(self._h, capsule_id, ctypes.byref(D), ctypes.byref(dks),
                                      ctypes.byref(duw), _d(gX0), _d(gx0)), self._h)
        return {"D": D.value, "dD_dks": dks.value, "dD_duw": duw.value, "dD_dX0": gX0, "dD_dx0": gx0}

    def adjoint_taylor(self, n_steps: int, checkpoint_every: int, capsule_id: int = 0) -> dict:
        """Forward run with checkpoints and reverse sweep in one call: D and its
        derivatives with respect to k_s, the capillary number (through u_wall)
        and the reference (= initial) shape X0."""
        n = self.n_nodes(capsule_id)
        D, dks, dca = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        gX0 = np.empty((n, 3), np.float64)
        _check(iblbm_adjoint_taylor(self._h, capsule_id, int(n_steps), int(checkpoint_every), ctypes.byref(dks),
                                    ctypes.byref(dca), _d(gX0), ctypes.byref(D)), self._h)
        return {"D": D.value, "dD_dks": dks.value, "dD_dCa": dca.value, "dD_dX0": gX0}

    def mesh_quality(self, capsule_id: int = 0) -> dict:
        """Face-area deviation statistics and volume drift of a capsule."""
        out = np.zeros(4)
        _check(iblbm_mesh_quality(self._h, capsule_id, _d(out)), self._h)
        return {"dA_mean": out[0], "dA_std": out[1], "dA_max": out[2], "dV": out[3]}

    def set_integrator(self, mode: int):
        """0: Euler (Eq. positionupdate); 1: Adams-Bashforth (Sec. II.C)."""
        _check(iblbm_set_integrator(self._h, int(mode)), self._h)

    def set_equilibrium(self, order: int):
        """2: Eq. (equilibrium); 1: the linearised form of Sec. IV.A."""
        _check(iblbm_set_equilibrium(self._h, int(order)), self._h)

    def set_interp_mode(self, mode: int):
        """-1 automatic (default), 0 gather at the stencil cells, 1 cell velocities first."""
        _check(iblbm_set_interp_mode(self._h, int(mode)), self._h)

    def bounds_faults(self) -> int:
        """Index faults counted by the bounds-checked build since the last call."""
        n = ctypes.c_ulonglong()
        _check(iblbm_bounds_faults(self._h, ctypes.byref(n)), self._h)
        return n.value

    def set_deterministic_spreading(self, on: bool):
        """Force density summed in 64-bit fixed point: bit-reproducible steps."""
        _check(iblbm_set_deterministic_spreading(self._h, 1 if on else 0), self._h)

    def set_launch_overlap(self, mode):
        """Programmatic dependent launch of the step kernels: True/1 on,
        False/0 off, -1 automatic (default: on for dense suspensions)."""
        m = -1 if mode == -1 else (1 if mode else 0)
        _check(iblbm_set_launch_overlap(self._h, m), self._h)

    def checkpoint_size(self) -> int:
        n = ctypes.c_size_t()
        _check(iblbm_checkpoint_size(self._h, ctypes.byref(n)), self._h)
        return n.value

    def checkpoint_save(self, buf=None):
        """Writes a checkpoint into buf (a uint8 torch tensor on the device or a
        numpy uint8 array on the host, at least checkpoint_size() bytes) or, with
        buf None, into a new numpy array, which is returned."""
        if buf is None:
            buf = np.empty(self.checkpoint_size(), np.uint8)
        ptr, dev = _buffer(buf, self.checkpoint_size())
        _check(iblbm_checkpoint_save(self._h, ptr, dev), self._h)
        return buf

    def checkpoint_restore(self, buf):
        """Restores from buf (as checkpoint_save writes it); the library checks
        the header, the length and the sections' checksums first."""
        ptr, dev = _buffer(buf, 0)
        nbytes = buf.nbytes if isinstance(buf, np.ndarray) else buf.numel() * buf.element_size()
        _check(iblbm_checkpoint_restore(self._h, ptr, nbytes, dev), self._h)

    def taylor(self, capsule_id: int = 0) -> dict:
        out = np.empty(16, np.float64)
        _check(iblbm_get_taylor(self._h, capsule_id, _d(out)), self._h)
        return dict(zip(TAYLOR_KEYS, out.tolist()))

    def read_async(self, nodes_out=None, sums_out=None):
        """Enqueues copies of all node positions ([n][3] doubles) and of every
        capsule's 12 reduced sums ([n_capsules][12] doubles) into the given
        host arrays (numpy or CPU torch, preferably pinned) and returns at
        once; they hold the values after the next synchronising call."""
        inf = self.info()
        n, nc = inf.n_nodes, inf.n_capsules
        pn = _buffer(nodes_out, 24 * n)[0] if nodes_out is not None else None
        ps = _buffer(sums_out, 96 * nc)[0] if sums_out is not None else None
        _check(iblbm_read_async(self._h, pn, ps), self._h)


def tank_treading(x_then, x_now, c_then, c_now, dt: float):
    """Per-node angular velocities [n] about the centroid in the xz plane, and
    their mean (host only)."""
    x0 = np.ascontiguousarray(x_then, np.float64)
    x1 = np.ascontiguousarray(x_now, np.float64)
    om = np.empty(x0.shape[0], np.float64)
    mean = ctypes.c_double()
    _check(iblbm_tank_treading(_d(x0), _d(x1), x0.shape[0], _d(np.ascontiguousarray(c_then, np.float64)),
                               _d(np.ascontiguousarray(c_now, np.float64)), float(dt), _d(om), ctypes.byref(mean)))
    return om, mean.value


def taylor_from_sums(sums) -> dict:
    """The shape values of Sim.taylor from one capsule's 12 reduced sums (host only)."""
    r = np.ascontiguousarray(sums, np.float64).reshape(12)
    out = np.empty(16, np.float64)
    _check(iblbm_taylor_from_sums(_d(r), _d(out)))
    return dict(zip(TAYLOR_KEYS, out.tolist()))


FIT_KEYS = ("zeta_x", "zeta_y", "zeta_z", "zeta_xz", "r_a", "r_b", "r_c", "D", "theta")


def ellipsoid_fit(nodes, center) -> dict:
    """The fit of Eq. (chisquare) about center (host only)."""
    x = np.ascontiguousarray(nodes, np.float64)
    out = np.empty(9, np.float64)
    _check(iblbm_ellipsoid_fit(_d(x), x.shape[0], _d(np.ascontiguousarray(center, np.float64)), _d(out)))
    return dict(zip(FIT_KEYS, out.tolist()))

