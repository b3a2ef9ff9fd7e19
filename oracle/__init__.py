"""FP64 CPU oracle of the IB-LBM-FEM time step (arXiv:1004.2416), ctypes side.

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(``paper_1004_2416_gb300``) never imports it, and the C sources here share no
code with the CUDA library.

The C library is built by :func:`build` with plain gcc (``-O2
-ffp-contract=off -fopenmp``).  It runs single-threaded unless
:func:`set_threads` asks for more; the thread count changes no result
(the whole-lattice loops write disjoint outputs, and the spreading, the
membrane forces and every reduction stay serial in their fixed order).  Array conventions are those of
``oracle.h``: populations ``[19][nz][ny][nx]``, vector fields
``[3][nz][ny][nx]``, node arrays ``[n][3]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_CS_LIB_PATH = os.path.join(_BUILD, "liboracle_cs.so")
_SOURCES = ["lattice.c", "ibm.c", "membrane.c", "mesh.c", "taylor.c", "diag.c", "sim.c"]
# the complex-step build: the method's sources with real = double _Complex
_CS_SOURCES = ["lattice.c", "ibm.c", "membrane.c", "taylor.c", "sim.c", "tangent.c"]
_lock = threading.Lock()
_lib = None

ERR_STENCIL = -5


def _compile(path: str, sources, defines, force: bool) -> str:
    srcs = [os.path.join(_HERE, s) for s in sources] + [os.path.join(_HERE, "oracle.h")]
    if not force and os.path.exists(path):
        t_lib = os.path.getmtime(path)
        if all(os.path.getmtime(s) <= t_lib for s in srcs):
            return path
    os.makedirs(_BUILD, exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp", *defines,
           "-o", tmp] + [os.path.join(_HERE, s) for s in sources] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` (gcc, FP64, no FMA contraction) and its
    complex-step twin ``liboracle_cs.so`` (the same sources with
    real = double _Complex, for tangent derivatives)."""
    _compile(_CS_LIB_PATH, _CS_SOURCES, ["-DORC_COMPLEX_STEP"], force)
    return _compile(_LIB_PATH, _SOURCES, [], force)


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            _lib = ctypes.CDLL(path)
            _declare(_lib)
    return _lib


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def _declare(L):
    c_int, c_double, c_void_p = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    L.orc_d3q19.argtypes = [_ip, _dp, _ip]
    L.orc_feq.argtypes = [c_int, c_double, _dp]
    L.orc_feq.restype = c_double
    L.orc_feq_linear.argtypes = [c_int, c_double, _dp]
    L.orc_feq_linear.restype = c_double
    L.orc_guo.argtypes = [c_int, c_double, _dp, _dp]
    L.orc_guo.restype = c_double
    L.orc_moments.argtypes = [_dp, _dp, _dp, _dp]
    L.orc_lbm_step.argtypes = [c_int, c_int, c_int, c_double, c_double, _dp, _dp, _dp]
    L.orc_lbm_step_eq.argtypes = [c_int, c_int, c_int, c_double, c_double, _dp, _dp, _dp, c_int]
    L.orc_set_threads.argtypes = [c_int]
    L.orc_get_threads.restype = c_int
    L.orc_sim_set_integrator.argtypes = [c_void_p, c_int]
    L.orc_sim_set_equilibrium.argtypes = [c_void_p, c_int]
    L.orc_init_couette.argtypes = [c_int, c_int, c_int, c_double, _dp]
    L.orc_phi.argtypes = [c_int, c_double]
    L.orc_phi.restype = c_double
    L.orc_stencil_base.argtypes = [c_int, c_double]
    L.orc_spread.argtypes = [c_int, c_int, c_int, c_int, c_int, _dp, _dp, _dp]
    L.orc_interpolate.argtypes = [c_int, c_int, c_int, c_int, c_int, _dp, _dp, _dp]
    L.orc_face_energy.argtypes = [_dp, _dp, c_double, c_double]
    L.orc_face_energy.restype = c_double
    L.orc_face_forces.argtypes = [_dp, _dp, c_double, c_double, _dp]
    L.orc_face_forces.restype = c_double
    L.orc_face_invariants.argtypes = [_dp, _dp, _dp, _dp]
    L.orc_membrane_forces.argtypes = [c_int, _dp, _dp, c_int, _ip, c_double, c_double, _dp]
    L.orc_membrane_forces.restype = c_double
    L.orc_icosphere.argtypes = [c_int, c_double, _dp, _dp, _ip]
    L.orc_taylor.argtypes = [c_int, _dp, c_int, _ip, _dp]
    L.orc_eig3.argtypes = [_dp, _dp, _dp]
    L.orc_tank_treading.argtypes = [c_int, _dp, _dp, _dp, _dp, c_double, _dp]
    L.orc_tank_treading.restype = c_double
    L.orc_ellipsoid_fit.argtypes = [c_int, _dp, _dp, _dp]
    L.orc_face_area_stats.argtypes = [c_int, _ip, _dp, _dp, _dp]
    L.orc_sim_create.argtypes = [c_int, c_int, c_int, c_double, c_int, c_double]
    L.orc_sim_create.restype = c_void_p
    L.orc_sim_destroy.argtypes = [c_void_p]
    L.orc_sim_add_capsule.argtypes = [c_void_p, c_int, _dp, c_int, _ip, c_double, c_double]
    L.orc_sim_n_nodes.argtypes = [c_void_p]
    L.orc_sim_init_couette.argtypes = [c_void_p]
    L.orc_sim_step.argtypes = [c_void_p, c_int]
    for name in ("get_f", "set_f", "get_nodes", "set_nodes", "get_force_field",
                 "get_node_forces", "get_node_velocities", "get_density", "get_velocity"):
        getattr(L, "orc_sim_" + name).argtypes = [c_void_p, _dp]


_cs_lib = None


def cs_lib() -> ctypes.CDLL:
    """The complex-step build (real = double _Complex) of the oracle."""
    global _cs_lib
    with _lock:
        if _cs_lib is None:
            build()
            L = ctypes.CDLL(_CS_LIB_PATH)
            L.orc_tangent_taylor_D.argtypes = [
                ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                ctypes.c_double, ctypes.c_int, _dp, _dp, ctypes.c_int, _ip, ctypes.c_double, ctypes.c_double,
                ctypes.c_double, ctypes.c_int, ctypes.c_double, _dp]
            L.orc_set_threads.argtypes = [ctypes.c_int]
            _cs_lib = L
    return _cs_lib


def tangent_taylor_D(shape, tau: float, delta_n: int, u_wall: float, X0, tri, ks: float, C: float,
                     n_steps: int, du_wall: float = 0.0, dX0=None, dks: float = 0.0, h: float = 1e-30,
                     threads: int = 1):
    """(D, dD): the Taylor deformation of the final shape after n_steps of the
    coupled step (one capsule starting in its reference shape X0, Couette start)
    and its derivative along (du_wall, dX0, dks) at fixed C = k_alpha / k_s, by
    the complex-step method on the whole oracle."""
    L = cs_lib()
    L.orc_set_threads(int(threads))
    X0, tri = _f64(X0), _i32(tri)
    dX = np.zeros_like(X0) if dX0 is None else _f64(dX0)
    out = np.zeros(2)
    nx, ny, nz = shape
    rc = L.orc_tangent_taylor_D(nx, ny, nz, tau, delta_n, u_wall, du_wall, X0.shape[0], _d(X0), _d(dX),
                                tri.shape[0], _i(tri), ks, dks, C, int(n_steps), h, _d(out))
    if rc:
        raise ValueError(f"orc_tangent_taylor_D returned {rc}")
    return float(out[0]), float(out[1])


def set_threads(n: int) -> None:
    """Threads of the whole-lattice loops (1 = none); results do not change."""
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _i(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(_ip)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


# ---- lattice ----------------------------------------------------------------

def d3q19():
    """(c [19,3] int, w [19], opp [19]) of the oracle's velocity set."""
    c = np.zeros((19, 3), np.int32)
    w = np.zeros(19)
    opp = np.zeros(19, np.int32)
    lib().orc_d3q19(_i(c), _d(w), _i(opp))
    return c, w, opp


def feq(i: int, rho: float, u) -> float:
    return lib().orc_feq(i, rho, _d(_f64(u)))


def feq_linear(i: int, rho: float, u) -> float:
    """The linearised equilibrium of Sec. IV.A."""
    return lib().orc_feq_linear(i, rho, _d(_f64(u)))


def guo(i: int, tau: float, u, f) -> float:
    return lib().orc_guo(i, tau, _d(_f64(u)), _d(_f64(f)))


def moments(fi, force):
    rho = np.zeros(1)
    u = np.zeros(3)
    lib().orc_moments(_d(_f64(fi)), _d(_f64(force)), _d(rho), _d(u))
    return float(rho[0]), u


def lbm_step(f: np.ndarray, tau: float, u_wall: float, force: np.ndarray | None = None, order: int = 2):
    """One Eq. (lbequation) step of ``f`` shaped [19, nz, ny, nx] with the
    equilibrium of Eq. (equilibrium) (order 2) or the linearised one of
    Sec. IV.A (order 1)."""
    f = _f64(f)
    _, nz, ny, nx = f.shape
    out = np.zeros_like(f)
    fp = _d(_f64(force)) if force is not None else None
    keep = _f64(force) if force is not None else None
    if keep is not None:
        fp = _d(keep)
    rc = lib().orc_lbm_step_eq(nx, ny, nz, tau, u_wall, _d(f), fp, _d(out), order)
    if rc:
        raise ValueError(f"orc_lbm_step returned {rc}")
    return out


def init_couette(nx: int, ny: int, nz: int, u_wall: float) -> np.ndarray:
    f = np.zeros((19, nz, ny, nx))
    lib().orc_init_couette(nx, ny, nz, u_wall, _d(f))
    return f


# ---- IBM ----------------------------------------------------------------------

def phi(n: int, r: float) -> float:
    return lib().orc_phi(n, float(r))


def stencil_base(n: int, x: float) -> int:
    return lib().orc_stencil_base(n, float(x))


def spread(shape, n: int, x, F) -> np.ndarray:
    nx, ny, nz = shape
    x, F = _f64(x), _f64(F)
    out = np.zeros((3, nz, ny, nx))
    rc = lib().orc_spread(nx, ny, nz, n, x.shape[0], _d(x), _d(F), _d(out))
    if rc:
        raise ValueError(f"orc_spread returned {rc}")
    return out


def interpolate(n: int, x, u_field) -> np.ndarray:
    u_field = _f64(u_field)
    _, nz, ny, nx = u_field.shape
    x = _f64(x)
    out = np.zeros_like(x)
    rc = lib().orc_interpolate(nx, ny, nz, n, x.shape[0], _d(x), _d(u_field), _d(out))
    if rc:
        raise ValueError(f"orc_interpolate returned {rc}")
    return out


# ---- membrane -----------------------------------------------------------------

def face_energy(X0, x, ks: float, ka: float) -> float:
    return lib().orc_face_energy(_d(_f64(X0).ravel().copy()), _d(_f64(x).ravel().copy()), ks, ka)


def face_forces(X0, x, ks: float, ka: float):
    F = np.zeros(9)
    W = lib().orc_face_forces(_d(_f64(X0).ravel().copy()), _d(_f64(x).ravel().copy()), ks, ka, _d(F))
    return W, F.reshape(3, 3)


def face_invariants(X0, x):
    i1 = np.zeros(1)
    i2 = np.zeros(1)
    lib().orc_face_invariants(_d(_f64(X0).ravel().copy()), _d(_f64(x).ravel().copy()), _d(i1), _d(i2))
    return float(i1[0]), float(i2[0])


def membrane_forces(X0, x, tri, ks: float, ka: float):
    X0, x, tri = _f64(X0), _f64(x), _i32(tri)
    F = np.zeros_like(x)
    W = lib().orc_membrane_forces(x.shape[0], _d(X0), _d(x), tri.shape[0], _i(tri), ks, ka, _d(F))
    return W, F


# ---- mesh / Taylor ---------------------------------------------------------------

def icosphere(m: int, r: float, center=(0.0, 0.0, 0.0)):
    nf = 20 * 4 ** m
    nn = nf // 2 + 2
    nodes = np.zeros((nn, 3))
    tri = np.zeros((nf, 3), np.int32)
    got = lib().orc_icosphere(m, r, _d(_f64(center)), _d(nodes), _i(tri))
    if got != nn:
        raise ValueError(f"orc_icosphere returned {got}")
    return nodes, tri


TAYLOR_KEYS = ("D", "theta", "r_a", "r_b", "r_c", "V", "A", "c_x", "c_y", "c_z",
               "I_xx", "I_yy", "I_zz", "I_xy", "I_xz", "I_yz")


def taylor(x, tri) -> dict:
    x, tri = _f64(x), _i32(tri)
    out = np.zeros(16)
    rc = lib().orc_taylor(x.shape[0], _d(x), tri.shape[0], _i(tri), _d(out))
    if rc:
        raise ValueError(f"orc_taylor returned {rc}")
    return dict(zip(TAYLOR_KEYS, out.tolist()))


def eig3(A):
    A = _f64(A).reshape(9).copy()
    ev = np.zeros(3)
    vec = np.zeros(9)
    lib().orc_eig3(_d(A), _d(ev), _d(vec))
    return ev, vec.reshape(3, 3)


# ---- coupled simulation --------------------------------------------------------------

class Sim:
    """The sub-step list of Sec. II.C on one lattice with any number of capsules."""

    def __init__(self, nx: int, ny: int, nz: int, tau: float, delta_n: int, u_wall: float):
        self.shape = (nx, ny, nz)
        self.N = nx * ny * nz
        self._h = lib().orc_sim_create(nx, ny, nz, tau, delta_n, u_wall)
        if not self._h:
            raise ValueError("orc_sim_create failed")
        self._caps = []

    def close(self):
        if self._h:
            lib().orc_sim_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_capsule(self, X0, tri, ks: float, ka: float) -> int:
        X0, tri = _f64(X0), _i32(tri)
        cid = lib().orc_sim_add_capsule(self._h, X0.shape[0], _d(X0), tri.shape[0], _i(tri), ks, ka)
        if cid < 0:
            raise ValueError(f"orc_sim_add_capsule returned {cid}")
        self._caps.append((X0.shape[0], tri))
        return cid

    @property
    def n_nodes(self) -> int:
        return lib().orc_sim_n_nodes(self._h)

    def init_couette(self):
        lib().orc_sim_init_couette(self._h)

    def set_integrator(self, mode: int):
        """0: Euler, Eq. (positionupdate); 1: Adams-Bashforth (Sec. II.C)."""
        if lib().orc_sim_set_integrator(self._h, mode):
            raise ValueError("integrator must be 0 or 1")

    def set_equilibrium(self, order: int):
        """2: Eq. (equilibrium); 1: linearised (Sec. IV.A)."""
        if lib().orc_sim_set_equilibrium(self._h, order):
            raise ValueError("equilibrium order must be 1 or 2")

    def step(self, n: int = 1):
        rc = lib().orc_sim_step(self._h, n)
        if rc:
            raise ValueError(f"orc_sim_step returned {rc}")

    def _get(self, name, shape):
        a = np.zeros(shape)
        getattr(lib(), "orc_sim_" + name)(self._h, _d(a))
        return a

    def get_f(self):
        nx, ny, nz = self.shape
        return self._get("get_f", (19, nz, ny, nx))

    def set_f(self, f):
        lib().orc_sim_set_f(self._h, _d(_f64(f)))

    def get_nodes(self):
        return self._get("get_nodes", (self.n_nodes, 3))

    def set_nodes(self, x):
        x = _f64(x)
        assert x.shape == (self.n_nodes, 3)
        lib().orc_sim_set_nodes(self._h, _d(x))

    def get_force_field(self):
        nx, ny, nz = self.shape
        return self._get("get_force_field", (3, nz, ny, nx))

    def get_node_forces(self):
        return self._get("get_node_forces", (self.n_nodes, 3))

    def get_node_velocities(self):
        return self._get("get_node_velocities", (self.n_nodes, 3))

    def get_density(self):
        nx, ny, nz = self.shape
        return self._get("get_density", (nz, ny, nx))

    def get_velocity(self):
        nx, ny, nz = self.shape
        return self._get("get_velocity", (3, nz, ny, nx))

    def taylor(self, cid: int = 0) -> dict:
        x = self.get_nodes()
        start = sum(n for n, _ in self._caps[:cid])
        n, tri = self._caps[cid]
        return taylor(x[start:start + n], tri)


# ---- diagnostics ------------------------------------------------------------------------------

def tank_treading(x0, x1, c0, c1, dt: float):
    """(per-node omega [n], mean omega) about the centroids in the xz plane."""
    x0, x1 = _f64(x0), _f64(x1)
    om = np.zeros(x0.shape[0])
    mean = lib().orc_tank_treading(x0.shape[0], _d(x0), _d(x1), _d(_f64(c0)), _d(_f64(c1)), dt, _d(om))
    return om, mean


FIT_KEYS = ("zeta_x", "zeta_y", "zeta_z", "zeta_xz", "r_a", "r_b", "r_c", "D", "theta")


def ellipsoid_fit(x, c) -> dict:
    x = _f64(x)
    out = np.zeros(9)
    rc = lib().orc_ellipsoid_fit(x.shape[0], _d(x), _d(_f64(c)), _d(out))
    if rc:
        raise ValueError(f"orc_ellipsoid_fit returned {rc}")
    return dict(zip(FIT_KEYS, out.tolist()))


def face_area_stats(tri, X0, x):
    tri = _i32(tri)
    out = np.zeros(3)
    rc = lib().orc_face_area_stats(tri.shape[0], _i(tri), _d(_f64(X0)), _d(_f64(x)), _d(out))
    if rc:
        raise ValueError(f"orc_face_area_stats returned {rc}")
    return {"mean": out[0], "std": out[1], "max": out[2]}

