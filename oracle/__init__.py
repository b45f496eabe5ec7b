"""FP64 CPU oracle for the DG Euler right-hand side and LSERK45 step.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
CPU-baseline leg of bench.py -- never by the product path, which shares no
code with it.  This module only marshals numpy arrays into the C oracle
(dg_oracle.c), where all of the arithmetic lives.

Arrays use the layout Q[field][element][k][j][i] (C order), fields
(rho, rho u, rho v, rho w, rho E), element e = ex + nx*(ey + ny*ez).
"""
import ctypes
import os

import numpy as np

from .build import build_oracle

NF = 5


class _Mesh(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("p", ctypes.c_int),
                ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("z0", ctypes.c_double),
                ("Lx", ctypes.c_double), ("Ly", ctypes.c_double), ("Lz", ctypes.c_double),
                ("gamma", ctypes.c_double)]


_ODE_CB = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_int64,
                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double))
_DP = ctypes.POINTER(ctypes.c_double)

_lib = None


def load(path=None):
    """Load (building first if needed) the oracle library; a path selects a variant."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build_oracle()))
    return _lib


def _bind(lib):
    M = ctypes.POINTER(_Mesh)
    lib.dgo_gl_nodes.argtypes = [ctypes.c_int, _DP, _DP]
    lib.dgo_lagrange.argtypes = [ctypes.c_int, _DP, ctypes.c_int, ctypes.c_double]
    lib.dgo_lagrange.restype = ctypes.c_double
    lib.dgo_lagrange_deriv.argtypes = [ctypes.c_int, _DP, ctypes.c_int, ctypes.c_double]
    lib.dgo_lagrange_deriv.restype = ctypes.c_double
    lib.dgo_flux.argtypes = [ctypes.c_int, _DP, ctypes.c_double, _DP]
    lib.dgo_flux.restype = None
    lib.dgo_lf_flux.argtypes = [ctypes.c_int, _DP, _DP, ctypes.c_double, _DP]
    lib.dgo_lf_flux.restype = None
    lib.dgo_rhs_o1.argtypes = [M, _DP, _DP]
    lib.dgo_rhs_o2.argtypes = [M, _DP, _DP]
    lib.dgo_rhs_o2_elements.argtypes = [M, _DP, ctypes.c_int64,
                                        ctypes.POINTER(ctypes.c_int64), _DP]
    lib.dgo_lserk_coeffs.argtypes = [_DP, _DP]
    lib.dgo_lserk_coeffs.restype = None
    lib.dgo_lserk_ode.argtypes = [ctypes.c_int64, _DP, ctypes.c_int, ctypes.c_double, _ODE_CB]
    lib.dgo_rk_steps.argtypes = [M, _DP, _DP, ctypes.c_double, ctypes.c_int]
    lib.dgo_cfl_dt.argtypes = [M, _DP, ctypes.c_double, _DP]
    lib.dgo_cfl_dt.restype = ctypes.c_double
    lib.dgo_norms.argtypes = [M, _DP, _DP, _DP]
    lib.dgo_state_init.argtypes = [M, ctypes.c_int, _DP, ctypes.c_int, _DP]
    lib.dgo_ztraces.argtypes = [M, _DP, _DP, _DP]
    lib.dgo_rhs_o2_zhalo.argtypes = [M, _DP, _DP, _DP, _DP]
    lib.dgo_rk_stage.argtypes = [M, _DP, _DP, ctypes.c_double, ctypes.c_int, _DP, _DP]
    lib.dgo_num_threads.restype = ctypes.c_int
    lib.dgo_set_num_threads.argtypes = [ctypes.c_int]
    lib.dgo_set_num_threads.restype = None
    return lib


def _ptr(a):
    return a.ctypes.data_as(_DP)


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


class Mesh:
    """Periodic Cartesian box [x0, x0+Lx] x ... split into nx*ny*nz elements of degree p."""

    def __init__(self, nx, ny, nz, p, x0=0.0, y0=0.0, z0=0.0, Lx=1.0, Ly=1.0, Lz=1.0,
                 gamma=1.4, lib=None):
        self.nx, self.ny, self.nz, self.p = nx, ny, nz, p
        self.N = p + 1
        self.E = nx * ny * nz
        self.gamma = gamma
        self.box = (x0, y0, z0, Lx, Ly, Lz)
        self._m = _Mesh(nx, ny, nz, p, x0, y0, z0, Lx, Ly, Lz, gamma)
        self.lib = lib or load()

    @property
    def shape(self):
        N = self.N
        return (NF, self.E, N, N, N)

    def zeros(self):
        return np.zeros(self.shape, dtype=np.float64)

    def rhs(self, Q, form="o2"):
        Q = _f64(Q)
        R = np.empty_like(Q)
        fn = self.lib.dgo_rhs_o2 if form == "o2" else self.lib.dgo_rhs_o1
        st = fn(ctypes.byref(self._m), _ptr(Q), _ptr(R))
        if st:
            raise RuntimeError(f"oracle rhs failed ({st})")
        return R

    def rhs_elements(self, Q, elems):
        """O2 right-hand side of the listed elements only: shape (5, len(elems), N, N, N)."""
        Q = _f64(Q)
        el = np.ascontiguousarray(np.asarray(elems, dtype=np.int64))
        R = np.empty((NF, el.size, self.N, self.N, self.N))
        st = self.lib.dgo_rhs_o2_elements(ctypes.byref(self._m), _ptr(Q), el.size,
                                          el.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _ptr(R))
        if st:
            raise RuntimeError(f"oracle rhs_elements failed ({st})")
        return R

    def rk_steps(self, Q, dt, nsteps=1):
        """nsteps LSERK45 steps at fixed dt; returns (Q_new, dQ) as new arrays."""
        Q = _f64(Q).copy()
        dQ = np.zeros_like(Q)
        st = self.lib.dgo_rk_steps(ctypes.byref(self._m), _ptr(Q), _ptr(dQ), float(dt), int(nsteps))
        if st:
            raise RuntimeError(f"oracle rk step failed ({st})")
        return Q, dQ

    def cfl_dt(self, Q, cfl):
        Q = _f64(Q)
        lam = ctypes.c_double(0.0)
        dt = self.lib.dgo_cfl_dt(ctypes.byref(self._m), _ptr(Q), float(cfl), ctypes.byref(lam))
        return dt, lam.value

    def norms(self, Q, Qref=None):
        Q = _f64(Q)
        out = np.zeros(7)
        ref = _ptr(_f64(Qref)) if Qref is not None else None
        st = self.lib.dgo_norms(ctypes.byref(self._m), _ptr(Q), ref, _ptr(out))
        if st:
            raise RuntimeError("oracle norms failed")
        return out

    # --- z slabs: the mesh is one slab of a taller box; its z neighbours
    # beyond its own layers enter through halo traces [5][ny*nx][N*N]

    @property
    def halo_shape(self):
        return (NF, self.nx * self.ny, self.N * self.N)

    def ztraces(self, Q):
        """(lo, hi): the traces of layer 0 at its -z end and of the last layer
        at its +z end, in the halo layout."""
        Q = _f64(Q)
        lo, hi = np.empty(self.halo_shape), np.empty(self.halo_shape)
        if self.lib.dgo_ztraces(ctypes.byref(self._m), _ptr(Q), _ptr(lo), _ptr(hi)):
            raise RuntimeError("oracle ztraces failed")
        return lo, hi

    def rhs_zhalo(self, Q, halo_lo, halo_hi):
        """O2 right-hand side with the z neighbours' traces taken from the halos."""
        Q = _f64(Q)
        R = np.empty_like(Q)
        lo, hi = _f64(halo_lo), _f64(halo_hi)
        if self.lib.dgo_rhs_o2_zhalo(ctypes.byref(self._m), _ptr(Q), _ptr(lo), _ptr(hi), _ptr(R)):
            raise RuntimeError("oracle rhs_zhalo failed")
        return R

    def rk_stage(self, Q, dQ, dt, stage, halo_lo=None, halo_hi=None):
        """LSERK45 stage `stage` (0..4) in place on the float64 arrays Q, dQ."""
        assert Q.dtype == np.float64 and dQ.dtype == np.float64
        assert Q.flags.c_contiguous and dQ.flags.c_contiguous
        lo = None if halo_lo is None else _ptr(_f64(halo_lo))
        hi = None if halo_hi is None else _ptr(_f64(halo_hi))
        if self.lib.dgo_rk_stage(ctypes.byref(self._m), _ptr(Q), _ptr(dQ), float(dt), int(stage),
                                 lo, hi):
            raise RuntimeError("oracle rk_stage failed")

    def init(self, kind, params):
        kinds = {"uniform": 0, "vortex": 1, "tgv": 2}
        k = kinds[kind] if isinstance(kind, str) else int(kind)
        pr = _f64(np.asarray(params, dtype=np.float64))
        Q = self.zeros()
        st = self.lib.dgo_state_init(ctypes.byref(self._m), k, _ptr(pr), len(pr), _ptr(Q))
        if st:
            raise RuntimeError("oracle init failed")
        return Q


def gl_nodes(N, lib=None):
    lib = lib or load()
    xi = np.zeros(N)
    w = np.zeros(N)
    if lib.dgo_gl_nodes(N, _ptr(xi), _ptr(w)):
        raise ValueError("unsupported N")
    return xi, w


def lagrange(N, xi, s, x, lib=None):
    lib = lib or load()
    xi = _f64(xi)
    return lib.dgo_lagrange(N, _ptr(xi), s, float(x))


def lagrange_deriv(N, xi, s, x, lib=None):
    lib = lib or load()
    xi = _f64(xi)
    return lib.dgo_lagrange_deriv(N, _ptr(xi), s, float(x))


def flux(d, q, gamma=1.4, lib=None):
    lib = lib or load()
    q = _f64(q)
    f = np.zeros(NF)
    lib.dgo_flux(d, _ptr(q), gamma, _ptr(f))
    return f


def lf_flux(d, qL, qR, gamma=1.4, lib=None):
    lib = lib or load()
    qL, qR = _f64(qL), _f64(qR)
    f = np.zeros(NF)
    lib.dgo_lf_flux(d, _ptr(qL), _ptr(qR), gamma, _ptr(f))
    return f


def lserk_coeffs(lib=None):
    lib = lib or load()
    A = np.zeros(5)
    B = np.zeros(5)
    lib.dgo_lserk_coeffs(_ptr(A), _ptr(B))
    return A, B


def lserk_ode(y0, fun, dt, nsteps, lib=None):
    """Integrate y' = fun(y) with the oracle's LSERK45 stepper."""
    lib = lib or load()
    y = _f64(np.array(y0, dtype=np.float64)).copy()
    n = y.size

    def cb(nn, yp, fp):
        yy = np.ctypeslib.as_array(yp, shape=(nn,))
        ff = np.ctypeslib.as_array(fp, shape=(nn,))
        ff[:] = fun(yy.copy())
        return 0

    c = _ODE_CB(cb)
    st = lib.dgo_lserk_ode(n, _ptr(y), int(nsteps), float(dt), c)
    if st:
        raise RuntimeError("oracle ode failed")
    return y


def num_threads(lib=None):
    return (lib or load()).dgo_num_threads()


def set_num_threads(n, lib=None):
    (lib or load()).dgo_set_num_threads(int(n))
