"""ctypes binding of the C ABI in include/dg.h (argument marshalling only).

Every step of the computation runs in the CUDA library
``paper_2006_15698_gb300/lib/libdg_gb300.so``; this module only turns torch
tensors into device pointers and the current torch stream into the
``stream`` argument.  Importing it raises if the library has not been built
(``python -c "import __graft_entry__ as g; g.build()"``): there is no CPU
fallback.

The functions named ``dg_*`` mirror the C entry points one to one; ``Mesh``
is a small convenience wrapper over them.
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libdg_gb300.so")

DG_OK, DG_ERR_ARG, DG_ERR_UNSUPPORTED, DG_ERR_OOM, DG_ERR_CUDA, DG_ERR_NONFINITE, \
    DG_ERR_BOUNDS, DG_ERR_TIMEOUT = range(8)
DG_FP64, DG_FP32 = 0, 1
DG_INIT_UNIFORM, DG_INIT_VORTEX, DG_INIT_TGV = 0, 1, 2
DG_MAX_P = 6
DG_NORMS_LEN = 7
NF = 5

if not os.path.exists(LIB_PATH):
    raise ImportError(f"CUDA library not built: {LIB_PATH} is missing "
                      "(run paper_2006_15698_gb300/build.py or __graft_entry__.build())")

_lib = ctypes.CDLL(LIB_PATH)
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_szp = ctypes.POINTER(ctypes.c_size_t)

_lib.dg_mesh_create.argtypes = [ctypes.c_int] * 4 + [ctypes.c_double] * 7 + [
    ctypes.c_int, ctypes.POINTER(_vp)]
_lib.dg_mesh_create.restype = ctypes.c_int
_lib.dg_mesh_destroy.argtypes = [_vp]
_lib.dg_mesh_destroy.restype = None
_lib.dg_mesh_sizes.argtypes = [_vp, _i64p, _i64p, _szp, _szp]
_lib.dg_mesh_sizes.restype = ctypes.c_int
_lib.dg_state_init.argtypes = [_vp, ctypes.c_int, _dp, ctypes.c_int, _vp, _vp]
_lib.dg_state_init.restype = ctypes.c_int
_lib.dg_rhs.argtypes = [_vp, _vp, _vp, _vp]
_lib.dg_rhs.restype = ctypes.c_int
_lib.dg_cfl_dt.argtypes = [_vp, _vp, ctypes.c_double, _vp, _vp]
_lib.dg_cfl_dt.restype = ctypes.c_int
_lib.dg_rk_step.argtypes = [_vp, _vp, _vp, _vp, _vp]
_lib.dg_rk_step.restype = ctypes.c_int
_lib.dg_norms.argtypes = [_vp, _vp, _vp, _vp, _vp]
_lib.dg_norms.restype = ctypes.c_int
_lib.dg_advance.argtypes = [_vp, _vp, _vp, ctypes.c_double, ctypes.c_int, _vp, _vp, _vp]
_lib.dg_advance.restype = ctypes.c_int
_lib.dg_advance_host.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_double, ctypes.c_int, _vp, _vp, _vp]
_lib.dg_advance_host.restype = ctypes.c_int
_lib.dg_rk_stage.argtypes = [_vp, _vp, _vp, _vp, _vp, ctypes.c_int, _vp]
_lib.dg_rk_stage.restype = ctypes.c_int
_lib.dg_mesh_set_zhalo.argtypes = [_vp, _vp, _vp]
_lib.dg_mesh_set_zhalo.restype = ctypes.c_int
_lib.dg_zhalo_traces.argtypes = [_vp, _vp, _vp, _vp, _vp]
_lib.dg_zhalo_traces.restype = ctypes.c_int
_lib.dg_status_string.argtypes = [ctypes.c_int]
_lib.dg_status_string.restype = ctypes.c_char_p
_lib.dg_last_error.argtypes = [_vp]
_lib.dg_last_error.restype = ctypes.c_int
_lib.dg_profile_begin.argtypes = [_vp]
_lib.dg_profile_begin.restype = ctypes.c_int
_lib.dg_profile_end.argtypes = [_vp, _dp, _i64p]
_lib.dg_profile_end.restype = ctypes.c_int

_lib.dg_rhs_static.argtypes = [ctypes.c_int] * 4 + [ctypes.c_double] * 7 + [
    ctypes.c_int, _vp, _vp, _vp]
_lib.dg_rhs_static.restype = ctypes.c_int

_lib.dg_tile_variant_count.argtypes = [ctypes.c_int]
_lib.dg_tile_variant_count.restype = ctypes.c_int
_lib.dg_tile_shape.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                               ctypes.POINTER(ctypes.c_int)]
_lib.dg_tile_shape.restype = ctypes.c_int
_lib.dg_set_tile_variant.argtypes = [ctypes.c_int, ctypes.c_int]
_lib.dg_set_tile_variant.restype = ctypes.c_int
_lib.dg_get_tile_variant.argtypes = [ctypes.c_int]
_lib.dg_get_tile_variant.restype = ctypes.c_int
_lib.dg_set_stage_kernel.argtypes = [ctypes.c_int, ctypes.c_int]
_lib.dg_set_stage_kernel.restype = ctypes.c_int
_lib.dg_get_stage_kernel.argtypes = [ctypes.c_int]
_lib.dg_get_stage_kernel.restype = ctypes.c_int


class DgInstance(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("p", ctypes.c_int),
                ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("z0", ctypes.c_double),
                ("Lx", ctypes.c_double), ("Ly", ctypes.c_double), ("Lz", ctypes.c_double),
                ("gamma", ctypes.c_double), ("Q", ctypes.c_void_p), ("dQ", ctypes.c_void_p),
                ("Qt", ctypes.c_void_p)]


_lib.dg_batch_create.argtypes = [ctypes.c_int, ctypes.POINTER(DgInstance), ctypes.POINTER(_vp)]
_lib.dg_batch_create.restype = ctypes.c_int
_lib.dg_batch_destroy.argtypes = [_vp]
_lib.dg_batch_destroy.restype = None
_lib.dg_batch_update.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(DgInstance)]
_lib.dg_batch_update.restype = ctypes.c_int
_lib.dg_set_batch_direct_nodes.argtypes = [ctypes.c_int64]
_lib.dg_set_batch_direct_nodes.restype = ctypes.c_int
_lib.dg_get_batch_direct_nodes.argtypes = []
_lib.dg_get_batch_direct_nodes.restype = ctypes.c_int64
_lib.dg_batch_sizes.argtypes = [_vp, _i64p, _i64p]
_lib.dg_batch_sizes.restype = ctypes.c_int
_lib.dg_batch_state_init.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _vp]
_lib.dg_batch_state_init.restype = ctypes.c_int
_lib.dg_batch_step.argtypes = [_vp, ctypes.c_double, ctypes.c_int, ctypes.c_int, _vp]
_lib.dg_batch_step.restype = ctypes.c_int
_lib.dg_batch_dt.argtypes = [_vp, _dp]
_lib.dg_batch_dt.restype = ctypes.c_int
_lib.dg_batch_norms.argtypes = [_vp, ctypes.c_int, _vp, _vp, _vp]
_lib.dg_batch_norms.restype = ctypes.c_int
_lib.dg_batch_last_error.argtypes = [_vp]
_lib.dg_batch_last_error.restype = ctypes.c_int

_lib.dg_fma_throughput.argtypes = [ctypes.c_int, _dp, _dp]
_lib.dg_fma_throughput.restype = ctypes.c_int


def dg_fma_throughput(precision):
    """(flop/s, ms of the timed launch) of independent FMA chains on the
    current device at the given precision (the roofline denominator of the
    arithmetic-bound kernels)."""
    f, ms = ctypes.c_double(), ctypes.c_double()
    _check(_lib.dg_fma_throughput(precision, ctypes.byref(f), ctypes.byref(ms)),
           "dg_fma_throughput")
    return f.value, ms.value


_lib.dg_dmma_throughput.argtypes = [ctypes.c_int, _dp, _dp]
_lib.dg_dmma_throughput.restype = ctypes.c_int


def dg_dmma_throughput(mix=False):
    """(flop/s, ms) of FP64 mma.sync m8n8k4 chains on the current device
    (mix: odd warps run FP64 FMA chains of the same flop count instead)."""
    f, ms = ctypes.c_double(), ctypes.c_double()
    _check(_lib.dg_dmma_throughput(1 if mix else 0, ctypes.byref(f), ctypes.byref(ms)),
           "dg_dmma_throughput")
    return f.value, ms.value


_lib.dg_selfcheck_sqrt.argtypes = [_vp, _vp, _vp, ctypes.c_int64, _vp]
_lib.dg_selfcheck_sqrt.restype = ctypes.c_int


def dg_selfcheck_sqrt(a, stream=None):
    """(fast, ieee): the double kernels' sound-speed root and CUDA's sqrt of
    the positive float64 CUDA tensor a."""
    if a.dtype != torch.float64 or not a.is_cuda or not a.is_contiguous():
        raise ValueError("a must be a contiguous float64 CUDA tensor")
    fast, ieee = torch.empty_like(a), torch.empty_like(a)
    _check(_lib.dg_selfcheck_sqrt(_ptr(a), _ptr(fast), _ptr(ieee), a.numel(), _stream(stream)),
           "dg_selfcheck_sqrt")
    return fast, ieee


DG_PROFILE_KINDS = 8
KERNEL_KINDS = ("face", "volume", "cfl", "norms", "init", "stage", "copy", "epilogue")
DG_ERR_TOO_LARGE = 8
DG_STATIC_SCRATCH_BYTES = 16 * 1024 * 1024


class DGError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {dg_status_string(status)} ({status})")


def _check(st, where):
    if st != DG_OK:
        raise DGError(st, where)


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


# --- one-to-one mirrors of the C entry points ------------------------------

def dg_mesh_create(nx, ny, nz, p, x0, y0, z0, Lx, Ly, Lz, gamma, precision):
    h = _vp()
    _check(_lib.dg_mesh_create(nx, ny, nz, p, x0, y0, z0, Lx, Ly, Lz, gamma, precision,
                               ctypes.byref(h)), "dg_mesh_create")
    return h


def dg_mesh_destroy(h):
    _lib.dg_mesh_destroy(h)


def dg_mesh_sizes(h):
    a, b = ctypes.c_int64(), ctypes.c_int64()
    c, d = ctypes.c_size_t(), ctypes.c_size_t()
    _check(_lib.dg_mesh_sizes(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                              ctypes.byref(d)), "dg_mesh_sizes")
    return a.value, b.value, c.value, d.value


def dg_state_init(h, kind, params, Q, stream=None):
    arr = (ctypes.c_double * len(params))(*[float(x) for x in params])
    _check(_lib.dg_state_init(h, kind, arr, len(params), _ptr(Q), _stream(stream)),
           "dg_state_init")


def dg_rhs(h, Q, R, stream=None):
    _check(_lib.dg_rhs(h, _ptr(Q), _ptr(R), _stream(stream)), "dg_rhs")


def dg_cfl_dt(h, Q, cfl, dt_dev, stream=None):
    _check(_lib.dg_cfl_dt(h, _ptr(Q), float(cfl), _ptr(dt_dev), _stream(stream)), "dg_cfl_dt")


def dg_rk_step(h, Q, dQ, dt_dev, stream=None):
    _check(_lib.dg_rk_step(h, _ptr(Q), _ptr(dQ), _ptr(dt_dev), _stream(stream)), "dg_rk_step")


def dg_norms(h, Q, Qref, out_dev, stream=None):
    _check(_lib.dg_norms(h, _ptr(Q), _ptr(Qref), _ptr(out_dev), _stream(stream)), "dg_norms")


def dg_advance(h, Q, dQ, cfl, nsteps, dts_dev, integ_dev, stream=None):
    _check(_lib.dg_advance(h, _ptr(Q), _ptr(dQ), cfl, nsteps, _ptr(dts_dev), _ptr(integ_dev),
                           _stream(stream)), "dg_advance")


def dg_advance_host(h, Q_host, Q, dQ, cfl, nsteps, dts_host, integ_host, stream=None):
    _check(_lib.dg_advance_host(h, _ptr(Q_host), _ptr(Q), _ptr(dQ), cfl, nsteps, _ptr(dts_host),
                                _ptr(integ_host), _stream(stream)), "dg_advance_host")


def dg_rk_stage(h, Qin, Qout, dQ, dt_dev, stage, stream=None):
    _check(_lib.dg_rk_stage(h, _ptr(Qin), _ptr(Qout), _ptr(dQ), _ptr(dt_dev), int(stage),
                            _stream(stream)), "dg_rk_stage")


def dg_mesh_set_zhalo(h, halo_lo, halo_hi):
    _check(_lib.dg_mesh_set_zhalo(h, _ptr(halo_lo), _ptr(halo_hi)), "dg_mesh_set_zhalo")


def dg_zhalo_traces(h, Q, send_lo, send_hi, stream=None):
    _check(_lib.dg_zhalo_traces(h, _ptr(Q), _ptr(send_lo), _ptr(send_hi), _stream(stream)),
           "dg_zhalo_traces")


def dg_status_string(st):
    return _lib.dg_status_string(st).decode()


def dg_last_error(h):
    return _lib.dg_last_error(h)


def dg_rhs_static(nx, ny, nz, p, x0, y0, z0, Lx, Ly, Lz, gamma, precision, Q, R, stream=None):
    """Allocation-free right-hand side (no mesh handle; the double form's
    scratch is a static device array, see include/dg.h).  For callers that
    cannot let a library allocate device memory.

    The C function cannot see the size of Q and R, so they are checked here
    before the call: torch tensors on the current CUDA device, contiguous, of
    the precision's dtype and exactly 5 nx ny nz (p+1)^3 elements (when the
    mesh arguments are in range; otherwise the library rejects them)."""
    dtype = {DG_FP64: torch.float64, DG_FP32: torch.float32}.get(precision)
    for name, t in (("Q", Q), ("R", R)):
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"dg_rhs_static: {name} must be a torch tensor")
        if not t.is_cuda or t.device.index != torch.cuda.current_device():
            raise ValueError(f"dg_rhs_static: {name} must be on the current CUDA device")
        if not t.is_contiguous():
            raise ValueError(f"dg_rhs_static: {name} must be contiguous")
        if dtype is not None and t.dtype != dtype:
            raise ValueError(f"dg_rhs_static: {name} must be {dtype} for this precision")
        if min(nx, ny, nz) >= 1 and 0 <= p <= DG_MAX_P:
            need = NF * nx * ny * nz * (p + 1) ** 3
            if t.numel() != need:
                raise ValueError(f"dg_rhs_static: {name} has {t.numel()} elements, "
                                 f"the mesh needs {need}")
    _check(_lib.dg_rhs_static(nx, ny, nz, p, x0, y0, z0, Lx, Ly, Lz, gamma, precision,
                              _ptr(Q), _ptr(R), _stream(stream)), "dg_rhs_static")


def dg_profile_begin(h):
    _check(_lib.dg_profile_begin(h), "dg_profile_begin")


def dg_profile_end(h):
    ms = (ctypes.c_double * DG_PROFILE_KINDS)()
    n = (ctypes.c_int64 * DG_PROFILE_KINDS)()
    _check(_lib.dg_profile_end(h, ms, n), "dg_profile_end")
    return {k: (ms[i], n[i]) for i, k in enumerate(KERNEL_KINDS)}


# --- convenience wrapper ---------------------------------------------------

class Mesh:
    """A periodic Cartesian mesh handle; states are torch tensors on the GPU
    with shape (5, elements, N, N, N) (the ABI layout), dtype float64 for
    DG_FP64 and float32 for DG_FP32."""

    def __init__(self, nx, ny, nz, p, x0=0.0, y0=0.0, z0=0.0, Lx=1.0, Ly=1.0, Lz=1.0,
                 gamma=1.4, precision=DG_FP64, device=None):
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        with torch.cuda.device(self.device):
            self.h = dg_mesh_create(nx, ny, nz, p, x0, y0, z0, Lx, Ly, Lz, gamma, precision)
        self.nx, self.ny, self.nz, self.p = nx, ny, nz, p
        # the arguments that recreate this mesh (checkpoint.py)
        self.spec = dict(nx=nx, ny=ny, nz=nz, p=p, x0=x0, y0=y0, z0=z0, Lx=Lx, Ly=Ly, Lz=Lz,
                         gamma=gamma, precision=precision)
        self.N = p + 1
        self.E = nx * ny * nz
        self.precision = precision
        self.dtype = torch.float64 if precision == DG_FP64 else torch.float32
        self.n_dof, self.n_unknowns, self.state_bytes, self.workspace_bytes = dg_mesh_sizes(self.h)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            dg_mesh_destroy(h)
            self.h = None

    @property
    def shape(self):
        return (NF, self.E, self.N, self.N, self.N)

    def empty(self):
        return torch.empty(self.shape, dtype=self.dtype, device=self.device)

    def _chk(self, t):
        if (t.dtype != self.dtype or not t.is_cuda or not t.is_contiguous()
                or (tuple(t.shape) != self.shape and t.numel() != NF * self.n_dof)):
            raise ValueError("state tensor must be a contiguous CUDA tensor of the mesh's "
                             f"shape {self.shape} and dtype {self.dtype}")
        return t

    def init(self, kind, params, Q=None, stream=None):
        kinds = {"uniform": DG_INIT_UNIFORM, "vortex": DG_INIT_VORTEX, "tgv": DG_INIT_TGV}
        Q = self.empty() if Q is None else self._chk(Q)
        dg_state_init(self.h, kinds.get(kind, kind), params, Q, stream)
        return Q

    def rhs(self, Q, R=None, stream=None):
        R = self.empty() if R is None else self._chk(R)
        dg_rhs(self.h, self._chk(Q), R, stream)
        return R

    def cfl_dt(self, Q, cfl, dt=None, stream=None):
        dt = torch.empty(1, dtype=torch.float64, device=self.device) if dt is None else dt
        dg_cfl_dt(self.h, self._chk(Q), cfl, dt, stream)
        return dt

    def rk_step(self, Q, dQ, dt, stream=None):
        dg_rk_step(self.h, self._chk(Q), self._chk(dQ), dt, stream)

    def norms(self, Q, Qref=None, out=None, stream=None):
        out = torch.empty(DG_NORMS_LEN, dtype=torch.float64, device=self.device) if out is None else out
        dg_norms(self.h, self._chk(Q), None if Qref is None else self._chk(Qref), out, stream)
        return out

    def advance(self, Q, dQ, cfl, nsteps, dts=None, integ=None, with_integrals=True, stream=None):
        """nsteps x (time step, LSERK45 step, integrals of the new state) in
        one call; returns (dts, integ): device arrays of nsteps and
        (nsteps, DG_NORMS_LEN) doubles (integ None when not requested)."""
        if dts is None:
            dts = torch.empty(nsteps, dtype=torch.float64, device=self.device)
        if integ is None and with_integrals:
            integ = torch.empty((nsteps, DG_NORMS_LEN), dtype=torch.float64, device=self.device)
        dg_advance(self.h, self._chk(Q), self._chk(dQ), cfl, nsteps, dts, integ, stream)
        return dts, integ

    def advance_host(self, Q_host, Q, dQ, cfl, nsteps, dts=None, integ=None, with_integrals=True,
                     stream=None):
        """advance() on a state held in host memory (dg_advance_host):
        Q_host (a contiguous CPU tensor of the state, pinned for full copy
        bandwidth) is copied to the device state Q, stepped, and copied
        back; returns (dts, integ) as host tensors.  Synchronises."""
        if (Q_host.dtype != self.dtype or Q_host.is_cuda or not Q_host.is_contiguous()
                or Q_host.numel() != NF * self.n_dof):
            raise ValueError("host state must be a contiguous CPU tensor of the mesh's "
                             f"shape {self.shape} and dtype {self.dtype}")
        if dts is None:
            dts = torch.empty(nsteps, dtype=torch.float64, pin_memory=True)
        if integ is None and with_integrals:
            integ = torch.empty((nsteps, DG_NORMS_LEN), dtype=torch.float64, pin_memory=True)
        for t in (dts, integ):
            if t is not None and (t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous()):
                raise ValueError("dts / integ must be contiguous float64 CPU tensors")
        if dts.numel() < nsteps or (integ is not None and integ.numel() < nsteps * DG_NORMS_LEN):
            raise ValueError("dts / integ too small for nsteps")
        dg_advance_host(self.h, Q_host, self._chk(Q), self._chk(dQ), cfl, nsteps, dts, integ, stream)
        return dts, integ

    def rk_stage(self, Qin, Qout, dQ, dt, stage, stream=None):
        """LSERK45 stage `stage` (0..4): dQ <- A dQ + dt R(Qin), Qout <- Qin + B dQ."""
        dg_rk_stage(self.h, self._chk(Qin), self._chk(Qout), self._chk(dQ), dt, stage, stream)

    # --- z slabs -----------------------------------------------------------
    @property
    def halo_shape(self):
        """Shape of a halo / trace buffer: (5, nx*ny, N*N)."""
        return (NF, self.nx * self.ny, self.N * self.N)

    def empty_halo(self):
        return torch.empty(self.halo_shape, dtype=self.dtype, device=self.device)

    def _chk_halo(self, t):
        if (t.dtype != self.dtype or not t.is_cuda or not t.is_contiguous()
                or t.numel() != NF * self.nx * self.ny * self.N * self.N):
            raise ValueError(f"halo tensor must be a contiguous CUDA tensor of {self.halo_shape} "
                             f"and dtype {self.dtype}")
        return t

    def set_zhalo(self, halo_lo, halo_hi):
        """Make the z boundary an interface to other slabs whose traces the
        two halo tensors hold (kept by reference; None, None: periodic)."""
        if halo_lo is None and halo_hi is None:
            dg_mesh_set_zhalo(self.h, None, None)
            self._halos = None
            return
        dg_mesh_set_zhalo(self.h, self._chk_halo(halo_lo), self._chk_halo(halo_hi))
        self._halos = (halo_lo, halo_hi)  # the library keeps the pointers

    def ztraces(self, Q, send_lo=None, send_hi=None, stream=None):
        """(send_lo, send_hi): layer 0's -z-end and the last layer's +z-end traces."""
        send_lo = self.empty_halo() if send_lo is None else self._chk_halo(send_lo)
        send_hi = self.empty_halo() if send_hi is None else self._chk_halo(send_hi)
        dg_zhalo_traces(self.h, self._chk(Q), send_lo, send_hi, stream)
        return send_lo, send_hi

    def last_error(self):
        return dg_last_error(self.h)

    def profile_begin(self):
        dg_profile_begin(self.h)

    def profile_end(self):
        """{kind: (summed device ms, launches)} since profile_begin."""
        return dg_profile_end(self.h)


# --- tile-shape tuning table of the float form ------------------------------

def dg_tile_variant_count(p):
    return _lib.dg_tile_variant_count(p)


def dg_tile_shape(p, variant):
    tx, ty = ctypes.c_int(), ctypes.c_int()
    _check(_lib.dg_tile_shape(p, variant, ctypes.byref(tx), ctypes.byref(ty)), "dg_tile_shape")
    return tx.value, ty.value


def dg_set_tile_variant(p, variant):
    _check(_lib.dg_set_tile_variant(p, variant), "dg_set_tile_variant")


def dg_get_tile_variant(p):
    return _lib.dg_get_tile_variant(p)


DG_STAGE_TILE, DG_STAGE_COLUMN, DG_STAGE_LINES = 0, 1, 2
STAGE_KINDS = {"tile": DG_STAGE_TILE, "column": DG_STAGE_COLUMN, "lines": DG_STAGE_LINES}


def dg_set_stage_kernel(p, kind):
    _check(_lib.dg_set_stage_kernel(p, kind), "dg_set_stage_kernel")


def dg_get_stage_kernel(p):
    return _lib.dg_get_stage_kernel(p)


BATCH_NEVER_DIRECT = 2 ** 63 - 1


def dg_set_batch_direct_nodes(nodes):
    """Batches created afterwards give instances of at least `nodes` nodes
    their own stage launches (0: all of them; BATCH_NEVER_DIRECT: none)."""
    _check(_lib.dg_set_batch_direct_nodes(int(nodes)), "dg_set_batch_direct_nodes")


def dg_get_batch_direct_nodes():
    return _lib.dg_get_batch_direct_nodes()


TUNING_PATH = os.path.join(_HERE, "tuning", "fused_tiles.json")


def load_tuning(path=None):
    """Select the tile variant and the single-mesh stage kernel per degree
    from an autotuner table (JSON with "variant" and optionally "kernel"
    ("tile", "column" or "lines") entries per degree); returns the table, or
    None if absent."""
    import json
    path = path or TUNING_PATH
    if not os.path.exists(path):
        return None
    with open(path) as f:
        table = json.load(f)
    for p, ent in table.get("degrees", {}).items():
        v = int(ent["variant"])
        if 0 <= v < dg_tile_variant_count(int(p)):
            dg_set_tile_variant(int(p), v)
        kind = ent.get("kernel")
        if kind in STAGE_KINDS:
            dg_set_stage_kernel(int(p), STAGE_KINDS[kind])
    return table


# --- batches of independent float meshes ------------------------------------

def state_shape(spec):
    """Shape (5, elements, N, N, N) of an instance's state."""
    N = spec["p"] + 1
    return (NF, spec["nx"] * spec["ny"] * spec["nz"], N, N, N)


class Batch:
    """Independent DG_FP32 meshes advanced together (dg_batch_*).

    specs: list of dicts with nx, ny, nz, p and optionally x0..Lz, gamma, and
    optionally the instance's float tensors "Q", "dQ", "Qt" (else allocated
    here).  The tensors are caller-owned memory as far as the library is
    concerned; this object keeps references to them."""

    def __init__(self, specs, device=None):
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        arr = self._instances(specs)
        h = _vp()
        with torch.cuda.device(self.device):
            _check(_lib.dg_batch_create(len(specs), arr, ctypes.byref(h)), "dg_batch_create")
        self.h = h
        self._sizes()

    def update(self, specs):
        """Replace the instance list in place (dg_batch_update); the batch must
        be idle (its enqueued steps complete)."""
        arr = self._instances(specs)
        with torch.cuda.device(self.device):
            _check(_lib.dg_batch_update(self.h, len(specs), arr), "dg_batch_update")
        self._sizes()

    def _sizes(self):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(_lib.dg_batch_sizes(self.h, ctypes.byref(a), ctypes.byref(b)), "dg_batch_sizes")
        self.n_dof, self.n_items = a.value, b.value

    def _instances(self, specs):
        self.specs = [dict(s) for s in specs]
        self.Q, self.dQ, self.Qt = [], [], []
        arr = (DgInstance * len(specs))()
        for i, s in enumerate(self.specs):
            q = s.get("Q")
            if q is None:
                q = torch.empty(state_shape(s), dtype=torch.float32, device=self.device)
            dq = s.get("dQ")
            if dq is None:
                dq = torch.zeros_like(q)
            qt = s.get("Qt")
            self.Q.append(q)
            self.dQ.append(dq)
            self.Qt.append(qt)
            arr[i] = DgInstance(s["nx"], s["ny"], s["nz"], s["p"], s.get("x0", 0.0), s.get("y0", 0.0),
                                s.get("z0", 0.0), s.get("Lx", 1.0), s.get("Ly", 1.0), s.get("Lz", 1.0),
                                s.get("gamma", 1.4), q.data_ptr(), dq.data_ptr(),
                                None if qt is None else qt.data_ptr())
        return arr

    def __len__(self):
        return len(self.specs)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            _lib.dg_batch_destroy(h)
            self.h = None

    def init(self, idx, kind, params, stream=None):
        kinds = {"uniform": DG_INIT_UNIFORM, "vortex": DG_INIT_VORTEX, "tgv": DG_INIT_TGV}
        arr = (ctypes.c_double * len(params))(*[float(x) for x in params])
        _check(_lib.dg_batch_state_init(self.h, idx, kinds.get(kind, kind), arr, len(params),
                                        _stream(stream)), "dg_batch_state_init")

    def step(self, cfl, nsteps=1, use_graph=True, stream=None):
        """Advance every instance by nsteps LSERK45 steps (each with its own CFL dt)."""
        _check(_lib.dg_batch_step(self.h, float(cfl), int(nsteps), 1 if use_graph else 0,
                                  _stream(stream)), "dg_batch_step")

    def dts(self):
        out = (ctypes.c_double * len(self.specs))()
        _check(_lib.dg_batch_dt(self.h, out), "dg_batch_dt")
        return list(out)

    def norms(self, idx, Qref=None, out=None, stream=None):
        out = torch.empty(DG_NORMS_LEN, dtype=torch.float64, device=self.device) if out is None else out
        _check(_lib.dg_batch_norms(self.h, idx, _ptr(Qref), _ptr(out), _stream(stream)),
               "dg_batch_norms")
        return out

    def last_error(self):
        return _lib.dg_batch_last_error(self.h)
