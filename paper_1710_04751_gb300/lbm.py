"""Python binding of the C ABI in include/lbm.h (argument marshalling only).

Every step of the method runs in the CUDA library liblbm.so (built in-tree by
paper_1710_04751_gb300/build.py).  PyTorch only supplies device memory (the state
arena) and the CUDA stream.  There is no CPU fallback: without the library or a GPU
the constructor raises.
"""
import ctypes
import math
import os

import numpy as np

from . import build as _build

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EDIVERGED, LBM_ETIMEOUT = 0, -1, -2, -3, -4, -5
D3Q15, D3Q7 = 15, 7
FP64, FP32, FP16_DEV, BF16_DEV = 0, 1, 2, 3
BC_CAVITY, BC_XWALLS, BC_PERIODIC, BC_ADIABATIC_BOX = 0, 6, 7, 8
ADIABATIC_BOUNCE_BACK, ADIABATIC_SPECULAR = 0, 1

# Every entry point include/lbm.h declares (checked by tests/test_abi.py).
EXPORTS = (
    "lbm_default_options", "lbm_derive_params", "lbm_arena_bytes", "lbm_create",
    "lbm_create_params", "lbm_step", "lbm_fields", "lbm_nusselt", "lbm_residual",
    "lbm_get_populations", "lbm_set_populations", "lbm_get_params", "lbm_steps_done",
    "lbm_last_error", "lbm_synchronize", "lbm_destroy", "lbm_nusselt_noalloc", "lbm_set_fields",
    "lbm_init_fields", "lbm_save", "lbm_checkpoint_info", "lbm_restore",
    "lbm_get_populations_native", "lbm_set_populations_native", "lbm_set_timeout",
)


class LBMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (code {code})")
        self.code = code


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int)]


class Params(ctypes.Structure):
    _fields_ = [
        ("omega_f", ctypes.c_double * 15), ("omega_g", ctypes.c_double * 15),
        ("gbeta", ctypes.c_double), ("T_hot", ctypes.c_double), ("T_cold", ctypes.c_double),
        ("cs2_phi", ctypes.c_double), ("ext_force", ctypes.c_double * 3), ("U0", ctypes.c_double),
        ("heat_source", ctypes.c_double),
        ("e4_mode", ctypes.c_int), ("adiabatic_mode", ctypes.c_int), ("boundary", ctypes.c_int),
    ]

    def as_dict(self):
        return dict(omega_f=list(self.omega_f), omega_g=list(self.omega_g), gbeta=self.gbeta,
                    T_hot=self.T_hot, T_cold=self.T_cold, cs2_phi=self.cs2_phi,
                    ext_force=list(self.ext_force), U0=self.U0, heat_source=self.heat_source,
                    e4_mode=self.e4_mode,
                    adiabatic_mode=self.adiabatic_mode, boundary=self.boundary)


class Options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int), ("seed", ctypes.c_uint64), ("noise_amp", ctypes.c_double),
        ("cs2_phi", ctypes.c_double), ("e4_mode", ctypes.c_int), ("adiabatic_mode", ctypes.c_int),
        ("residual_interval", ctypes.c_int), ("cuda_stream", ctypes.c_void_p),
        ("device_arena", ctypes.c_void_p), ("device_arena_bytes", ctypes.c_size_t),
        ("timeout_s", ctypes.c_double),
    ]


class Nu(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "hot_wall_mean", "cold_wall_mean", "mid_mean", "mid_max", "mid_max_z", "mid_min",
        "mid_min_z", "umax", "umax_z", "wmax", "wmax_x")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


_lib = None
_D = ctypes.POINTER(ctypes.c_double)


def library_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load liblbm.so (building it when missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise LBMError(LBM_ECUDA, f"CUDA library not built: {path}")
    L = ctypes.CDLL(path)
    P = ctypes.POINTER
    L.lbm_default_options.argtypes = [P(Options)]
    L.lbm_default_options.restype = None
    L.lbm_derive_params.argtypes = [P(Grid), ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, P(Options), P(Params)]
    L.lbm_arena_bytes.argtypes = [P(Grid), ctypes.c_int, ctypes.c_int]
    L.lbm_arena_bytes.restype = ctypes.c_size_t
    L.lbm_create.argtypes = [P(Grid), ctypes.c_int, ctypes.c_double, ctypes.c_double,
                             ctypes.c_double, P(Options), P(ctypes.c_void_p)]
    L.lbm_create_params.argtypes = [P(Grid), ctypes.c_int, P(Params), P(Options),
                                    P(ctypes.c_void_p)]
    L.lbm_step.argtypes = [ctypes.c_void_p, ctypes.c_int64]
    L.lbm_fields.argtypes = [ctypes.c_void_p] + [_D] * 5
    L.lbm_nusselt.argtypes = [ctypes.c_void_p, P(Nu)]
    L.lbm_residual.argtypes = [ctypes.c_void_p, _D]
    L.lbm_get_populations.argtypes = [ctypes.c_void_p, _D, _D]
    L.lbm_set_populations.argtypes = [ctypes.c_void_p, _D, _D]
    L.lbm_get_params.argtypes = [ctypes.c_void_p, P(Params)]
    L.lbm_set_fields.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 5
    L.lbm_init_fields.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 5 + [ctypes.c_int]
    L.lbm_steps_done.argtypes = [ctypes.c_void_p]
    L.lbm_steps_done.restype = ctypes.c_int64
    L.lbm_last_error.argtypes = [ctypes.c_void_p]
    L.lbm_last_error.restype = ctypes.c_char_p
    L.lbm_synchronize.argtypes = [ctypes.c_void_p]
    L.lbm_set_timeout.argtypes = [ctypes.c_void_p, ctypes.c_double]
    L.lbm_destroy.argtypes = [ctypes.c_void_p]
    L.lbm_destroy.restype = None
    L.lbm_get_populations_native.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.lbm_set_populations_native.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.lbm_save.argtypes = [ctypes.c_void_p, ctypes.c_char_p]
    L.lbm_checkpoint_info.argtypes = [ctypes.c_char_p, P(Grid), P(ctypes.c_int), P(ctypes.c_int),
                                      P(Params), P(ctypes.c_int64)]
    L.lbm_restore.argtypes = [ctypes.c_void_p, ctypes.c_char_p]
    L.lbm_nusselt_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                      ctypes.c_int, P(Grid), ctypes.c_int, P(Params),
                                      ctypes.c_void_p, P(Nu)]
    _lib = L
    return L


def default_options():
    o = Options()
    load().lbm_default_options(ctypes.byref(o))
    return o


def derive_params(grid, lattice, Ra, Pr, Ma, **opts):
    """Host-only parameter derivation (Sec. 3): returns a Params structure."""
    L = load()
    o = default_options()
    for k, v in opts.items():
        setattr(o, k, v)
    p = Params()
    g = Grid(*grid)
    rc = L.lbm_derive_params(ctypes.byref(g), int(lattice), float(Ra), float(Pr), float(Ma),
                             ctypes.byref(o), ctypes.byref(p))
    if rc != LBM_OK:
        raise LBMError(rc, L.lbm_last_error(None).decode())
    return p


def checkpoint_info(path):
    """The header of a checkpoint file written by LBM.save: grid, lattice, precision,
    parameters (a dict, as LBM.params()) and step count."""
    L = load()
    g, lat, prec, p, steps = Grid(), ctypes.c_int(), ctypes.c_int(), Params(), ctypes.c_int64()
    rc = L.lbm_checkpoint_info(os.fsencode(path), ctypes.byref(g), ctypes.byref(lat), ctypes.byref(prec),
                               ctypes.byref(p), ctypes.byref(steps))
    if rc != LBM_OK:
        raise LBMError(rc, L.lbm_last_error(None).decode())
    return dict(grid=(g.nx, g.ny, g.nz), lattice=lat.value, precision=prec.value,
                params=p.as_dict(), steps=steps.value)


def arena_bytes(grid, lattice, precision):
    return int(load().lbm_arena_bytes(ctypes.byref(Grid(*grid)), int(lattice), int(precision)))


def _dp(a):
    return a.ctypes.data_as(_D)


def nusselt_noalloc(f_dev, g_dev, plane, precision, grid, lattice, params, stream=None):
    """lbm_nusselt for populations held in caller-owned device buffers (integer device
    addresses), without any allocation by the library.  params: a Params structure
    (e.g. from LBM.params_struct()).  stream: a cudaStream_t as an integer, or None."""
    L = load()
    nu = Nu()
    rc = L.lbm_nusselt_noalloc(ctypes.c_void_p(int(f_dev)), ctypes.c_void_p(int(g_dev)),
                               int(plane), int(precision), ctypes.byref(Grid(*grid)),
                               int(lattice), ctypes.byref(params),
                               ctypes.c_void_p(int(stream) if stream else None), ctypes.byref(nu))
    if rc != LBM_OK:
        raise LBMError(rc, L.lbm_last_error(None).decode())
    return nu.as_dict()


class LBM:
    """A cavity (or test box) advanced by the CUDA library on one GPU.

    grid: (nx, ny, nz).  Either (Ra, Pr, Ma) or an explicit `params` (Params or dict of
    Params fields) must be given.  cs2_phi = 0 selects the lattice default (1/3 for
    D3Q15, 1/4 for D3Q7).  The state arena is a torch CUDA tensor and the work
    runs on torch's current stream unless `stream` is given.
    """

    def __init__(self, grid, lattice=D3Q15, Ra=None, Pr=0.71, Ma=0.05 * math.sqrt(3.0),
                 params=None, precision=FP32, seed=1, noise_amp=1e-6, cs2_phi=0.0,
                 e4_mode=0, adiabatic_mode=ADIABATIC_SPECULAR, residual_interval=100,
                 stream=None, device=None, timeout_s=600.0, torch_arena=True):
        import torch

        if not torch.cuda.is_available():
            raise LBMError(LBM_ECUDA, "no CUDA device: the library has no CPU path")
        self._L = load()
        self._ctx = ctypes.c_void_p()
        self.grid = tuple(int(v) for v in grid)
        self.lattice = int(lattice)
        self.precision = int(precision)
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.device = dev
        o = Options()
        self._L.lbm_default_options(ctypes.byref(o))
        o.precision, o.seed, o.noise_amp = self.precision, int(seed) & (2**64 - 1), float(noise_amp)
        o.cs2_phi, o.e4_mode, o.adiabatic_mode = float(cs2_phi), int(e4_mode), int(adiabatic_mode)
        o.residual_interval, o.timeout_s = int(residual_interval), float(timeout_s)
        with torch.cuda.device(dev):
            self._stream = stream if stream is not None else torch.cuda.current_stream(dev)
            o.cuda_stream = self._stream.cuda_stream
            self._arena = None
            if torch_arena:
                nbytes = arena_bytes(self.grid, self.lattice, self.precision)
                # 256-byte aligned: torch's caching allocator returns 512-byte aligned blocks
                self._arena = torch.empty(nbytes, dtype=torch.uint8, device=dev)
                o.device_arena = self._arena.data_ptr()
                o.device_arena_bytes = nbytes
            g = Grid(*self.grid)
            if params is None:
                if Ra is None:
                    raise ValueError("give Ra (with Pr, Ma) or explicit params")
                rc = self._L.lbm_create(ctypes.byref(g), self.lattice, float(Ra), float(Pr),
                                        float(Ma), ctypes.byref(o), ctypes.byref(self._ctx))
            else:
                if isinstance(params, dict):
                    p = Params()
                    for k, v in params.items():
                        if isinstance(v, (list, tuple)):
                            arr = getattr(p, k)
                            for n, x in enumerate(v):
                                arr[n] = x
                        else:
                            setattr(p, k, v)
                    params = p
                rc = self._L.lbm_create_params(ctypes.byref(g), self.lattice, ctypes.byref(params),
                                               ctypes.byref(o), ctypes.byref(self._ctx))
            if rc != LBM_OK:
                raise LBMError(rc, self._L.lbm_last_error(None).decode())

    # -- helpers -------------------------------------------------------------------
    def _check(self, rc):
        if rc != LBM_OK:
            raise LBMError(rc, self._L.lbm_last_error(self._ctx).decode())

    @property
    def ncell(self):
        nx, ny, nz = self.grid
        return nx * ny * nz

    @property
    def handle(self):
        return self._ctx.value

    # -- the C ABI ---------------------------------------------------------------------
    def step(self, n=1):
        self._check(self._L.lbm_step(self._ctx, int(n)))

    def fields(self):
        nx, ny, nz = self.grid
        out = [np.empty((nz, ny, nx)) for _ in range(5)]
        self._check(self._L.lbm_fields(self._ctx, *[_dp(o) for o in out]))
        return dict(zip(("rho", "ux", "uy", "uz", "T"), out))

    def nusselt(self):
        nu = Nu()
        self._check(self._L.lbm_nusselt(self._ctx, ctypes.byref(nu)))
        return nu.as_dict()

    def residual(self):
        r = ctypes.c_double()
        self._check(self._L.lbm_residual(self._ctx, ctypes.byref(r)))
        return r.value

    def get_populations(self):
        nx, ny, nz = self.grid
        f = np.empty((15, nz, ny, nx))
        g = np.empty((self.lattice, nz, ny, nx))
        self._check(self._L.lbm_get_populations(self._ctx, _dp(f), _dp(g)))
        return f, g

    def set_populations(self, f, g):
        nx, ny, nz = self.grid
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(15, nz, ny, nx)
        g = np.ascontiguousarray(g, dtype=np.float64).reshape(self.lattice, nz, ny, nx)
        self._check(self._L.lbm_set_populations(self._ctx, _dp(f), _dp(g)))

    def _native_dtype(self):
        if self.precision not in (FP32, FP64):
            raise LBMError(LBM_EINVAL, "native transfers need an FP32 or FP64 context")
        return np.float32 if self.precision == FP32 else np.float64

    def get_populations_native(self, f=None, g=None):
        """The stored populations in the context's own precision (FP32 or FP64 contexts);
        f, g: optional preallocated C-contiguous arrays (e.g. page-locked) to fill."""
        nx, ny, nz = self.grid
        dt = self._native_dtype()
        f = np.empty((15, nz, ny, nx), dtype=dt) if f is None else f
        g = np.empty((self.lattice, nz, ny, nx), dtype=dt) if g is None else g
        for a, rows in ((f, 15), (g, self.lattice)):
            if a.dtype != dt or not a.flags.c_contiguous or a.size != rows * nx * ny * nz:
                raise ValueError("arrays must be C-contiguous, of the context's dtype and size")
        self._check(self._L.lbm_get_populations_native(self._ctx, f.ctypes.data, g.ctypes.data))
        return f, g

    def set_populations_native(self, f, g):
        """Upload populations in the context's own precision (no conversion pass)."""
        nx, ny, nz = self.grid
        dt = self._native_dtype()
        f = np.ascontiguousarray(f, dtype=dt).reshape(15, nz, ny, nx)
        g = np.ascontiguousarray(g, dtype=dt).reshape(self.lattice, nz, ny, nx)
        self._check(self._L.lbm_set_populations_native(self._ctx, f.ctypes.data, g.ctypes.data))

    def set_fields(self, ux, uy, uz, T, rho=None, iterations=0):
        """Populations at the equilibria of the fields: torch CUDA float64 tensors of
        shape (nz, ny, nx) on this context's device (rho None: 1); with iterations > 0
        followed by that many rounds of the consistent initialisation (lbm_init_fields)."""
        import torch
        arrs = [rho, ux, uy, uz, T]
        for a in arrs:
            if a is not None and (a.dtype != torch.float64 or not a.is_cuda or not a.is_contiguous()
                                  or a.numel() != self.ncell):
                raise ValueError("fields must be contiguous CUDA float64 tensors of ncell values")
        ptr = [ctypes.c_void_p(a.data_ptr()) if a is not None else None for a in arrs]
        self._check(self._L.lbm_init_fields(self._ctx, *ptr, int(iterations)))

    def save(self, path):
        """Write the state, parameters and step count to a checkpoint file (lbm_save)."""
        self._check(self._L.lbm_save(self._ctx, os.fsencode(path)))

    def restore(self, path):
        """Load the populations and step count of a checkpoint file of the same grid,
        lattice and precision (lbm_restore)."""
        self._check(self._L.lbm_restore(self._ctx, os.fsencode(path)))

    @classmethod
    def load(cls, path, **kw):
        """A context created from a checkpoint file: its grid, lattice, precision and
        parameters, then its populations and step count.  kw: further LBM options."""
        info = checkpoint_info(path)
        sim = cls(info["grid"], info["lattice"], params=info["params"], precision=info["precision"], **kw)
        sim.restore(path)
        return sim

    def params(self):
        return self.params_struct().as_dict()

    def params_struct(self):
        p = Params()
        self._check(self._L.lbm_get_params(self._ctx, ctypes.byref(p)))
        return p

    @property
    def steps_done(self):
        return int(self._L.lbm_steps_done(self._ctx))

    def synchronize(self):
        self._check(self._L.lbm_synchronize(self._ctx))

    def set_timeout(self, seconds):
        """Bound of every later host wait for the GPU (lbm_set_timeout)."""
        self._check(self._L.lbm_set_timeout(self._ctx, float(seconds)))

    @classmethod
    def _view(cls, handle, owner):
        """A member of a batch as an LBM object (not owned: the batch frees it)."""
        self = object.__new__(cls)
        self._L = load()
        self._ctx = ctypes.c_void_p(handle)
        self._owner = owner
        self.grid = tuple(owner._grids[owner._handles.index(handle)])
        self.lattice = owner.lattice
        self.precision = owner.precision
        self.device = owner.device
        self._stream = owner._stream
        self._arena = None
        return self

    def close(self):
        if getattr(self, "_owner", None) is not None:
            self._ctx = ctypes.c_void_p()
            self._owner = None
            return
        if getattr(self, "_ctx", None) is not None and self._ctx.value:
            self._L.lbm_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()
        self._arena = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
