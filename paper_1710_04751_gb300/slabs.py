"""Python binding of include/lbm_slabs.h (argument marshalling only): one cavity split
into z-slabs, each a context of its own with halo planes, exchanged after every step by
a copy kernel in liblbm.so.  The owned nodes follow the undivided grid's trajectory bit
for bit; the slabs share one GPU and one CUDA stream.

    python -m paper_1710_04751_gb300.slabs [--n 128] [--slabs 2] [--steps 1000] [--warmup 300]
        [--skip-undivided]

times the cavity (Ra = 1e5, Pr = 0.71, U0 = 0.05, D3Q15 + D3Q15, FP32) undivided and in
slabs with CUDA events and prints one JSON object.
"""
import argparse
import ctypes
import json
import math

import numpy as np

from . import lbm as _b
from .lbm import D3Q15, FP32, Grid, LBMError, LBM_OK, LBM_ECUDA, Options, Params, load

# Every entry point include/lbm_slabs.h declares (checked by tests/test_abi.py).
EXPORTS = (
    "lbm_slabs_plan", "lbm_slabs_create", "lbm_slabs_step", "lbm_slabs_residual",
    "lbm_slabs_get_populations", "lbm_slabs_set_populations", "lbm_slabs_fields",
    "lbm_slabs_count", "lbm_slabs_steps_done", "lbm_slabs_halo_bytes", "lbm_slabs_synchronize",
    "lbm_slabs_last_error", "lbm_slabs_destroy", "lbm_slabs_cut_populations",
    "lbm_slabs_cut_values", "lbm_slabs_pack_cut", "lbm_slabs_unpack_cut",
)

_bound = False
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def _lib():
    global _bound
    L = load()
    if _bound:
        return L
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    L.lbm_slabs_plan.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _I, _I, _I, _I, _I]
    L.lbm_slabs_create.argtypes = [P(Grid), ctypes.c_int, P(Params), P(Options), ctypes.c_int, _I,
                                   P(vp)]
    L.lbm_slabs_step.argtypes = [vp, ctypes.c_int64]
    L.lbm_slabs_residual.argtypes = [vp, _D]
    L.lbm_slabs_get_populations.argtypes = [vp, _D, _D]
    L.lbm_slabs_set_populations.argtypes = [vp, _D, _D]
    L.lbm_slabs_fields.argtypes = [vp] + [_D] * 5
    L.lbm_slabs_count.argtypes = [vp]
    L.lbm_slabs_steps_done.argtypes = [vp]
    L.lbm_slabs_steps_done.restype = ctypes.c_int64
    L.lbm_slabs_halo_bytes.argtypes = [vp]
    L.lbm_slabs_halo_bytes.restype = ctypes.c_int64
    L.lbm_slabs_synchronize.argtypes = [vp]
    L.lbm_slabs_last_error.argtypes = [vp]
    L.lbm_slabs_last_error.restype = ctypes.c_char_p
    L.lbm_slabs_destroy.argtypes = [vp]
    L.lbm_slabs_destroy.restype = None
    L.lbm_slabs_cut_populations.argtypes = [ctypes.c_int, ctypes.c_int, _I, _I, _I, _I]
    L.lbm_slabs_cut_values.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.lbm_slabs_cut_values.restype = ctypes.c_int64
    L.lbm_slabs_pack_cut.argtypes = [P(Grid), ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, _D]
    L.lbm_slabs_unpack_cut.argtypes = [P(Grid), ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, _D]
    _bound = True
    return L


def _ints(values):
    return None if values is None else (ctypes.c_int * len(values))(*[int(v) for v in values])


def cut_populations(lattice, direction):
    """The flow and scalar directions that cross a cut upwards (+1) or downwards (-1)."""
    L = _lib()
    f, g = (ctypes.c_int * 15)(), (ctypes.c_int * 15)()
    nf, ng = ctypes.c_int(), ctypes.c_int()
    rc = L.lbm_slabs_cut_populations(int(lattice), int(direction), f, ctypes.byref(nf), g, ctypes.byref(ng))
    if rc != LBM_OK:
        raise LBMError(rc, L.lbm_slabs_last_error(None).decode())
    return list(f)[:nf.value], list(g)[:ng.value]


def _cut_args(f, g, lattice):
    if f.dtype != np.float64 or g.dtype != np.float64 or not (f.flags.c_contiguous and g.flags.c_contiguous):
        raise ValueError("populations must be C-contiguous float64 arrays")
    if f.ndim != 4 or g.ndim != 4 or f.shape[0] != 15 or g.shape[0] != lattice or f.shape[1:] != g.shape[1:]:
        raise ValueError("populations must be shaped (15, nz, ny, nx) and (lattice, nz, ny, nx)")
    nz, ny, nx = f.shape[1:]
    return Grid(nx, ny, nz)


def pack_cut(f, g, lattice, plane, direction):
    """The message of one cut (lbm_slabs_pack_cut): the populations of local plane `plane`
    of a slab's host state (f, g) that cross the cut in `direction`."""
    L = _lib()
    grid = _cut_args(f, g, lattice)
    msg = np.empty(L.lbm_slabs_cut_values(grid.nx, grid.ny, int(lattice)))
    rc = L.lbm_slabs_pack_cut(ctypes.byref(grid), int(lattice), int(plane), int(direction),
                              f.ctypes.data_as(_D), g.ctypes.data_as(_D), msg.ctypes.data_as(_D))
    if rc != LBM_OK:
        raise LBMError(rc, L.lbm_slabs_last_error(None).decode())
    return msg


def unpack_cut(msg, f, g, lattice, plane, direction):
    """Write a message into local plane `plane` of a slab's host state (lbm_slabs_unpack_cut)."""
    L = _lib()
    grid = _cut_args(f, g, lattice)
    msg = np.ascontiguousarray(msg, dtype=np.float64)
    if msg.size != L.lbm_slabs_cut_values(grid.nx, grid.ny, int(lattice)):
        raise ValueError("message of the wrong size")
    rc = L.lbm_slabs_unpack_cut(ctypes.byref(grid), int(lattice), int(plane), int(direction),
                                msg.ctypes.data_as(_D), f.ctypes.data_as(_D), g.ctypes.data_as(_D))
    if rc != LBM_OK:
        raise LBMError(rc, L.lbm_slabs_last_error(None).decode())


def plan(nz, nslabs, boundary=_b.BC_CAVITY, owned=None):
    """Host-only split of nz planes into slabs: dict of lists z0, nz_owned, halo_lo,
    halo_hi (lbm_slabs_plan)."""
    L = _lib()
    n = int(nslabs)
    outs = [(ctypes.c_int * max(n, 1))() for _ in range(4)]
    if owned is not None and len(owned) != n:
        raise ValueError("owned needs one plane count per slab")
    rc = L.lbm_slabs_plan(int(nz), n, int(boundary), _ints(owned), *outs)
    if rc != LBM_OK:
        raise LBMError(rc, L.lbm_slabs_last_error(None).decode())
    return {k: list(o)[:n] for k, o in zip(("z0", "nz_owned", "halo_lo", "halo_hi"), outs)}


class Slabs:
    """One cavity on `grid` split into `nslabs` z-slabs (even split, or the plane counts
    `owned`).  Either (Ra, Pr, Ma) or explicit `params` (a Params structure or a dict of
    its fields, for the whole grid) must be given; the options are those of lbm.LBM.
    The slabs allocate their own device memory and run on torch's current stream unless
    `stream` is given."""

    def __init__(self, grid, nslabs=2, lattice=D3Q15, Ra=None, Pr=0.71, Ma=0.05 * math.sqrt(3.0),
                 params=None, owned=None, precision=FP32, seed=1, noise_amp=1e-6, cs2_phi=0.0,
                 e4_mode=0, adiabatic_mode=_b.ADIABATIC_SPECULAR, residual_interval=100,
                 stream=None, timeout_s=600.0):
        import torch

        if not torch.cuda.is_available():
            raise LBMError(LBM_ECUDA, "no CUDA device: the library has no CPU path")
        self._L = _lib()
        self._h = ctypes.c_void_p()
        self.grid = tuple(int(v) for v in grid)
        self.lattice = int(lattice)
        self.precision = int(precision)
        o = Options()
        self._L.lbm_default_options(ctypes.byref(o))
        o.precision, o.seed, o.noise_amp = self.precision, int(seed) & (2**64 - 1), float(noise_amp)
        o.cs2_phi, o.e4_mode, o.adiabatic_mode = float(cs2_phi), int(e4_mode), int(adiabatic_mode)
        o.residual_interval, o.timeout_s = int(residual_interval), float(timeout_s)
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        o.cuda_stream = self._stream.cuda_stream
        if params is None:
            if Ra is None:
                raise ValueError("give Ra (with Pr, Ma) or explicit params")
            params = _b.derive_params(self.grid, self.lattice, Ra, Pr, Ma, cs2_phi=float(cs2_phi),
                                      e4_mode=int(e4_mode), adiabatic_mode=int(adiabatic_mode))
        elif isinstance(params, dict):
            p = Params()
            for k, v in params.items():
                if isinstance(v, (list, tuple)):
                    arr = getattr(p, k)
                    for n, x in enumerate(v):
                        arr[n] = x
                else:
                    setattr(p, k, v)
            params = p
        self.params = params
        rc = self._L.lbm_slabs_create(ctypes.byref(Grid(*self.grid)), self.lattice, ctypes.byref(params),
                                      ctypes.byref(o), int(nslabs), _ints(owned), ctypes.byref(self._h))
        if rc != LBM_OK:
            raise LBMError(rc, self._L.lbm_slabs_last_error(None).decode())
        self.plan = plan(self.grid[2], nslabs, params.boundary, owned)

    def _check(self, rc):
        if rc != LBM_OK:
            raise LBMError(rc, self._L.lbm_slabs_last_error(self._h).decode())

    @property
    def count(self):
        return int(self._L.lbm_slabs_count(self._h))

    @property
    def steps_done(self):
        return int(self._L.lbm_slabs_steps_done(self._h))

    @property
    def halo_bytes(self):
        """Bytes the exchange copies per time step."""
        return int(self._L.lbm_slabs_halo_bytes(self._h))

    def step(self, n=1):
        self._check(self._L.lbm_slabs_step(self._h, int(n)))

    def residual(self):
        r = ctypes.c_double()
        self._check(self._L.lbm_slabs_residual(self._h, ctypes.byref(r)))
        return r.value

    def get_populations(self):
        nx, ny, nz = self.grid
        f = np.empty((15, nz, ny, nx))
        g = np.empty((self.lattice, nz, ny, nx))
        self._check(self._L.lbm_slabs_get_populations(self._h, f.ctypes.data_as(_D), g.ctypes.data_as(_D)))
        return f, g

    def set_populations(self, f, g):
        nx, ny, nz = self.grid
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(15, nz, ny, nx)
        g = np.ascontiguousarray(g, dtype=np.float64).reshape(self.lattice, nz, ny, nx)
        self._check(self._L.lbm_slabs_set_populations(self._h, f.ctypes.data_as(_D), g.ctypes.data_as(_D)))

    def fields(self):
        nx, ny, nz = self.grid
        out = [np.empty((nz, ny, nx)) for _ in range(5)]
        self._check(self._L.lbm_slabs_fields(self._h, *[o.ctypes.data_as(_D) for o in out]))
        return dict(zip(("rho", "ux", "uy", "uz", "T"), out))

    def synchronize(self):
        self._check(self._L.lbm_slabs_synchronize(self._h))

    def close(self):
        if self._h and self._h.value:
            self._L.lbm_slabs_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _time(sim, steps):
    import torch
    stream = torch.cuda.current_stream()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    sim.step(steps)
    end.record(stream)
    torch.cuda.synchronize()
    return start.elapsed_time(end) / 1e3


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--slabs", type=int, default=2)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=300)
    ap.add_argument("--skip-undivided", action="store_true", help="time the slabs only")
    args = ap.parse_args(argv)
    grid = (args.n,) * 3
    kw = dict(Ra=1e5, Pr=0.71, Ma=0.05 * math.sqrt(3.0))
    t1 = None
    if not args.skip_undivided:
        one = _b.LBM(grid, D3Q15, **kw)
        one.step(args.warmup)
        t1 = _time(one, args.steps)
        one.close()
    dec = Slabs(grid, args.slabs, D3Q15, **kw)
    dec.step(args.warmup)
    t2 = _time(dec, args.steps)
    out = {"grid": list(grid), "slabs": args.slabs, "plan": dec.plan, "steps": args.steps,
           "undivided_ms_per_step": round(t1 / args.steps * 1e3, 5) if t1 else None,
           "slabs_ms_per_step": round(t2 / args.steps * 1e3, 5),
           "time_vs_undivided": round(t2 / t1, 4) if t1 else None,
           "halo_bytes_per_step": dec.halo_bytes}
    dec.close()
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
