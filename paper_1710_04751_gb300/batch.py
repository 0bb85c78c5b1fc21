"""Python binding of include/lbm_batch.h (argument marshalling only): many independent
cavities advanced by one persistent CUDA kernel per step, captured in graphs, with a
batched convergence check and a tiling autotuner.  PyTorch supplies the device memory
and the stream; every step runs in liblbm.so."""
import ctypes
import math

from . import lbm as _b
from .lbm import D3Q15, FP32, Grid, LBMError, LBM_OK, LBM_ECUDA, Params, load

MEMBER_ACTIVE, MEMBER_CONVERGED, MEMBER_DIVERGED = 0, 1, 2
TILE_LINEAR, TILE_ROWS = 0, 1
MODES = {"graph": 0, "launch": 1, "sequential": 2}
STATE_NAMES = {0: "active", 1: "converged", 2: "diverged"}

# Every entry point include/lbm_batch.h declares (checked by tests/test_abi.py).
EXPORTS = (
    "lbm_batch_default_options", "lbm_batch_arena_bytes", "lbm_batch_create", "lbm_batch_step",
    "lbm_batch_step_with", "lbm_batch_status", "lbm_batch_member", "lbm_batch_count",
    "lbm_batch_steps_done", "lbm_batch_active_nodes", "lbm_batch_autotune",
    "lbm_batch_get_tiling", "lbm_batch_set_tiling", "lbm_batch_synchronize",
    "lbm_batch_last_error", "lbm_batch_destroy",
)


class Tiling(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int), ("min_blocks", ctypes.c_int), ("mapping", ctypes.c_int),
                ("blocks_per_sm", ctypes.c_int), ("tile_factor", ctypes.c_int)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class Trial(ctypes.Structure):
    _fields_ = [("tiling", Tiling), ("ms_per_step", ctypes.c_double)]


class BatchOptions(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int), ("seed", ctypes.c_uint64), ("noise_amp", ctypes.c_double),
        ("residual_interval", ctypes.c_int), ("steady_tol", ctypes.c_double),
        ("cuda_stream", ctypes.c_void_p), ("device_arena", ctypes.c_void_p),
        ("device_arena_bytes", ctypes.c_size_t), ("autotune_steps", ctypes.c_int),
        ("tiling", Tiling), ("timeout_s", ctypes.c_double),
    ]


_bound = False


def _lib():
    global _bound
    L = load()
    if _bound:
        return L
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    L.lbm_batch_default_options.argtypes = [P(BatchOptions)]
    L.lbm_batch_default_options.restype = None
    L.lbm_batch_arena_bytes.argtypes = [ctypes.c_int, P(Grid), ctypes.c_int, ctypes.c_int]
    L.lbm_batch_arena_bytes.restype = ctypes.c_size_t
    L.lbm_batch_create.argtypes = [ctypes.c_int, P(Grid), ctypes.c_int, P(Params), P(BatchOptions),
                                   P(vp)]
    L.lbm_batch_step.argtypes = [vp, ctypes.c_int64]
    L.lbm_batch_step_with.argtypes = [vp, ctypes.c_int64, ctypes.c_int]
    L.lbm_batch_status.argtypes = [vp, P(ctypes.c_int), P(ctypes.c_int64), P(ctypes.c_double)]
    L.lbm_batch_member.argtypes = [vp, ctypes.c_int, P(vp)]
    L.lbm_batch_count.argtypes = [vp]
    L.lbm_batch_steps_done.argtypes = [vp]
    L.lbm_batch_steps_done.restype = ctypes.c_int64
    L.lbm_batch_active_nodes.argtypes = [vp]
    L.lbm_batch_active_nodes.restype = ctypes.c_int64
    L.lbm_batch_autotune.argtypes = [vp, ctypes.c_int, P(Trial), ctypes.c_int, P(ctypes.c_int)]
    L.lbm_batch_get_tiling.argtypes = [vp, P(Tiling)]
    L.lbm_batch_set_tiling.argtypes = [vp, P(Tiling)]
    L.lbm_batch_synchronize.argtypes = [vp]
    L.lbm_batch_last_error.argtypes = [vp]
    L.lbm_batch_last_error.restype = ctypes.c_char_p
    L.lbm_batch_destroy.argtypes = [vp]
    L.lbm_batch_destroy.restype = None
    _bound = True
    return L


def default_options():
    o = BatchOptions()
    _lib().lbm_batch_default_options(ctypes.byref(o))
    return o


def arena_bytes(grids, lattice, precision):
    arr = (Grid * len(grids))(*[Grid(*g) for g in grids])
    return int(_lib().lbm_batch_arena_bytes(len(grids), arr, int(lattice), int(precision)))


def _params_struct(p):
    if isinstance(p, Params):
        return p
    out = Params()
    for k, v in p.items():
        if isinstance(v, (list, tuple)):
            arr = getattr(out, k)
            for n, x in enumerate(v):
                arr[n] = x
        else:
            setattr(out, k, v)
    return out


class Batch:
    """Independent cavities advanced together on one GPU.

    members: a list whose entries are dicts with "grid" (nx, ny, nz) and either
    "params" (Params or dict of its fields) or "Ra" and "Pr" (then the parameters come
    from lbm_derive_params with Ma and the derivation options given here).
    tiling: None (tune at creation) or a dict of Tiling fields.
    """

    def __init__(self, members, lattice=D3Q15, precision=FP32, seed=1, noise_amp=1e-6,
                 residual_interval=100, steady_tol=0.0, tiling=None, autotune_steps=3,
                 Ma=0.05 * math.sqrt(3.0), stream=None, device=None, timeout_s=600.0,
                 **derive_opts):
        import torch

        if not torch.cuda.is_available():
            raise LBMError(LBM_ECUDA, "no CUDA device: the library has no CPU path")
        L = _lib()
        self._L = L
        self._b = ctypes.c_void_p()
        self.lattice, self.precision = int(lattice), int(precision)
        self._grids = [tuple(int(v) for v in m["grid"]) for m in members]
        plist = []
        for m in members:
            if "params" in m:
                plist.append(_params_struct(m["params"]))
            else:
                plist.append(_b.derive_params(m["grid"], lattice, m["Ra"], m["Pr"], Ma, **derive_opts))
        n = len(members)
        grids = (Grid * n)(*[Grid(*g) for g in self._grids])
        params = (Params * n)(*plist)
        o = default_options()
        o.precision, o.seed, o.noise_amp = self.precision, int(seed) & (2**64 - 1), float(noise_amp)
        o.residual_interval, o.steady_tol = int(residual_interval), float(steady_tol)
        o.autotune_steps, o.timeout_s = int(autotune_steps), float(timeout_s)
        if tiling is not None:
            for k, v in dict(tiling).items():
                setattr(o.tiling, k, int(v))
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.device = dev
        with torch.cuda.device(dev):
            self._stream = stream if stream is not None else torch.cuda.current_stream(dev)
            o.cuda_stream = self._stream.cuda_stream
            nbytes = int(L.lbm_batch_arena_bytes(n, grids, self.lattice, self.precision))
            if nbytes == 0:
                raise LBMError(_b.LBM_EINVAL, "invalid batch (grids, lattice or precision)")
            self._arena = torch.empty(nbytes, dtype=torch.uint8, device=dev)
            o.device_arena, o.device_arena_bytes = self._arena.data_ptr(), nbytes
            rc = L.lbm_batch_create(n, grids, self.lattice, params, ctypes.byref(o),
                                    ctypes.byref(self._b))
            if rc != LBM_OK:
                raise LBMError(rc, L.lbm_batch_last_error(None).decode())
        self._handles = []
        for i in range(n):
            h = ctypes.c_void_p()
            self._check(L.lbm_batch_member(self._b, i, ctypes.byref(h)))
            self._handles.append(h.value)

    def _check(self, rc):
        if rc != LBM_OK:
            raise LBMError(rc, self._L.lbm_batch_last_error(self._b).decode())

    @property
    def count(self):
        return len(self._grids)

    @property
    def grids(self):
        return list(self._grids)

    def step(self, n=1, mode="graph"):
        self._check(self._L.lbm_batch_step_with(self._b, int(n), MODES[mode]))

    def status(self):
        n = self.count
        st = (ctypes.c_int * n)()
        steps = (ctypes.c_int64 * n)()
        res = (ctypes.c_double * n)()
        self._check(self._L.lbm_batch_status(self._b, st, steps, res))
        return [dict(state=STATE_NAMES[st[i]], steps=int(steps[i]), residual=float(res[i]))
                for i in range(n)]

    def member(self, i):
        return _b.LBM._view(self._handles[i], self)

    @property
    def steps_done(self):
        return int(self._L.lbm_batch_steps_done(self._b))

    @property
    def active_nodes(self):
        return int(self._L.lbm_batch_active_nodes(self._b))

    @property
    def tiling(self):
        t = Tiling()
        self._check(self._L.lbm_batch_get_tiling(self._b, ctypes.byref(t)))
        return t.as_dict()

    def set_tiling(self, **kw):
        t = Tiling(**{k: int(v) for k, v in kw.items()})
        self._check(self._L.lbm_batch_set_tiling(self._b, ctypes.byref(t)))

    def autotune(self, trial_steps=3):
        trials = (Trial * 128)()
        n = ctypes.c_int()
        self._check(self._L.lbm_batch_autotune(self._b, int(trial_steps), trials, 128, ctypes.byref(n)))
        return [dict(t.tiling.as_dict(), ms_per_step=t.ms_per_step) for t in trials[:n.value]]

    def synchronize(self):
        self._check(self._L.lbm_batch_synchronize(self._b))

    def close(self):
        if getattr(self, "_b", None) is not None and self._b.value:
            self._L.lbm_batch_destroy(self._b)
            self._b = ctypes.c_void_p()
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
