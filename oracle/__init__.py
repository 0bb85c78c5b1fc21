"""FP64 CPU oracle of the cascaded central-moment thermal LBM (arXiv:1710.04751).

TEST INFRASTRUCTURE.  This package is the reference the CUDA library is checked
against: a plain restatement of the paper's equations in C (lbm_oracle.c, the paper's
closed-form cascades, "Form A") and in numpy (formb.py, the generic relaxation of
central moments, "Form B").  It shares no code with the CUDA path.  Only tests/,
__graft_entry__.smoke() and bench.py's cpu_baseline / reference legs may import it.

Parity pins (see tests/test_oracle_*.py): K against the paper's printed
back-transform and source inversions, Form A == Form B for random states and rates,
fixed point of equilibrium, exact conservation on periodic / closed boxes, shear-wave
decay (viscosity), advected Gaussian (diffusivity), conduction (Nu = 1) and the
paper's Table 1 at Ra = 1e3.
"""
import ctypes
import math
import os

import numpy as np

from . import build as _build

BC_CAVITY, BC_PERIODIC, BC_XWALLS, BC_ADIABATIC_BOX = 0, 7, 6, 8

_lib = None


class _Problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("q_g", ctypes.c_int), ("boundary", ctypes.c_int), ("e4_mode", ctypes.c_int),
        ("adiabatic_mode", ctypes.c_int),
        ("omega_f", ctypes.c_double * 15), ("omega_g", ctypes.c_double * 15),
        ("gbeta", ctypes.c_double), ("T_hot", ctypes.c_double), ("T_cold", ctypes.c_double),
        ("cs2_phi", ctypes.c_double), ("ext_force", ctypes.c_double * 3),
        ("U0", ctypes.c_double), ("heat_source", ctypes.c_double),
    ]


class _Nu(ctypes.Structure):
    _fields_ = [(name, ctypes.c_double) for name in (
        "hot_wall_mean", "cold_wall_mean", "mid_mean", "mid_max", "mid_max_z", "mid_min",
        "mid_min_z", "umax", "umax_z", "wmax", "wmax_x")]


_D = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        L = _lib
        L.orc_collide_flow.argtypes = [_D, _D, _D, ctypes.c_int, _D, _D, _D]
        L.orc_collide_thermal15.argtypes = [_D, _D, _D, ctypes.c_double, ctypes.c_double, _D]
        L.orc_collide_thermal7.argtypes = [_D, _D, _D, ctypes.c_double, ctypes.c_double, _D]
        L.orc_scalar_source.argtypes = [ctypes.c_int, ctypes.c_double, _D, _D]
        L.orc_flow_source.argtypes = [_D, _D, _D]
        L.orc_init.argtypes = [ctypes.POINTER(_Problem), ctypes.c_uint64, ctypes.c_double, _D, _D]
        L.orc_step.argtypes = [ctypes.POINTER(_Problem), _D, _D, _D, _D]
        L.orc_run.argtypes = [ctypes.POINTER(_Problem), _D, _D, _D, _D, ctypes.c_int64]
        L.orc_cell_update.argtypes = [ctypes.POINTER(_Problem), _D, _D, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_int, _D, _D]
        L.orc_fields.argtypes = [ctypes.POINTER(_Problem), _D, _D, _D, _D, _D, _D, _D]
        L.orc_nusselt.argtypes = [ctypes.POINTER(_Problem), _D, _D, ctypes.POINTER(_Nu)]
        L.orc_splitmix64.argtypes = [ctypes.c_uint64]
        L.orc_splitmix64.restype = ctypes.c_uint64
        L.orc_kmatrix15.argtypes = [ctypes.POINTER(ctypes.c_int)]
        L.orc_kmatrix7.argtypes = [ctypes.POINTER(ctypes.c_int)]
        L.orc_weights_flow.argtypes = [_D]
        L.orc_weights_thermal.argtypes = [ctypes.c_int, ctypes.c_double, _D]
        L.orc_velocities.argtypes = [ctypes.c_int] + [ctypes.POINTER(ctypes.c_int)] * 3
        L.orc_opposite.argtypes = [ctypes.c_int, ctypes.c_int]
        L.orc_set_num_threads.argtypes = [ctypes.c_int]
        L.orc_set_num_threads.restype = None
    return _lib


def _dp(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


# ----------------------------------------------------------------------------------
# Tables
# ----------------------------------------------------------------------------------

def velocities(q=15):
    ex, ey, ez = ((ctypes.c_int * q)() for _ in range(3))
    lib().orc_velocities(q, ex, ey, ez)
    return np.array([list(ex), list(ey), list(ez)], dtype=np.int64).T  # (q, 3)


def kmatrix(q=15):
    buf = (ctypes.c_int * (q * q))()
    (lib().orc_kmatrix15 if q == 15 else lib().orc_kmatrix7)(buf)
    return np.array(list(buf), dtype=np.int64).reshape(q, q)  # K[b, a] = K_b(e_a)


def weights_flow():
    w = np.zeros(15)
    lib().orc_weights_flow(_dp(w))
    return w


def weights_thermal(q=15, cs2_phi=1.0 / 3.0):
    w = np.zeros(q)
    lib().orc_weights_thermal(q, cs2_phi, _dp(w))
    return w


def opposite(q=15):
    return np.array([lib().orc_opposite(q, a) for a in range(q)])


def splitmix64(x):
    return int(lib().orc_splitmix64(x & 0xFFFFFFFFFFFFFFFF))


# ----------------------------------------------------------------------------------
# One-cell collisions (Form A)
# ----------------------------------------------------------------------------------

def flow_source(F, u):
    S = np.zeros(15)
    lib().orc_flow_source(_dp(_f64(F)), _dp(_f64(u)), _dp(S))
    return S


def collide_flow(fbar, F, omega, e4_mode=0):
    """Appendix A: returns (f~, rho, u) for one cell."""
    out = np.zeros(15)
    rho = np.zeros(1)
    u = np.zeros(3)
    lib().orc_collide_flow(_dp(_f64(fbar)), _dp(_f64(F)), _dp(_f64(omega)), int(e4_mode),
                           _dp(out), _dp(rho), _dp(u))
    return out, float(rho[0]), u


def collide_thermal(gbar, u, omega, cs2_phi=1.0 / 3.0, R=0.0):
    """Sec. 2.2 (15 populations) or Appendix C (7 populations) for one cell, with the
    scalar source R of Eq. (4)."""
    gbar = _f64(gbar)
    q = gbar.shape[0]
    out = np.zeros(q)
    fn = lib().orc_collide_thermal15 if q == 15 else lib().orc_collide_thermal7
    fn(_dp(gbar), _dp(_f64(u)), _dp(_f64(omega)), float(cs2_phi), float(R), _dp(out))
    return out


def scalar_source(q, R, u):
    """S^phi of Appendix B (q = 15) or C (q = 7)."""
    S = np.zeros(q)
    lib().orc_scalar_source(int(q), float(R), _dp(_f64(u)), _dp(S))
    return S


# ----------------------------------------------------------------------------------
# Problems and grids
# ----------------------------------------------------------------------------------

def physical_parameters(L, Ra, Pr, Ma, cs2_phi=1.0 / 3.0, dT=1.0):
    """Sec. 3: Ra = g beta dT L^3/(alpha nu), Pr = nu/alpha; U0 = sqrt(g beta dT L) = Ma c_s.
    Relaxation rates from nu = c_s^2 (1/omega - 1/2) (App. A) and
    D = c_sphi^2 (1/omega - 1/2) (Eq. 23)."""
    U0 = Ma / math.sqrt(3.0)
    gbeta = U0 * U0 / (dT * L)
    nu = math.sqrt(Pr / Ra) * U0 * L
    alpha = nu / Pr
    omega_nu = 1.0 / (3.0 * nu + 0.5)
    omega_phi = 1.0 / (alpha / cs2_phi + 0.5)
    return dict(U0=U0, gbeta=gbeta, nu=nu, alpha=alpha, omega_nu=omega_nu, omega_phi=omega_phi)


class Problem:
    """A grid problem for the oracle.  Relaxation rates default to the paper's choice:
    flow omega_4..8 = omega_nu (shear), the rest 1 (App. A); thermal omega_1..3 =
    omega_phi, the rest 1 (Sec. 2.2 / App. C)."""

    def __init__(self, nx, ny, nz, q_g=15, boundary=BC_CAVITY, omega_nu=1.0, omega_phi=1.0,
                 gbeta=0.0, T_hot=0.5, T_cold=-0.5, cs2_phi=1.0 / 3.0, e4_mode=0,
                 ext_force=(0.0, 0.0, 0.0), U0=0.0, omega_f=None, omega_g=None,
                 adiabatic_mode=1, heat_source=0.0):
        self.nx, self.ny, self.nz, self.q_g = int(nx), int(ny), int(nz), int(q_g)
        self.boundary, self.e4_mode = int(boundary), int(e4_mode)
        self.adiabatic_mode = int(adiabatic_mode)
        self.heat_source = float(heat_source)
        if omega_f is None:
            # App. A: "nu = cs^2 (1/omega_j - 1/2), j = 5..9", counted from 1: the five
            # shear moments g^_4..g^_8; the bulk moment g^_9 and the rest relax at 1
            omega_f = [1.0] * 15
            for b in range(4, 9):
                omega_f[b] = omega_nu
        if omega_g is None:
            omega_g = [1.0] * 15
            for b in range(1, 4):
                omega_g[b] = omega_phi
        self.omega_f = list(map(float, omega_f)) + [1.0] * (15 - len(omega_f))
        self.omega_g = list(map(float, omega_g)) + [1.0] * (15 - len(omega_g))
        self.gbeta, self.T_hot, self.T_cold = float(gbeta), float(T_hot), float(T_cold)
        self.cs2_phi, self.U0 = float(cs2_phi), float(U0)
        self.ext_force = tuple(map(float, ext_force))

    @classmethod
    def cavity(cls, n, Ra, Pr=0.71, Ma=0.05 * math.sqrt(3.0), q_g=15, cs2_phi=None,
               e4_mode=0, ny=None, nz=None, adiabatic_mode=1):
        """The cavity of Sec. 3.  cs2_phi defaults to 1/3 (D3Q15) or 1/4 (D3Q7: at 1/3 its
        rest equilibrium phi (1 - 3 cs2_phi - u^2) turns negative)."""
        if cs2_phi is None:
            cs2_phi = 1.0 / 3.0 if q_g == 15 else 0.25
        par = physical_parameters(n, Ra, Pr, Ma, cs2_phi)
        return cls(n, ny or n, nz or n, q_g=q_g, omega_nu=par["omega_nu"],
                   omega_phi=par["omega_phi"], gbeta=par["gbeta"], cs2_phi=cs2_phi,
                   e4_mode=e4_mode, U0=par["U0"], adiabatic_mode=adiabatic_mode)

    @property
    def ncell(self):
        return self.nx * self.ny * self.nz

    def _c(self):
        p = _Problem()
        p.nx, p.ny, p.nz, p.q_g = self.nx, self.ny, self.nz, self.q_g
        p.boundary, p.e4_mode = self.boundary, self.e4_mode
        p.adiabatic_mode = self.adiabatic_mode
        for b in range(15):
            p.omega_f[b] = self.omega_f[b]
            p.omega_g[b] = self.omega_g[b]
        p.gbeta, p.T_hot, p.T_cold = self.gbeta, self.T_hot, self.T_cold
        p.cs2_phi, p.U0 = self.cs2_phi, self.U0
        p.heat_source = self.heat_source
        for d in range(3):
            p.ext_force[d] = self.ext_force[d]
        return p

    def shapes(self):
        return (15, self.nz, self.ny, self.nx), (self.q_g, self.nz, self.ny, self.nx)

    def init(self, seed=1, noise_amp=1e-6):
        fs, gs = self.shapes()
        F, G = np.zeros(fs), np.zeros(gs)
        lib().orc_init(ctypes.byref(self._c()), seed & 0xFFFFFFFFFFFFFFFF, float(noise_amp),
                       _dp(F), _dp(G))
        return F, G

    def step(self, F, G):
        F, G = _f64(F, self.shapes()[0]), _f64(G, self.shapes()[1])
        Fo, Go = np.empty_like(F), np.empty_like(G)
        rc = lib().orc_step(ctypes.byref(self._c()), _dp(F), _dp(G), _dp(Fo), _dp(Go))
        if rc:
            raise ValueError(f"orc_step failed ({rc})")
        return Fo, Go

    def run(self, F, G, nsteps):
        F, G = _f64(F, self.shapes()[0]).copy(), _f64(G, self.shapes()[1]).copy()
        Fs, Gs = np.empty_like(F), np.empty_like(G)
        rc = lib().orc_run(ctypes.byref(self._c()), _dp(F), _dp(G), _dp(Fs), _dp(Gs), int(nsteps))
        if rc:
            raise ValueError(f"orc_run failed ({rc})")
        return F, G

    def cell_update(self, F, G, i, j, k):
        """Post-step populations of one cell (pull + collide) without a whole-grid step."""
        F, G = _f64(F, self.shapes()[0]), _f64(G, self.shapes()[1])
        fo, go = np.zeros(15), np.zeros(self.q_g)
        lib().orc_cell_update(ctypes.byref(self._c()), _dp(F), _dp(G), int(i), int(j), int(k),
                              _dp(fo), _dp(go))
        return fo, go

    def fields(self, F, G):
        F, G = _f64(F, self.shapes()[0]), _f64(G, self.shapes()[1])
        shp = (self.nz, self.ny, self.nx)
        out = [np.zeros(shp) for _ in range(5)]
        lib().orc_fields(ctypes.byref(self._c()), _dp(F), _dp(G), *[_dp(o) for o in out])
        return dict(zip(("rho", "ux", "uy", "uz", "T"), out))

    def nusselt(self, F, G):
        F, G = _f64(F, self.shapes()[0]), _f64(G, self.shapes()[1])
        nu = _Nu()
        rc = lib().orc_nusselt(ctypes.byref(self._c()), _dp(F), _dp(G), ctypes.byref(nu))
        if rc:
            raise ValueError(f"orc_nusselt failed ({rc})")
        return {name: getattr(nu, name) for name, _ in _Nu._fields_}


def num_threads():
    return int(lib().orc_num_threads())


def set_num_threads(n):
    """Threads of the oracle's OpenMP loop (results do not depend on it)."""
    lib().orc_set_num_threads(int(n))
