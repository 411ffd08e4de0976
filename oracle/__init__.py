"""Python handle on the FP64 CPU oracle (``lbm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the oracle is the slow, plain statement of the
porous-media lattice Boltzmann step (Gusev & Karlin, Sec. 3) that the CUDA
library is checked against.  Only the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package; the product path
never does, and the oracle imports nothing from the product.

Every function of the C file cites the equation it follows.  This module only
marshals numpy arrays to it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

CORR_DELTA_NU = 1
CORR_PHI_EXT = 2
CORR_PHI_ETA = 4
CORR_FULL = CORR_DELTA_NU | CORR_PHI_EXT | CORR_PHI_ETA
PLANES_NEEM, PLANES_EQUILIBRIUM, PLANES_TMS = 0, 1, 2
DENSITY_CONTINUITY, DENSITY_BOUNCE_BACK = 0, 1
OUTLET_PRESSURE, OUTLET_ZERO_GRADIENT = 0, 1
INLET_UNIFORM, INLET_POISEUILLE = 0, 1
LID_UNIFORM, LID_REGULARISED = 0, 1

D2Q9 = 0
D3Q27 = 1


class _Params(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int),
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("nz", ctypes.c_int),
        ("wall", ctypes.c_int * 3),
        ("RT", ctypes.c_double),
        ("nu_f", ctypes.c_double),
        ("J_nu", ctypes.c_double),
        ("J_eta", ctypes.c_double),
        ("forch", ctypes.c_double),
        ("b", ctypes.c_double * 3),
        ("corr", ctypes.c_int),
        ("v_in", ctypes.c_double * 3),
        ("rho_out", ctypes.c_double),
        ("picard_iters", ctypes.c_int),
        ("picard_omega", ctypes.c_double),
        ("plane_scheme", ctypes.c_int),
        ("wall_v", ctypes.c_double * 6),
        ("plane_density", ctypes.c_int),
        ("outlet", ctypes.c_int),
        ("inlet_profile", ctypes.c_int),
        ("lid_profile", ctypes.c_int),
        ("lid_delta", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, OpenMP over nodes)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
             "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER(ctypes.c_double)
        lib.or_create.restype = ctypes.c_void_p
        lib.or_create.argtypes = [ctypes.POINTER(_Params), P, P]
        lib.or_free.argtypes = [ctypes.c_void_p]
        lib.or_init.argtypes = [ctypes.c_void_p, P, P]
        lib.or_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
        lib.or_moments.argtypes = [ctypes.c_void_p, P, P]
        lib.or_forces.argtypes = [ctypes.c_void_p, P, P, P]
        lib.or_get_f.argtypes = [ctypes.c_void_p, P]
        lib.or_set_f.argtypes = [ctypes.c_void_p, P]
        lib.or_num_steps.restype = ctypes.c_long
        lib.or_num_steps.argtypes = [ctypes.c_void_p]
        lib.or_beta.restype = ctypes.c_double
        lib.or_beta.argtypes = [ctypes.c_void_p]
        lib.or_weights.argtypes = [ctypes.c_void_p, P, ctypes.POINTER(ctypes.c_int)]
        lib.or_static.argtypes = [ctypes.c_void_p, P, P, P, P]
        lib.or_delta_nu.argtypes = [ctypes.c_void_p, P, P]
        lib.or_corrections.argtypes = [ctypes.c_void_p, P, P, P, P]
        lib.or_product_form.argtypes = [ctypes.c_void_p, ctypes.c_double, P, P, P]
        lib.or_threads.restype = ctypes.c_int
        lib.or_threads.argtypes = []
        lib.or_set_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def threads() -> int:
    """Threads the oracle's node loops run on."""
    return int(_load().or_threads())


def set_threads(n: int) -> None:
    """Sets the oracle's thread count (the result does not depend on it)."""
    _load().or_set_threads(int(n))


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Oracle:
    """One oracle simulation.

    eps, kappa: node fields of shape (nz, ny, nx) (x fastest); kappa = inf marks
    free fluid.  wall: per-axis flags (x, y, z), 1 = halfway bounce-back walls.
    forch: F_eps >= 0, or negative for the Ergun correlation.
    """

    def __init__(self, lattice, eps, kappa, *, nu_f, b=(0.0, 0.0, 0.0), forch=0.0, RT=1.0 / 3.0,
                 J_nu=1.0, J_eta=1.0, wall=(0, 0, 0), corr=CORR_FULL, v_in=(0.0, 0.0, 0.0), rho_out=1.0,
                 picard_iters=0, picard_omega=1.0, plane_scheme=0, wall_v=((0.0, 0.0, 0.0), (0.0, 0.0, 0.0)),
                 plane_density=0, outlet=0, inlet_profile=0, lid_profile=0, lid_delta=0.1):
        lib = _load()
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        kappa = np.ascontiguousarray(kappa, dtype=np.float64)
        if eps.ndim == 2:
            eps = eps[None]
            kappa = kappa[None]
        nz, ny, nx = eps.shape
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self.D = 2 if lattice == D2Q9 else 3
        self.Q = 9 if lattice == D2Q9 else 27
        p = _Params()
        p.lattice, p.nx, p.ny, p.nz = lattice, nx, ny, nz
        for k in range(3):
            p.wall[k] = int(wall[k])
            p.b[k] = float(b[k]) if k < len(b) else 0.0
        p.RT, p.nu_f, p.J_nu, p.J_eta, p.forch, p.corr = RT, nu_f, J_nu, J_eta, forch, corr
        for k in range(3):
            p.v_in[k] = float(v_in[k]) if k < len(v_in) else 0.0
        p.rho_out = rho_out
        p.picard_iters = int(picard_iters)
        p.picard_omega = float(picard_omega)
        p.plane_scheme = int(plane_scheme)
        for face in range(2):
            for k in range(3):
                p.wall_v[3 * face + k] = float(wall_v[face][k]) if k < len(wall_v[face]) else 0.0
        p.plane_density = int(plane_density)
        p.outlet = int(outlet)
        p.inlet_profile = int(inlet_profile)
        p.lid_profile = int(lid_profile)
        p.lid_delta = float(lid_delta)
        self._eps = eps
        self._h = lib.or_create(ctypes.byref(p), _p(eps), _p(kappa))
        if not self._h:
            raise ValueError("oracle rejected the parameters")
        self._lib = lib

    def __del__(self):
        if getattr(self, "_h", None):
            self._lib.or_free(self._h)
            self._h = None

    def init(self, rho0=None, v0=None):
        rho = np.ones(self.N) if rho0 is None else np.ascontiguousarray(np.broadcast_to(rho0, self.shape), np.float64).ravel()
        v = np.zeros((self.N, 3))
        if v0 is not None:
            v0 = np.asarray(v0, dtype=np.float64)
            if v0.ndim == 1:
                v[:, : v0.shape[0]] = v0
            else:  # (D or 3, nz, ny, nx)
                for k in range(v0.shape[0]):
                    v[:, k] = np.broadcast_to(v0[k], self.shape).ravel()
        v = np.ascontiguousarray(v)
        rho = np.ascontiguousarray(rho)
        self._lib.or_init(self._h, _p(rho), _p(v))
        return self

    def step(self, n=1):
        self._lib.or_step(self._h, int(n))
        return self

    @property
    def steps(self):
        return self._lib.or_num_steps(self._h)

    @property
    def beta(self):
        return self._lib.or_beta(self._h)

    def moments(self):
        """(rho (nz,ny,nx), v (3,nz,ny,nx)) of the current post-stream state."""
        rho = np.empty(self.N)
        v = np.empty((self.N, 3))
        self._lib.or_moments(self._h, _p(rho), _p(v))
        return rho.reshape(self.shape), np.ascontiguousarray(v.T).reshape((3,) + self.shape)

    def forces(self):
        a = np.empty((self.N, 3))
        phx = np.empty((self.N, 3))
        phe = np.empty(self.N)
        self._lib.or_forces(self._h, _p(a), _p(phx), _p(phe))
        t = lambda x: np.ascontiguousarray(x.T).reshape((3,) + self.shape)
        return t(a), t(phx), phe.reshape(self.shape)

    def get_f(self):
        f = np.empty(self.Q * self.N)
        self._lib.or_get_f(self._h, _p(f))
        return f.reshape((self.Q,) + self.shape)

    def set_f(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).ravel()
        assert f.size == self.Q * self.N
        self._lib.or_set_f(self._h, _p(f))

    def lattice(self):
        w = np.empty(self.Q)
        c = np.empty(3 * self.Q, dtype=np.int32)
        self._lib.or_weights(self._h, _p(w), c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        return w, c.reshape(self.Q, 3)

    def static(self):
        muD = np.empty(self.N)
        muF = np.empty(self.N)
        g = np.empty((self.N, 3))
        h = np.empty((self.N, 9))
        self._lib.or_static(self._h, _p(muD), _p(muF), _p(g), _p(h))
        return (muD.reshape(self.shape), muF.reshape(self.shape),
                np.ascontiguousarray(g.T).reshape((3,) + self.shape),
                np.ascontiguousarray(h.T).reshape((3, 3) + self.shape))

    def delta_nu(self, m):
        """Delta_nu(m) for m of shape (3, nz, ny, nx) using this state's eps derivatives."""
        mm = np.ascontiguousarray(np.asarray(m, np.float64).reshape(3, self.N).T)
        out = np.empty((self.N, 3))
        self._lib.or_delta_nu(self._h, _p(mm), _p(out))
        return np.ascontiguousarray(out.T).reshape((3,) + self.shape)

    def corrections(self, rho, v):
        r = np.ascontiguousarray(np.broadcast_to(rho, self.shape), np.float64).ravel().copy()
        vv = np.ascontiguousarray(np.asarray(v, np.float64).reshape(3, self.N).T)
        phx = np.empty((self.N, 3))
        phe = np.empty(self.N)
        self._lib.or_corrections(self._h, _p(r), _p(vv), _p(phx), _p(phe))
        return np.ascontiguousarray(phx.T).reshape((3,) + self.shape), phe.reshape(self.shape)

    def product_form(self, eps_rho, xi, P):
        xi = np.ascontiguousarray(np.resize(np.asarray(xi, np.float64), 3))
        P = np.ascontiguousarray(np.resize(np.asarray(P, np.float64), 3))
        out = np.empty(self.Q)
        self._lib.or_product_form(self._h, float(eps_rho), _p(xi), _p(P), _p(out))
        return out

    def mass(self):
        return float(np.sum(self.get_f()))
