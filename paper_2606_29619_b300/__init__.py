"""B300-native porous-media lattice Boltzmann hot path (Gusev & Karlin, Sec. 3).

This module is the thin Python binding of ``liblbm.so`` (C ABI in
``include/lbm.h``): it marshals arguments only, every step of the method runs
in the library's CUDA kernels.  PyTorch supplies device memory (through the
allocator callbacks of the ABI) and streams.  There is no CPU fallback: if the
library is missing, importing the binding's functions raises.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblbm.so")

D2Q9, D3Q27 = 0, 1
STORAGE = {"fp64": 0, "fp32": 1, "fp16": 2, "bf16": 3}
BC = {"periodic": 0, "wall": 1, "inflow_outflow": 2, "moving_walls": 3}
KERNEL = {"auto": 0, "sweep": 1, "fused": 2, "split": 3}
PLANES = {"neem": 0, "equilibrium": 1, "tms": 2}
DENSITY = {"continuity": 0, "bounce_back": 1}
OUTLET = {"pressure": 0, "zero_gradient": 1}
INLET = {"uniform": 0, "poiseuille": 1}
LID = {"uniform": 0, "regularised": 1}
STREAMING = {"auto": 0, "two_arrays": 1, "in_place": 2}
CORR_DELTA_NU, CORR_PHI_EXT, CORR_PHI_ETA, CORR_FULL = 1, 2, 4, 7
F_ERGUN = -1.0

LBM_OK = 0
ERRORS = {-1: "LBM_E_INVALID", -2: "LBM_E_CUDA", -3: "LBM_E_NOMEM", -4: "LBM_E_DIVERGED", -5: "LBM_E_UNSUPPORTED",
          -6: "LBM_E_TIMEOUT"}

# symbols include/lbm.h declares; tests check the library exports all of them
EXPORTS = ["lbm_default_params", "lbm_create", "lbm_init_fields", "lbm_step", "lbm_sync", "lbm_moments",
           "lbm_moments_device", "lbm_get_populations", "lbm_set_populations", "lbm_reduce", "lbm_info",
           "lbm_time_kernels", "lbm_destroy", "lbm_last_error", "lbm_population_sums_noalloc", "lbm_save", "lbm_load",
           "lbm_server_create", "lbm_server_submit", "lbm_server_run", "lbm_server_clock", "lbm_server_stats",
           "lbm_server_destroy", "lbm_tuning", "lbm_tune_cache_lookup", "lbm_tune_cache_store"]

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class LbmParams(ctypes.Structure):
    _fields_ = [
        ("storage", ctypes.c_int),
        ("RT", ctypes.c_double),
        ("J_nu", ctypes.c_double),
        ("J_eta", ctypes.c_double),
        ("corrections", ctypes.c_int),
        ("bc", ctypes.c_int * 3),
        ("rho0", ctypes.c_double),
        ("v0", ctypes.c_double * 3),
        ("stream", ctypes.c_void_p),
        ("device", ctypes.c_int),
        ("alloc", ALLOC_FN),
        ("free", FREE_FN),
        ("alloc_user", ctypes.c_void_p),
        ("kernel", ctypes.c_int),
        ("inlet_v", ctypes.c_double * 3),
        ("outlet_rho", ctypes.c_double),
        ("picard_iters", ctypes.c_int),
        ("picard_omega", ctypes.c_double),
        ("plane_scheme", ctypes.c_int),
        ("wall_v_low", ctypes.c_double * 3),
        ("wall_v_high", ctypes.c_double * 3),
        ("plane_density", ctypes.c_int),
        ("outlet", ctypes.c_int),
        ("inlet_profile", ctypes.c_int),
        ("lid_profile", ctypes.c_int),
        ("lid_delta", ctypes.c_double),
        ("wait_probe", ctypes.c_int),
        ("streaming", ctypes.c_int),
        ("tile_y", ctypes.c_int),
        ("autotune", ctypes.c_int),
        ("tune_cache", ctypes.c_char_p),
    ]


class LbmStats(ctypes.Structure):
    _fields_ = [
        ("mass", ctypes.c_double),
        ("mean_v", ctypes.c_double * 3),
        ("v2_sum", ctypes.c_double),
        ("dv2_sum", ctypes.c_double),
        ("residual", ctypes.c_double),
        ("drag", ctypes.c_double * 3),
        ("k_app", ctypes.c_double * 3),
        ("steps", ctypes.c_long),
    ]


class LbmCaseResult(ctypes.Structure):
    _fields_ = [
        ("id", ctypes.c_longlong),
        ("status", ctypes.c_int),
        ("steps", ctypes.c_long),
        ("residual", ctypes.c_double),
        ("mean_v", ctypes.c_double * 3),
        ("k_app", ctypes.c_double),
        ("submit_time", ctypes.c_double),
        ("finish_time", ctypes.c_double),
    ]


class LbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load_library(path: str = LIB_PATH):
    """Loads liblbm.so (built by ``build.py``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"liblbm.so not built at {path}; run python -m paper_2606_29619_b300.build")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER(ctypes.c_double)
    V = ctypes.c_void_p
    lib.lbm_default_params.argtypes = [ctypes.POINTER(LbmParams)]
    lib.lbm_create.argtypes = [ctypes.POINTER(V), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P,
                               ctypes.c_double, ctypes.c_double, P, ctypes.POINTER(LbmParams)]
    lib.lbm_init_fields.argtypes = [V, P, P]
    lib.lbm_step.argtypes = [V, ctypes.c_long]
    lib.lbm_sync.argtypes = [V]
    lib.lbm_moments.argtypes = [V, P, P]
    lib.lbm_moments_device.argtypes = [V, V, V]
    lib.lbm_get_populations.argtypes = [V, P]
    lib.lbm_set_populations.argtypes = [V, P]
    lib.lbm_reduce.argtypes = [V, ctypes.POINTER(LbmStats), ctypes.c_int]
    lib.lbm_info.argtypes = [V, P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                             ctypes.POINTER(ctypes.c_int)]
    lib.lbm_time_kernels.argtypes = [V, ctypes.c_long, P, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    IP = ctypes.POINTER(ctypes.c_int)
    lib.lbm_tuning.argtypes = [V, IP, IP, IP, P, IP]
    lib.lbm_tune_cache_lookup.argtypes = [ctypes.c_char_p, ctypes.c_char_p, IP]
    lib.lbm_tune_cache_store.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.c_int, ctypes.c_int, IP, P]
    lib.lbm_destroy.argtypes = [V]
    lib.lbm_destroy.restype = None
    lib.lbm_last_error.restype = ctypes.c_char_p
    lib.lbm_save.argtypes = [V, ctypes.c_char_p]
    lib.lbm_load.argtypes = [ctypes.POINTER(V), ctypes.c_char_p, ctypes.POINTER(LbmParams)]
    lib.lbm_server_create.argtypes = [ctypes.POINTER(V), ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                      ctypes.POINTER(LbmParams)]
    lib.lbm_server_submit.argtypes = [V, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_double,
                                      ctypes.c_double, P, ctypes.c_double, ctypes.c_long,
                                      ctypes.POINTER(ctypes.c_longlong)]
    lib.lbm_server_run.argtypes = [V, ctypes.c_int, ctypes.POINTER(LbmCaseResult), ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_int)]
    lib.lbm_server_clock.restype = ctypes.c_double
    lib.lbm_server_clock.argtypes = [V]
    lib.lbm_server_stats.argtypes = [V, P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
    lib.lbm_server_destroy.argtypes = [V]
    lib.lbm_server_destroy.restype = None
    lib.lbm_population_sums_noalloc.argtypes = [ctypes.c_int, ctypes.c_longlong, V, V, V]
    _lib = lib
    return lib


def _check(code):
    if code != LBM_OK:
        raise LbmError(code, load_library().lbm_last_error().decode())


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class _TorchAllocator:
    """Allocator callbacks that route device memory through torch's caching allocator."""

    def __init__(self, device, stream_handle):
        import torch

        self._torch = torch
        self.device = device
        self.stream = stream_handle
        self.live = {}

        def _alloc(nbytes, _user):
            try:
                ptr = torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
            except Exception:
                return None
            self.live[int(ptr)] = nbytes
            return ptr

        def _free(ptr, _user):
            if ptr:
                self.live.pop(int(ptr), None)
                torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc = ALLOC_FN(_alloc)
        self.free = FREE_FN(_free)


class Simulation:
    """One porous-media LBM case on the GPU (see include/lbm.h for every argument).

    porosity, permeability: arrays of shape (nz, ny, nx) or (ny, nx), x fastest,
    permeability = inf marks free fluid.  force: body acceleration b.
    """

    def __init__(self, lattice, porosity, permeability, *, viscosity, force=(0.0, 0.0, 0.0), forchheimer=0.0,
                 storage="fp32", RT=1.0 / 3.0, J_nu=1.0, J_eta=1.0, corrections=CORR_FULL,
                 bc=("periodic", "periodic", "periodic"), rho0=1.0, v0=(0.0, 0.0, 0.0), stream=None, device=0,
                 kernel="auto", torch_allocator=True, inlet_v=(0.0, 0.0, 0.0), outlet_rho=1.0, picard_iters=0,
                 picard_omega=1.0, plane_scheme="neem", wall_v=((0.0, 0.0, 0.0), (0.0, 0.0, 0.0)),
                 plane_density="continuity", outlet="pressure", inlet_profile="uniform", lid_profile="uniform",
                 lid_delta=0.1, wait_probe=False, streaming="auto", tile_y=0, autotune=False, tune_cache=None,
                 allocator=None):
        lib = load_library()
        eps = np.ascontiguousarray(porosity, dtype=np.float64)
        kap = np.ascontiguousarray(permeability, dtype=np.float64)
        if eps.ndim == 2:
            eps, kap = eps[None], kap[None]
        if eps.shape != kap.shape:
            raise ValueError("porosity and permeability shapes differ")
        self.shape = eps.shape
        nz, ny, nx = eps.shape
        self.N = nx * ny * nz
        self.lattice = lattice
        self.D = 2 if lattice == D2Q9 else 3
        self.Q = 9 if lattice == D2Q9 else 27
        p = LbmParams()
        lib.lbm_default_params(ctypes.byref(p))
        p.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        p.RT, p.J_nu, p.J_eta, p.corrections = RT, J_nu, J_eta, corrections
        for a in range(3):
            p.bc[a] = BC[bc[a]] if isinstance(bc[a], str) else int(bc[a])
            p.v0[a] = float(v0[a]) if a < len(v0) else 0.0
        p.rho0 = rho0
        p.device = device
        for a in range(3):
            p.inlet_v[a] = float(inlet_v[a]) if a < len(inlet_v) else 0.0
        p.outlet_rho = float(outlet_rho)
        p.picard_iters = int(picard_iters)
        p.picard_omega = float(picard_omega)
        p.plane_scheme = PLANES[plane_scheme] if isinstance(plane_scheme, str) else int(plane_scheme)
        for k in range(3):
            p.wall_v_low[k] = float(wall_v[0][k]) if k < len(wall_v[0]) else 0.0
            p.wall_v_high[k] = float(wall_v[1][k]) if k < len(wall_v[1]) else 0.0
        p.plane_density = DENSITY[plane_density] if isinstance(plane_density, str) else int(plane_density)
        p.outlet = OUTLET[outlet] if isinstance(outlet, str) else int(outlet)
        p.inlet_profile = INLET[inlet_profile] if isinstance(inlet_profile, str) else int(inlet_profile)
        p.lid_profile = LID[lid_profile] if isinstance(lid_profile, str) else int(lid_profile)
        p.lid_delta = float(lid_delta)
        p.wait_probe = int(bool(wait_probe))
        p.streaming = STREAMING[streaming] if isinstance(streaming, str) else int(streaming)
        p.tile_y = int(tile_y)
        p.autotune = int(bool(autotune))
        p.tune_cache = None if tune_cache is None else os.fsencode(tune_cache)
        p.kernel = KERNEL[kernel] if isinstance(kernel, str) else int(kernel)
        self._stream_obj = None
        if stream is not None:
            handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
            p.stream = handle
            self._stream_obj = stream
        self._alloc = None
        if allocator is not None:
            # any object with ctypes `alloc` / `free` callbacks (ALLOC_FN / FREE_FN)
            self._alloc = allocator
            p.alloc = allocator.alloc
            p.free = allocator.free
        elif torch_allocator:
            self._alloc = _TorchAllocator(device, p.stream or 0)
            p.alloc = self._alloc.alloc
            p.free = self._alloc.free
        f = np.ascontiguousarray(np.resize(np.asarray(force, np.float64), 3))
        h = ctypes.c_void_p()
        self._lib = lib
        _check(lib.lbm_create(ctypes.byref(h), lattice, nx, ny, nz, _dptr(eps), _dptr(kap), float(forchheimer),
                              float(viscosity), _dptr(f), ctypes.byref(p)))
        self._h = h
        self.storage = storage
        self.params = p

    # ------------------------------------------------------------------ lifetime
    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_destroy(self._h)
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

    # ------------------------------------------------------------------ stepping
    def init_fields(self, rho0=None, v0=None):
        r = None if rho0 is None else np.ascontiguousarray(np.broadcast_to(rho0, self.shape), np.float64).ravel()
        v = None
        if v0 is not None:
            v0 = np.asarray(v0, np.float64)
            v = np.zeros((3, self.N))
            for a in range(v0.shape[0]):
                v[a] = np.broadcast_to(v0[a], self.shape).ravel()
        _check(self._lib.lbm_init_fields(self._h, None if r is None else _dptr(r), None if v is None else _dptr(v)))
        return self

    def step(self, n=1):
        _check(self._lib.lbm_step(self._h, int(n)))
        return self

    def sync(self):
        _check(self._lib.lbm_sync(self._h))
        return self

    # ------------------------------------------------------------------ outputs
    def moments(self):
        """(rho (nz,ny,nx), v (3,nz,ny,nx)) in FP64 on the host."""
        rho = np.empty(self.N)
        v = np.empty(3 * self.N)
        _check(self._lib.lbm_moments(self._h, _dptr(rho), _dptr(v)))
        return rho.reshape(self.shape), v.reshape((3,) + self.shape)

    def moments_device(self, rho_out, v_out):
        """Writes rho (N) and v (3N) into FP64 torch CUDA tensors without synchronising."""
        _check(self._lib.lbm_moments_device(self._h, ctypes.c_void_p(rho_out.data_ptr()),
                                            ctypes.c_void_p(v_out.data_ptr())))

    def get_populations(self):
        f = np.empty(self.Q * self.N)
        _check(self._lib.lbm_get_populations(self._h, _dptr(f)))
        return f.reshape((self.Q,) + self.shape)

    def set_populations(self, f):
        f = np.ascontiguousarray(f, np.float64).ravel()
        if f.size != self.Q * self.N:
            raise ValueError("population array has the wrong size")
        _check(self._lib.lbm_set_populations(self._h, _dptr(f)))

    def reduce(self, snapshot=False):
        st = LbmStats()
        _check(self._lib.lbm_reduce(self._h, ctypes.byref(st), int(bool(snapshot))))
        return {"mass": st.mass, "mean_v": list(st.mean_v), "v2_sum": st.v2_sum, "dv2_sum": st.dv2_sum,
                "residual": st.residual, "drag": list(st.drag), "k_app": list(st.k_app), "steps": st.steps}

    def save(self, path):
        """Checkpoint to `path` (lbm_save)."""
        _check(self._lib.lbm_save(self._h, os.fsencode(path)))

    @classmethod
    def load(cls, path, *, stream=None, device=0, torch_allocator=True, allocator=None):
        """Re-creates a simulation from a checkpoint (lbm_load)."""
        lib = load_library()
        self = cls.__new__(cls)
        p = LbmParams()
        lib.lbm_default_params(ctypes.byref(p))
        p.device = device
        self._stream_obj = None
        if stream is not None:
            p.stream = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
            self._stream_obj = stream
        self._alloc = None
        if allocator is not None:
            # any object with ctypes `alloc` / `free` callbacks (ALLOC_FN / FREE_FN)
            self._alloc = allocator
            p.alloc = allocator.alloc
            p.free = allocator.free
        elif torch_allocator:
            self._alloc = _TorchAllocator(device, p.stream or 0)
            p.alloc = self._alloc.alloc
            p.free = self._alloc.free
        h = ctypes.c_void_p()
        self._lib = lib
        _check(lib.lbm_load(ctypes.byref(h), os.fsencode(path), ctypes.byref(p)))
        self._h = h
        import struct
        with open(path, "rb") as fh:
            head = fh.read(8 + 4 * 10)
        lattice, nx, ny, nz, storage = struct.unpack_from("<5i", head, 8)
        self.lattice = lattice
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self.D = 2 if lattice == D2Q9 else 3
        self.Q = 9 if lattice == D2Q9 else 27
        self.storage = {v: k for k, v in STORAGE.items()}[storage]
        self.params = p
        return self

    def time_kernels(self, n):
        """Advances n steps with CUDA events around each kernel of a step
        (lbm_time_kernels) and returns the mean milliseconds per launch of
        each kernel, in launch order."""
        ms = (ctypes.c_double * 8)()
        k = ctypes.c_int()
        _check(self._lib.lbm_time_kernels(self._h, int(n), ms, 8, ctypes.byref(k)))
        return [ms[i] for i in range(k.value)]

    def info(self):
        b = ctypes.c_double()
        l = ctypes.c_int()
        k = ctypes.c_int()
        ip = ctypes.c_int()
        _check(self._lib.lbm_info(self._h, ctypes.byref(b), ctypes.byref(l), ctypes.byref(k), ctypes.byref(ip)))
        return {"bytes_per_node_update": b.value, "launches_per_step": l.value,
                "kernel": {v: s for s, v in KERNEL.items()}[k.value], "in_place": bool(ip.value)}

    def tuning(self):
        """The split kernels' tile height and the autotuner's measurements."""
        ty, n, src = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        tiles = (ctypes.c_int * 8)()
        ms = np.zeros(8)
        _check(self._lib.lbm_tuning(self._h, ctypes.byref(ty), ctypes.byref(n), tiles, _dptr(ms), ctypes.byref(src)))
        return {"tile_y": ty.value, "candidates": {int(tiles[j]): float(ms[j]) for j in range(n.value)},
                "source": ["default", "timed", "cache"][src.value]}


def tune_cache_lookup(path, key):
    """The tile height the cache file stores for key (0: none)."""
    lib = load_library()
    t = ctypes.c_int()
    _check(lib.lbm_tune_cache_lookup(os.fsencode(path), key.encode(), ctypes.byref(t)))
    return t.value


def tune_cache_store(path, key, tile_y, ms_by_tile=None):
    """Appends one choice to the cache file."""
    lib = load_library()
    ms_by_tile = ms_by_tile or {}
    tiles = (ctypes.c_int * max(1, len(ms_by_tile)))(*ms_by_tile.keys())
    ms = np.ascontiguousarray(list(ms_by_tile.values()) or [0.0], np.float64)
    _check(lib.lbm_tune_cache_store(os.fsencode(path), key.encode(), int(tile_y), len(ms_by_tile), tiles, _dptr(ms)))


class Server:
    """Continuous-batching server for independent periodic D3Q27 cases
    (lbm_server_* in include/lbm.h)."""

    def __init__(self, storage="fp16", hbm_cap_bytes=60e9, check_every=100, device=0, RT=1.0 / 3.0):
        lib = load_library()
        p = LbmParams()
        lib.lbm_default_params(ctypes.byref(p))
        p.device = device
        p.RT = RT
        h = ctypes.c_void_p()
        st = STORAGE[storage] if isinstance(storage, str) else int(storage)
        _check(lib.lbm_server_create(ctypes.byref(h), st, float(hbm_cap_bytes), int(check_every), ctypes.byref(p)))
        self._lib = lib
        self._h = h
        self.check_every = check_every

    def submit(self, porosity, permeability, *, viscosity, force, forchheimer=F_ERGUN, tol=1e-7, max_steps=200000):
        eps = np.ascontiguousarray(porosity, np.float64)
        kap = np.ascontiguousarray(permeability, np.float64)
        nz, ny, nx = eps.shape
        f = np.ascontiguousarray(np.resize(np.asarray(force, np.float64), 3))
        t = ctypes.c_longlong()
        _check(self._lib.lbm_server_submit(self._h, nx, ny, nz, _dptr(eps), _dptr(kap), float(forchheimer),
                                           float(viscosity), _dptr(f), float(tol), int(max_steps), ctypes.byref(t)))
        return t.value

    def run(self, batches=1, max_results=4096):
        res = (LbmCaseResult * max_results)()
        n, a, q = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(self._lib.lbm_server_run(self._h, int(batches), res, max_results, ctypes.byref(n), ctypes.byref(a),
                                        ctypes.byref(q)))
        out = [{"id": r.id, "status": r.status, "steps": r.steps, "residual": r.residual, "mean_v": list(r.mean_v),
                "k_app": r.k_app, "submit_time": r.submit_time, "finish_time": r.finish_time}
               for r in res[: n.value]]
        return out, a.value, q.value

    def clock(self):
        return self._lib.lbm_server_clock(self._h)

    def stats(self):
        u = ctypes.c_double()
        l = ctypes.c_longlong()
        nu = ctypes.c_longlong()
        _check(self._lib.lbm_server_stats(self._h, ctypes.byref(u), ctypes.byref(l), ctypes.byref(nu)))
        return {"used_bytes": u.value, "kernel_launches": l.value, "node_updates": nu.value}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
