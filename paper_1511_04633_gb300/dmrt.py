"""ctypes binding of the dmrt C ABI (``include/dmrt.h``).

Argument marshalling only: every step of the method runs in the CUDA library.
Functions carry the C names; ``Cavity`` is a small convenience wrapper over a
handle.  Arrays may be numpy (host) or torch CUDA tensors (device); torch is
only used for device memory and streams.

If ``libdmrt.so`` is missing or cannot be loaded, importing the binding
fails loudly: there is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

from . import build as _build

OK, ERR_ARG, ERR_CUDA, ERR_OOM, ERR_DIVERGED, ERR_TIMEOUT = range(6)
WALL_PERIODIC, WALL_TYPE1, WALL_TYPE2, WALL_TYPE3 = 0, 1, 2, 3
STORE_F32, STORE_BF16, STORE_F16 = 0, 1, 2
ROUND_AUTO, ROUND_NEAREST, ROUND_STOCHASTIC = 0, 1, 2

HEADER = os.path.join(_build.INCLUDE, "dmrt.h")


class DmrtError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


class dmrt_opts(ctypes.Structure):
    _fields_ = [("storage", ctypes.c_int), ("residual_interval", ctypes.c_int),
                ("rounding", ctypes.c_int)]


class dmrt_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("wall_type", ctypes.c_int), ("storage", ctypes.c_int),
                ("residual_interval", ctypes.c_int), ("rounding", ctypes.c_int),
                ("nu", ctypes.c_double), ("alpha", ctypes.c_double), ("gbeta", ctypes.c_double),
                ("tau_nu", ctypes.c_double), ("tau_alpha", ctypes.c_double),
                ("steps", ctypes.c_long)]


class dmrt_stats(ctypes.Structure):
    _fields_ = [("step_launches", ctypes.c_long), ("total_launches", ctypes.c_long),
                ("step_ms", ctypes.c_double), ("timed_steps", ctypes.c_long),
                ("bytes_per_cell", ctypes.c_double)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load ``libdmrt.so`` (building it first if allowed and needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise ImportError(f"dmrt CUDA library not built: {path} is missing")
        L = ctypes.CDLL(path)
        vp, i, d, l_ = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_long
        P = ctypes.POINTER
        grid_t = P(ctypes.c_int)
        sig = {
            "dmrt_create": ([P(vp), grid_t, d, d, d, i], i),
            "dmrt_create_ex": ([P(vp), grid_t, d, d, d, i, P(dmrt_opts)], i),
            "dmrt_create_lattice": ([P(vp), grid_t, d, d, d, i, P(dmrt_opts)], i),
            "dmrt_destroy": ([vp], None),
            "dmrt_set_stream": ([vp, vp], i),
            "dmrt_step": ([vp, l_], i),
            "dmrt_sync": ([vp], i),
            "dmrt_fields": ([vp, vp, vp, vp, i], i),
            "dmrt_nusselt": ([vp, i, P(d)], i),
            "dmrt_nusselt_local": ([vp, i, vp, i], i),
            "dmrt_nusselt_noalloc": ([vp, i, i, i, i, vp, P(d)], i),
            "dmrt_residual": ([vp, P(d)], i),
            "dmrt_run_to_steady": ([vp, d, l_, P(l_), P(d)], i),
            "dmrt_set_populations": ([vp, vp, vp, i], i),
            "dmrt_get_populations": ([vp, vp, vp, i], i),
            "dmrt_init_fields": ([vp, vp, vp, vp, i], i),
            "dmrt_get_params": ([vp, P(dmrt_params)], i),
            "dmrt_set_timing": ([vp, i], i),
            "dmrt_get_stats": ([vp, P(dmrt_stats), i], i),
            "dmrt_last_error": ([vp], ctypes.c_char_p),
            "dmrt_status_string": ([i], ctypes.c_char_p),
            "dmrt_version": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
        return L


def declared_functions():
    """Names of the functions declared in include/dmrt.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dmrt_[a-z_0-9]+)\s*\(", text)))


# ---------------------------------------------------------------- marshalling helpers

def _ptr(a):
    """(address, on_device) of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("host arrays must be C-contiguous float32")
        return a.ctypes.data, 0
    # torch tensor
    if str(a.dtype) != "torch.float32" or not a.is_contiguous():
        raise TypeError("tensors must be contiguous float32")
    return a.data_ptr(), 1 if a.is_cuda else 0


def _same_side(*arrs):
    sides = {s for _, s in (_ptr(a) for a in arrs if a is not None)}
    if len(sides) > 1:
        raise TypeError("mix of host and device arrays in one call")
    return sides.pop() if sides else 0


def check(h, status: int, what: str):
    if status != OK:
        L = load()
        name = L.dmrt_status_string(status).decode()
        msg = L.dmrt_last_error(h).decode() if h else ""
        raise DmrtError(status, f"{what}: {name} {msg}".strip())


# ---------------------------------------------------------------- C-named functions

def dmrt_create(grid, Ra: float, Pr: float = 0.71, Ma: float = 0.1, wall_type: int = 1,
                storage: int = STORE_F32, residual_interval: int = 0, rounding: int = ROUND_AUTO):
    L = load()
    h = ctypes.c_void_p()
    g = (ctypes.c_int * 3)(*grid)
    opts = dmrt_opts(storage, residual_interval, rounding)
    check(None, L.dmrt_create_ex(ctypes.byref(h), g, Ra, Pr, Ma, wall_type, ctypes.byref(opts)),
          "dmrt_create")
    return h


def dmrt_create_lattice(grid, nu: float, alpha: float, gbeta: float, wall_type: int = 1,
                        storage: int = STORE_F32, residual_interval: int = 0,
                        rounding: int = ROUND_AUTO):
    L = load()
    h = ctypes.c_void_p()
    g = (ctypes.c_int * 3)(*grid)
    opts = dmrt_opts(storage, residual_interval, rounding)
    check(None, L.dmrt_create_lattice(ctypes.byref(h), g, nu, alpha, gbeta, wall_type,
                                      ctypes.byref(opts)), "dmrt_create_lattice")
    return h


def dmrt_destroy(h):
    load().dmrt_destroy(h)


def dmrt_set_stream(h, stream):
    """`stream`: a torch.cuda.Stream, a raw cudaStream_t int, or None."""
    raw = getattr(stream, "cuda_stream", stream)
    check(h, load().dmrt_set_stream(h, raw), "dmrt_set_stream")


def dmrt_step(h, n: int):
    check(h, load().dmrt_step(h, int(n)), "dmrt_step")


def dmrt_sync(h):
    check(h, load().dmrt_sync(h), "dmrt_sync")


def dmrt_fields(h, rho=None, u=None, theta=None):
    side = _same_side(rho, u, theta)
    check(h, load().dmrt_fields(h, _ptr(rho)[0], _ptr(u)[0], _ptr(theta)[0], side), "dmrt_fields")


def dmrt_nusselt(h, wall: int = 0):
    out = (ctypes.c_double * 3)()
    check(h, load().dmrt_nusselt(h, wall, out), "dmrt_nusselt")
    return tuple(out)


def dmrt_nusselt_local(h, wall, local):
    p, side = _ptr(local)
    check(h, load().dmrt_nusselt_local(h, wall, p, side), "dmrt_nusselt_local")


def dmrt_nusselt_noalloc(theta, wall: int = 0, stream=None):
    """Nusselt numbers of a CUDA float32 tensor theta[z][y][x], computed
    without any device allocation (see include/dmrt.h)."""
    p, side = _ptr(theta)
    if side != 1:
        raise TypeError("theta must be a CUDA tensor")
    nz, ny, nx = theta.shape
    raw = getattr(stream, "cuda_stream", stream)
    out = (ctypes.c_double * 3)()
    check(None, load().dmrt_nusselt_noalloc(p, nx, ny, nz, wall, raw, out), "dmrt_nusselt_noalloc")
    return tuple(out)


def dmrt_residual(h) -> float:
    r = ctypes.c_double()
    check(h, load().dmrt_residual(h, ctypes.byref(r)), "dmrt_residual")
    return r.value


def dmrt_run_to_steady(h, tol: float, max_steps: int):
    n = ctypes.c_long()
    r = ctypes.c_double()
    st = load().dmrt_run_to_steady(h, tol, int(max_steps), ctypes.byref(n), ctypes.byref(r))
    if st not in (OK, ERR_TIMEOUT):
        check(h, st, "dmrt_run_to_steady")
    return st == OK, n.value, r.value


def dmrt_set_populations(h, f, g):
    side = _same_side(f, g)
    check(h, load().dmrt_set_populations(h, _ptr(f)[0], _ptr(g)[0], side), "dmrt_set_populations")


def dmrt_get_populations(h, f=None, g=None):
    side = _same_side(f, g)
    check(h, load().dmrt_get_populations(h, _ptr(f)[0], _ptr(g)[0], side), "dmrt_get_populations")


def dmrt_init_fields(h, rho, u, theta):
    side = _same_side(rho, u, theta)
    check(h, load().dmrt_init_fields(h, _ptr(rho)[0], _ptr(u)[0], _ptr(theta)[0], side),
          "dmrt_init_fields")


def dmrt_get_params(h) -> dict:
    p = dmrt_params()
    check(h, load().dmrt_get_params(h, ctypes.byref(p)), "dmrt_get_params")
    return {k: getattr(p, k) for k, _ in dmrt_params._fields_}


def dmrt_set_timing(h, enabled: bool):
    check(h, load().dmrt_set_timing(h, int(bool(enabled))), "dmrt_set_timing")


def dmrt_get_stats(h, reset: bool = False) -> dict:
    s = dmrt_stats()
    check(h, load().dmrt_get_stats(h, ctypes.byref(s), int(bool(reset))), "dmrt_get_stats")
    return {k: getattr(s, k) for k, _ in dmrt_stats._fields_}


def dmrt_last_error(h) -> str:
    return load().dmrt_last_error(h).decode()


def dmrt_status_string(status: int) -> str:
    return load().dmrt_status_string(status).decode()


def dmrt_version() -> str:
    return load().dmrt_version().decode()


# ---------------------------------------------------------------- convenience wrapper

class Cavity:
    """One cavity handle.  ``grid`` = (nx, ny, nz); fields come back as numpy
    arrays shaped [z][y][x] (velocity [3][z][y][x])."""

    def __init__(self, grid, Ra=None, Pr=0.71, Ma=0.1, wall_type=1, *, lattice=None,
                 storage=STORE_F32, residual_interval=0, rounding=ROUND_AUTO):
        self.grid = tuple(int(v) for v in grid)
        nx, ny, nz = self.grid
        self.shape = (nz, ny, nx)
        self.cells = nx * ny * nz
        if lattice is not None:
            nu, alpha, gbeta = lattice
            self.h = dmrt_create_lattice(self.grid, nu, alpha, gbeta, wall_type, storage,
                                         residual_interval, rounding)
        else:
            self.h = dmrt_create(self.grid, Ra, Pr, Ma, wall_type, storage, residual_interval,
                                 rounding)

    def close(self):
        if getattr(self, "h", None):
            dmrt_destroy(self.h)
            self.h = None

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
    def params(self):
        return dmrt_get_params(self.h)

    def step(self, n=1):
        dmrt_step(self.h, n)

    def sync(self):
        dmrt_sync(self.h)

    def fields(self):
        rho = np.empty(self.shape, np.float32)
        u = np.empty((3,) + self.shape, np.float32)
        th = np.empty(self.shape, np.float32)
        dmrt_fields(self.h, rho, u, th)
        return rho, u, th

    def nusselt(self, wall=0):
        return dmrt_nusselt(self.h, wall)

    def nusselt_local(self, wall=0):
        out = np.empty((self.grid[2], self.grid[0]), np.float32)
        dmrt_nusselt_local(self.h, wall, out)
        return out

    def residual(self):
        return dmrt_residual(self.h)

    def run_to_steady(self, tol, max_steps):
        return dmrt_run_to_steady(self.h, tol, max_steps)

    def set_populations(self, f, g):
        dmrt_set_populations(self.h, np.ascontiguousarray(f, np.float32),
                             np.ascontiguousarray(g, np.float32))

    def populations(self):
        f = np.empty((19,) + self.shape, np.float32)
        g = np.empty((7,) + self.shape, np.float32)
        dmrt_get_populations(self.h, f, g)
        return f, g

    def init_fields(self, rho, u, theta):
        dmrt_init_fields(self.h, np.ascontiguousarray(rho, np.float32),
                         np.ascontiguousarray(u, np.float32),
                         np.ascontiguousarray(theta, np.float32))
