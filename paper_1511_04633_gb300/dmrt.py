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
STREAM_AB, STREAM_INPLACE = 0, 1

HEADER = os.path.join(_build.INCLUDE, "dmrt.h")


class DmrtError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


class dmrt_opts(ctypes.Structure):
    _fields_ = [("storage", ctypes.c_int), ("residual_interval", ctypes.c_int),
                ("rounding", ctypes.c_int), ("streaming", ctypes.c_int),
                ("cells_per_thread", ctypes.c_int), ("pair_loads", ctypes.c_int)]


class dmrt_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("wall_type", ctypes.c_int), ("storage", ctypes.c_int),
                ("residual_interval", ctypes.c_int), ("rounding", ctypes.c_int),
                ("nu", ctypes.c_double), ("alpha", ctypes.c_double), ("gbeta", ctypes.c_double),
                ("tau_nu", ctypes.c_double), ("tau_alpha", ctypes.c_double),
                ("steps", ctypes.c_long), ("streaming", ctypes.c_int),
                ("device_bytes", ctypes.c_longlong), ("cells_per_thread", ctypes.c_int),
                ("pair_loads", ctypes.c_int)]


class dmrt_stats(ctypes.Structure):
    _fields_ = [("step_launches", ctypes.c_long), ("total_launches", ctypes.c_long),
                ("step_ms", ctypes.c_double), ("timed_steps", ctypes.c_long),
                ("bytes_per_cell", ctypes.c_double)]


class dmrt_cavity_desc(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_int * 3), ("Ra", ctypes.c_double), ("Pr", ctypes.c_double),
                ("Ma", ctypes.c_double), ("wall_type", ctypes.c_int)]


class dmrt_surrogate_cfg(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_int), ("depth", ctypes.c_int), ("channels", ctypes.c_int * 4),
                ("storage", ctypes.c_int), ("max_batch", ctypes.c_int), ("seed", ctypes.c_uint)]


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
            "dmrt_nusselt_flux": ([vp, i, P(d)], i),
            "dmrt_nusselt_noalloc": ([vp, i, i, i, i, vp, P(d)], i),
            "dmrt_round_to_storage": ([i, i, vp, vp, ctypes.c_longlong, ctypes.c_uint, vp], i),
            "dmrt_nn_tensor_core_errors": ([i], i),
            "dmrt_residual": ([vp, P(d)], i),
            "dmrt_run_to_steady": ([vp, d, l_, P(l_), P(d)], i),
            "dmrt_set_populations": ([vp, vp, vp, i], i),
            "dmrt_get_populations": ([vp, vp, vp, i], i),
            "dmrt_init_fields": ([vp, vp, vp, vp, i], i),
            "dmrt_get_params": ([vp, P(dmrt_params)], i),
            "dmrt_set_diffusion": ([vp, P(d)], i),
            "dmrt_checkpoint_size": ([vp], ctypes.c_longlong),
            "dmrt_checkpoint_save": ([vp, vp, ctypes.c_longlong], i),
            "dmrt_checkpoint_load": ([vp, vp, ctypes.c_longlong], i),
            "dmrt_set_timing": ([vp, i], i),
            "dmrt_get_stats": ([vp, P(dmrt_stats), i], i),
            "dmrt_last_error": ([vp], ctypes.c_char_p),
            "dmrt_ensemble_create": ([P(vp), i, P(dmrt_cavity_desc), P(dmrt_opts)], i),
            "dmrt_ensemble_destroy": ([vp], None),
            "dmrt_ensemble_set_stream": ([vp, vp], i),
            "dmrt_ensemble_sync": ([vp], i),
            "dmrt_ensemble_set_timing": ([vp, i], i),
            "dmrt_ensemble_get_stats": ([vp, P(dmrt_stats), i], i),
            "dmrt_ensemble_autotune": ([vp, i, ctypes.c_char_p, i], i),
            "dmrt_ensemble_step": ([vp, l_], i),
            "dmrt_ensemble_residual": ([vp, P(d)], i),
            "dmrt_ensemble_run_to_steady": ([vp, d, l_, P(l_), P(i)], i),
            "dmrt_ensemble_nusselt": ([vp, i, P(d)], i),
            "dmrt_ensemble_fields": ([vp, i, vp, vp, vp, i], i),
            "dmrt_ensemble_init_fields": ([vp, i, vp, vp, vp, i], i),
            "dmrt_ensemble_get_populations": ([vp, i, vp, vp, i], i),
            "dmrt_ensemble_member_params": ([vp, i, P(dmrt_params)], i),
            "dmrt_ensemble_last_error": ([vp], ctypes.c_char_p),
            "dmrt_surrogate_create": ([P(vp), P(dmrt_surrogate_cfg)], i),
            "dmrt_surrogate_destroy": ([vp], None),
            "dmrt_surrogate_set_stream": ([vp, vp], i),
            "dmrt_surrogate_param_count": ([vp], ctypes.c_longlong),
            "dmrt_surrogate_get_params": ([vp, P(ctypes.c_float), ctypes.c_longlong], i),
            "dmrt_surrogate_set_params": ([vp, P(ctypes.c_float), ctypes.c_longlong], i),
            "dmrt_surrogate_predict": ([vp, i, P(d), P(i), vp, i], i),
            "dmrt_surrogate_train_step": ([vp, i, P(d), P(i), vp, ctypes.c_float, P(d)], i),
            "dmrt_surrogate_gradients": ([vp, i, P(d), P(i), vp, P(ctypes.c_float), P(d)], i),
            "dmrt_surrogate_loss": ([vp, i, P(d), P(i), vp, P(d)], i),
            "dmrt_surrogate_target_from_fields": ([vp, vp, vp, i, d, vp, vp], i),
            "dmrt_warm_start": ([vp, vp, d, i], i),
            "dmrt_surrogate_last_error": ([vp], ctypes.c_char_p),
            "dmrt_nn_conv3d": ([vp, vp, vp, vp, i, i, i, i, i, i, i, i, vp], i),
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


def check(h, status: int, what: str, ensemble: bool = False, surrogate: bool = False):
    if status != OK:
        L = load()
        name = L.dmrt_status_string(status).decode()
        if h and surrogate:
            msg = L.dmrt_surrogate_last_error(h).decode()
        elif h:
            msg = (L.dmrt_ensemble_last_error(h) if ensemble else L.dmrt_last_error(h)).decode()
        else:
            msg = ""
        raise DmrtError(status, f"{what}: {name} {msg}".strip())


# ---------------------------------------------------------------- C-named functions

def dmrt_create(grid, Ra: float, Pr: float = 0.71, Ma: float = 0.1, wall_type: int = 1,
                storage: int = STORE_F32, residual_interval: int = 0, rounding: int = ROUND_AUTO,
                streaming: int = STREAM_AB, cells_per_thread: int = 0, pair_loads: int = 0):
    L = load()
    h = ctypes.c_void_p()
    g = (ctypes.c_int * 3)(*grid)
    opts = dmrt_opts(storage, residual_interval, rounding, streaming, cells_per_thread, pair_loads)
    check(None, L.dmrt_create_ex(ctypes.byref(h), g, Ra, Pr, Ma, wall_type, ctypes.byref(opts)),
          "dmrt_create")
    return h


def dmrt_create_lattice(grid, nu: float, alpha: float, gbeta: float, wall_type: int = 1,
                        storage: int = STORE_F32, residual_interval: int = 0,
                        rounding: int = ROUND_AUTO, streaming: int = STREAM_AB,
                        cells_per_thread: int = 0, pair_loads: int = 0):
    L = load()
    h = ctypes.c_void_p()
    g = (ctypes.c_int * 3)(*grid)
    opts = dmrt_opts(storage, residual_interval, rounding, streaming, cells_per_thread, pair_loads)
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


def dmrt_nusselt_flux(h, wall: int = 0):
    out = (ctypes.c_double * 3)()
    check(h, load().dmrt_nusselt_flux(h, wall, out), "dmrt_nusselt_flux")
    return tuple(out)


def dmrt_nusselt_local(h, wall, local):
    p, side = _ptr(local)
    check(h, load().dmrt_nusselt_local(h, wall, p, side), "dmrt_nusselt_local")


def dmrt_nusselt_noalloc(theta, wall: int = 0, stream=None):
    """Nusselt numbers of a CUDA float32 tensor theta[z][y][x], computed
    without any device allocation (see include/dmrt.h)."""
    import torch

    p, side = _ptr(theta)
    if side != 1:
        raise TypeError("theta must be a CUDA tensor")
    if theta.dim() != 3:
        raise ValueError("theta must be a 3-D tensor [z][y][x]")
    nz, ny, nx = theta.shape
    raw = getattr(stream, "cuda_stream", stream)
    out = (ctypes.c_double * 3)()
    # the entry point works on the current device: make it theta's
    with torch.cuda.device(theta.device):
        check(None, load().dmrt_nusselt_noalloc(p, nx, ny, nz, wall, raw, out), "dmrt_nusselt_noalloc")
    return tuple(out)


def dmrt_round_to_storage(x, storage: int, rounding: int = ROUND_AUTO, seed: int = 0, out=None,
                          stream=None):
    """Round a CUDA float32 tensor to a population storage format and back
    with the step kernel's rounding; returns `out` (a new tensor if None)."""
    p, side = _ptr(x)
    if side != 1:
        raise TypeError("x must be a CUDA tensor")
    if out is None:
        out = x.new_empty(x.shape)
    q, _ = _ptr(out)
    raw = getattr(stream, "cuda_stream", stream)
    check(None, load().dmrt_round_to_storage(storage, rounding, p, q, x.numel(), seed, raw),
          "dmrt_round_to_storage")
    return out


def dmrt_nn_tensor_core_errors(reset: bool = False) -> int:
    """Launches of the tcgen05 convolution whose bounded wait ran out."""
    return int(load().dmrt_nn_tensor_core_errors(1 if reset else 0))


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


def dmrt_set_diffusion(h, D):
    arr = (ctypes.c_double * 9)(*np.asarray(D, dtype=np.float64).reshape(9).tolist())
    check(h, load().dmrt_set_diffusion(h, arr), "dmrt_set_diffusion")


def dmrt_checkpoint_size(h) -> int:
    return int(load().dmrt_checkpoint_size(h))


def dmrt_checkpoint_save(h) -> bytes:
    n = dmrt_checkpoint_size(h)
    buf = ctypes.create_string_buffer(n)
    check(h, load().dmrt_checkpoint_save(h, buf, n), "dmrt_checkpoint_save")
    return buf.raw


def dmrt_checkpoint_load(h, blob: bytes):
    buf = ctypes.create_string_buffer(bytes(blob), len(blob))
    check(h, load().dmrt_checkpoint_load(h, buf, len(blob)), "dmrt_checkpoint_load")


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
                 storage=STORE_F32, residual_interval=0, rounding=ROUND_AUTO,
                 streaming=STREAM_AB, cells_per_thread=0, pair_loads=0):
        self.grid = tuple(int(v) for v in grid)
        nx, ny, nz = self.grid
        self.shape = (nz, ny, nx)
        self.cells = nx * ny * nz
        if lattice is not None:
            nu, alpha, gbeta = lattice
            self.h = dmrt_create_lattice(self.grid, nu, alpha, gbeta, wall_type, storage,
                                         residual_interval, rounding, streaming, cells_per_thread,
                                         pair_loads)
        else:
            self.h = dmrt_create(self.grid, Ra, Pr, Ma, wall_type, storage, residual_interval,
                                 rounding, streaming, cells_per_thread, pair_loads)

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

    def nusselt_flux(self, wall=0):
        return dmrt_nusselt_flux(self.h, wall)

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

    def set_diffusion(self, D):
        dmrt_set_diffusion(self.h, D)

    def save(self) -> bytes:
        return dmrt_checkpoint_save(self.h)

    def load(self, blob: bytes):
        dmrt_checkpoint_load(self.h, blob)

    def populations(self):
        f = np.empty((19,) + self.shape, np.float32)
        g = np.empty((7,) + self.shape, np.float32)
        dmrt_get_populations(self.h, f, g)
        return f, g

    def init_fields(self, rho, u, theta):
        dmrt_init_fields(self.h, np.ascontiguousarray(rho, np.float32),
                         np.ascontiguousarray(u, np.float32),
                         np.ascontiguousarray(theta, np.float32))


# ---------------------------------------------------------------- ensembles

def _echeck(e, status, what):
    check(e, status, what, ensemble=True)


def dmrt_ensemble_create(cavities, storage: int = STORE_F32, residual_interval: int = 0,
                         rounding: int = ROUND_AUTO, streaming: int = STREAM_AB,
                         cells_per_thread: int = 0):
    """cavities: iterable of dicts {"grid": (nx, ny, nz), "Ra", "Pr", "Ma", "wall"}."""
    L = load()
    cav = list(cavities)
    arr = (dmrt_cavity_desc * len(cav))()
    for k, c in enumerate(cav):
        arr[k].grid[:] = list(c["grid"])
        arr[k].Ra = c["Ra"]
        arr[k].Pr = c.get("Pr", 0.71)
        arr[k].Ma = c.get("Ma", 0.1)
        arr[k].wall_type = c["wall"]
    e = ctypes.c_void_p()
    opts = dmrt_opts(storage, residual_interval, rounding, streaming, cells_per_thread)
    _echeck(None, L.dmrt_ensemble_create(ctypes.byref(e), len(cav), arr, ctypes.byref(opts)),
            "dmrt_ensemble_create")
    return e


def dmrt_ensemble_destroy(e):
    load().dmrt_ensemble_destroy(e)


def dmrt_ensemble_set_stream(e, stream):
    raw = getattr(stream, "cuda_stream", stream)
    _echeck(e, load().dmrt_ensemble_set_stream(e, raw), "dmrt_ensemble_set_stream")


def dmrt_ensemble_sync(e):
    _echeck(e, load().dmrt_ensemble_sync(e), "dmrt_ensemble_sync")


def dmrt_ensemble_set_timing(e, enabled: bool):
    _echeck(e, load().dmrt_ensemble_set_timing(e, int(bool(enabled))), "dmrt_ensemble_set_timing")


def dmrt_ensemble_get_stats(e, reset: bool = False) -> dict:
    s = dmrt_stats()
    _echeck(e, load().dmrt_ensemble_get_stats(e, ctypes.byref(s), int(bool(reset))),
            "dmrt_ensemble_get_stats")
    return {k: getattr(s, k) for k, _ in dmrt_stats._fields_}


def dmrt_ensemble_autotune(e, trials: int = 5) -> str:
    buf = ctypes.create_string_buffer(4096)
    _echeck(e, load().dmrt_ensemble_autotune(e, trials, buf, len(buf)), "dmrt_ensemble_autotune")
    return buf.value.decode()


def dmrt_ensemble_step(e, n: int):
    _echeck(e, load().dmrt_ensemble_step(e, int(n)), "dmrt_ensemble_step")


def dmrt_ensemble_residual(e, count: int) -> np.ndarray:
    r = np.zeros(count)
    _echeck(e, load().dmrt_ensemble_residual(e, r.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
            "dmrt_ensemble_residual")
    return r


def dmrt_ensemble_run_to_steady(e, tol: float, max_steps: int):
    n = ctypes.c_long()
    conv = ctypes.c_int()
    st = load().dmrt_ensemble_run_to_steady(e, tol, int(max_steps), ctypes.byref(n), ctypes.byref(conv))
    if st not in (OK, ERR_TIMEOUT):
        _echeck(e, st, "dmrt_ensemble_run_to_steady")
    return st == OK, n.value, conv.value


def dmrt_ensemble_nusselt(e, count: int, wall: int = 0) -> np.ndarray:
    out = np.zeros((count, 3))
    _echeck(e, load().dmrt_ensemble_nusselt(e, wall, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
            "dmrt_ensemble_nusselt")
    return out


def dmrt_ensemble_fields(e, member: int, rho=None, u=None, theta=None):
    side = _same_side(rho, u, theta)
    _echeck(e, load().dmrt_ensemble_fields(e, member, _ptr(rho)[0], _ptr(u)[0], _ptr(theta)[0], side),
            "dmrt_ensemble_fields")


def dmrt_ensemble_init_fields(e, member: int, rho, u, theta):
    side = _same_side(rho, u, theta)
    _echeck(e, load().dmrt_ensemble_init_fields(e, member, _ptr(rho)[0], _ptr(u)[0], _ptr(theta)[0],
                                                side), "dmrt_ensemble_init_fields")


def dmrt_ensemble_get_populations(e, member: int, f=None, g=None):
    side = _same_side(f, g)
    _echeck(e, load().dmrt_ensemble_get_populations(e, member, _ptr(f)[0], _ptr(g)[0], side),
            "dmrt_ensemble_get_populations")


def dmrt_ensemble_member_params(e, member: int) -> dict:
    p = dmrt_params()
    _echeck(e, load().dmrt_ensemble_member_params(e, member, ctypes.byref(p)),
            "dmrt_ensemble_member_params")
    return {k: getattr(p, k) for k, _ in dmrt_params._fields_}


class Ensemble:
    """Many cavities stepped together, a few launches per time step.  ``cavities`` is a
    list of dicts {"grid": (nx, ny, nz), "Ra": .., "wall": 1..3, ["Pr", "Ma"]}."""

    def __init__(self, cavities, storage=STORE_F32, residual_interval=0, rounding=ROUND_AUTO,
                 streaming=STREAM_AB, cells_per_thread=0):
        self.cavities = [dict(c) for c in cavities]
        self.count = len(self.cavities)
        self.e = dmrt_ensemble_create(self.cavities, storage, residual_interval, rounding, streaming,
                                      cells_per_thread)

    def close(self):
        if getattr(self, "e", None):
            dmrt_ensemble_destroy(self.e)
            self.e = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def cells(self) -> int:
        return sum(int(np.prod(c["grid"])) for c in self.cavities)

    def autotune(self, trials=5):
        return dmrt_ensemble_autotune(self.e, trials)

    def step(self, n=1):
        dmrt_ensemble_step(self.e, n)

    def sync(self):
        dmrt_ensemble_sync(self.e)

    def residual(self):
        return dmrt_ensemble_residual(self.e, self.count)

    def run_to_steady(self, tol, max_steps):
        return dmrt_ensemble_run_to_steady(self.e, tol, max_steps)

    def nusselt(self, wall=0):
        return dmrt_ensemble_nusselt(self.e, self.count, wall)

    def params(self, member):
        return dmrt_ensemble_member_params(self.e, member)

    def fields(self, member):
        nx, ny, nz = self.cavities[member]["grid"]
        shape = (nz, ny, nx)
        rho = np.empty(shape, np.float32)
        u = np.empty((3,) + shape, np.float32)
        th = np.empty(shape, np.float32)
        dmrt_ensemble_fields(self.e, member, rho, u, th)
        return rho, u, th

    def init_fields(self, member, rho, u, theta):
        dmrt_ensemble_init_fields(self.e, member, np.ascontiguousarray(rho, np.float32),
                                  np.ascontiguousarray(u, np.float32),
                                  np.ascontiguousarray(theta, np.float32))

    def populations(self, member):
        nx, ny, nz = self.cavities[member]["grid"]
        shape = (nz, ny, nx)
        f = np.empty((19,) + shape, np.float32)
        g = np.empty((7,) + shape, np.float32)
        dmrt_ensemble_get_populations(self.e, member, f, g)
        return f, g


# ---------------------------------------------------------------- warm-start surrogate

def _scheck(s, status, what):
    check(s, status, what, surrogate=True)


def _samples(ra, wall):
    ra = np.ascontiguousarray(np.atleast_1d(ra), dtype=np.float64)
    wall = np.ascontiguousarray(np.atleast_1d(wall), dtype=np.int32)
    if ra.shape != wall.shape:
        raise ValueError("Ra and wall must have the same length")
    return (len(ra), ra, ra.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), wall,
            wall.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))


def dmrt_surrogate_create(grid: int, depth: int, channels, storage: int = STORE_BF16,
                          max_batch: int = 1, seed: int = 1):
    cfg = dmrt_surrogate_cfg()
    cfg.grid, cfg.depth, cfg.storage, cfg.max_batch, cfg.seed = grid, depth, storage, max_batch, seed
    ch = list(channels) + [0] * (4 - len(channels))
    cfg.channels[:] = ch[:4]
    s = ctypes.c_void_p()
    _scheck(None, load().dmrt_surrogate_create(ctypes.byref(s), ctypes.byref(cfg)), "dmrt_surrogate_create")
    return s


def dmrt_surrogate_destroy(s):
    load().dmrt_surrogate_destroy(s)


def dmrt_surrogate_set_stream(s, stream):
    raw = getattr(stream, "cuda_stream", stream)
    _scheck(s, load().dmrt_surrogate_set_stream(s, raw), "dmrt_surrogate_set_stream")


def dmrt_surrogate_param_count(s) -> int:
    return int(load().dmrt_surrogate_param_count(s))


def dmrt_surrogate_get_params(s) -> np.ndarray:
    n = dmrt_surrogate_param_count(s)
    out = np.empty(n, np.float32)
    _scheck(s, load().dmrt_surrogate_get_params(s, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), n),
            "dmrt_surrogate_get_params")
    return out


def dmrt_surrogate_set_params(s, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    _scheck(s, load().dmrt_surrogate_set_params(s, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), p.size),
            "dmrt_surrogate_set_params")


def dmrt_surrogate_predict(s, ra, wall, out):
    """out: float32 array / tensor [batch][n^3][5] (host or CUDA)."""
    b, _, rp, _, wp = _samples(ra, wall)
    ptr, side = _ptr(out)
    _scheck(s, load().dmrt_surrogate_predict(s, b, rp, wp, ptr, side), "dmrt_surrogate_predict")


def dmrt_surrogate_train_step(s, ra, wall, target, lr: float) -> float:
    """target: CUDA float32 tensor [batch][n^3][5]; returns the batch loss."""
    b, _, rp, _, wp = _samples(ra, wall)
    ptr, side = _ptr(target)
    if side != 1:
        raise TypeError("target must be a CUDA tensor")
    loss = ctypes.c_double()
    _scheck(s, load().dmrt_surrogate_train_step(s, b, rp, wp, ptr, lr, ctypes.byref(loss)),
            "dmrt_surrogate_train_step")
    return loss.value


def dmrt_surrogate_gradients(s, ra, wall, target):
    b, _, rp, _, wp = _samples(ra, wall)
    ptr, side = _ptr(target)
    if side != 1:
        raise TypeError("target must be a CUDA tensor")
    g = np.empty(dmrt_surrogate_param_count(s), np.float32)
    loss = ctypes.c_double()
    _scheck(s, load().dmrt_surrogate_gradients(s, b, rp, wp, ptr, g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                               ctypes.byref(loss)), "dmrt_surrogate_gradients")
    return g, loss.value


def dmrt_surrogate_loss(s, ra, wall, target) -> float:
    b, _, rp, _, wp = _samples(ra, wall)
    ptr, side = _ptr(target)
    if side != 1:
        raise TypeError("target must be a CUDA tensor")
    loss = ctypes.c_double()
    _scheck(s, load().dmrt_surrogate_loss(s, b, rp, wp, ptr, ctypes.byref(loss)), "dmrt_surrogate_loss")
    return loss.value


def dmrt_surrogate_target_from_fields(u, theta, rho, n: int, uc: float, target, stream=None):
    raw = getattr(stream, "cuda_stream", stream)
    st = load().dmrt_surrogate_target_from_fields(_ptr(u)[0], _ptr(theta)[0], _ptr(rho)[0], n, uc,
                                                  _ptr(target)[0], raw)
    check(None, st, "dmrt_surrogate_target_from_fields")


def dmrt_warm_start(h, s, Ra: float, wall: int):
    _scheck(s, load().dmrt_warm_start(h, s, Ra, wall), "dmrt_warm_start")


class Surrogate:
    """The warm-start network (see include/dmrt.h)."""

    def __init__(self, grid=64, depth=3, channels=(16, 32, 64, 128), storage=STORE_BF16, max_batch=1,
                 seed=1):
        self.grid, self.depth, self.channels = grid, depth, tuple(channels)
        self.storage = storage
        self.max_batch = max_batch
        self.s = dmrt_surrogate_create(grid, depth, channels, storage, max_batch, seed)

    def close(self):
        if getattr(self, "s", None):
            dmrt_surrogate_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def param_count(self):
        return dmrt_surrogate_param_count(self.s)

    def params(self):
        return dmrt_surrogate_get_params(self.s)

    def set_params(self, p):
        dmrt_surrogate_set_params(self.s, p)

    def predict(self, ra, wall):
        b = len(np.atleast_1d(ra))
        out = np.empty((b, self.grid ** 3, 5), np.float32)
        dmrt_surrogate_predict(self.s, ra, wall, out)
        return out

    def train_step(self, ra, wall, target, lr):
        return dmrt_surrogate_train_step(self.s, ra, wall, target, lr)

    def gradients(self, ra, wall, target):
        return dmrt_surrogate_gradients(self.s, ra, wall, target)

    def loss(self, ra, wall, target):
        return dmrt_surrogate_loss(self.s, ra, wall, target)

    def warm_start(self, cavity, Ra, wall):
        h = cavity.h if hasattr(cavity, "h") else cavity
        dmrt_warm_start(h, self.s, Ra, wall)


def dmrt_nn_conv3d(x, w, bias, y, batch, n, cin, cout, k, act=0, storage=STORE_BF16, stream=None):
    """One surrogate convolution on CUDA tensors (see include/dmrt.h)."""
    raw = getattr(stream, "cuda_stream", stream)
    out_f32 = 1 if str(y.dtype) == "torch.float32" else 0
    bp = None if bias is None else bias.data_ptr()
    check(None, load().dmrt_nn_conv3d(x.data_ptr(), w.data_ptr(), bp, y.data_ptr(), batch, n, cin, cout,
                                      k, act, storage, out_f32, raw), "dmrt_nn_conv3d")
