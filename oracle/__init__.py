"""FP64 CPU oracle of the double-MRT thermal LBM (arXiv:1511.04633).

TEST INFRASTRUCTURE ONLY.  This package is the independent reference the CUDA
library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it; the library never does, and
it shares no code with the CUDA path.

The arithmetic lives in ``dmrt_oracle.c`` (plain C, FP64, dense matrices, one
function per step of the method, each citing the paper's equation).  This file
only compiles it with gcc and marshals arrays through ctypes.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dmrt_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

Q19, Q7 = 19, 7


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, -O2, OpenMP,
    no FMA contraction so x86 and Arm give the same bits)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.POINTER(ctypes.c_double)
            IP = ctypes.POINTER(ctypes.c_int)
            vp = ctypes.c_void_p
            L.orc_create.restype = vp
            L.orc_create.argtypes = [ctypes.c_int] * 4 + [ctypes.c_double] * 3
            L.orc_destroy.argtypes = [vp]
            L.orc_set_options.argtypes = [vp, ctypes.c_double, ctypes.c_int]
            L.orc_set_rates.argtypes = [vp, P, P]
            L.orc_get_rates.argtypes = [vp, P, P]
            L.orc_set_diffusion.restype = ctypes.c_int
            L.orc_set_diffusion.argtypes = [vp, P]
            L.orc_steps.restype = ctypes.c_long
            L.orc_steps.argtypes = [vp]
            L.orc_set_populations.argtypes = [vp, P, P]
            L.orc_get_populations.argtypes = [vp, P, P]
            L.orc_init_fields.argtypes = [vp, P, P, P]
            L.orc_collide.argtypes = [vp, P, P, P, P]
            L.orc_step.argtypes = [vp, ctypes.c_long]
            L.orc_fields.argtypes = [vp, P, P, P]
            L.orc_nusselt.restype = ctypes.c_int
            L.orc_nusselt.argtypes = [vp, ctypes.c_int, P, P]
            L.orc_nusselt_flux.restype = ctypes.c_int
            L.orc_nusselt_flux.argtypes = [vp, ctypes.c_int, P, P]
            L.orc_nusselt_from_theta.restype = ctypes.c_int
            L.orc_nusselt_from_theta.argtypes = [P] + [ctypes.c_int] * 4 + [P, P]
            L.orc_residual.restype = ctypes.c_double
            L.orc_residual.argtypes = [P, P, P, P, ctypes.c_long, ctypes.c_int]
            L.orc_invert.restype = ctypes.c_int
            L.orc_invert.argtypes = [P, ctypes.c_int, P]
            L.orc_matrix_M.argtypes = [P, ctypes.c_int]
            L.orc_matrix_N.argtypes = [P]
            L.orc_velocities19.argtypes = [IP]
            L.orc_weights19.argtypes = [P]
            L.orc_velocities7.argtypes = [IP]
            L.orc_weights7.argtypes = [P]
            L.orc_feq.argtypes = [ctypes.c_double, P, P]
            L.orc_meq.argtypes = [ctypes.c_double, P, ctypes.c_double, P]
            L.orc_neq.argtypes = [ctypes.c_double, P, P]
            L.orc_force.argtypes = [ctypes.c_double, P, P, P]
            L.orc_lattice_from_physics.argtypes = [ctypes.c_int] + [ctypes.c_double] * 3 + [P]
            _lib = L
    return _lib


# ---------------------------------------------------------------- pure functions

def matrix_M(printed: bool = False) -> np.ndarray:
    """Eq. (21); ``printed=True`` returns it exactly as printed (singular)."""
    out = np.zeros((Q19, Q19))
    lib().orc_matrix_M(_d(out), int(printed))
    return out


def matrix_N() -> np.ndarray:
    """Eq. (32)."""
    out = np.zeros((Q7, Q7))
    lib().orc_matrix_N(_d(out))
    return out


def invert(A: np.ndarray) -> np.ndarray:
    """The oracle's own Gauss-Jordan inverse."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    out = np.zeros_like(A)
    rc = lib().orc_invert(_d(A), A.shape[0], _d(out))
    if rc != 0:
        raise np.linalg.LinAlgError("singular")
    return out


def velocities19() -> np.ndarray:
    out = np.zeros((Q19, 3), dtype=np.int32)
    lib().orc_velocities19(out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return out


def weights19() -> np.ndarray:
    out = np.zeros(Q19)
    lib().orc_weights19(_d(out))
    return out


def velocities7() -> np.ndarray:
    out = np.zeros((Q7, 3), dtype=np.int32)
    lib().orc_velocities7(out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return out


def weights7() -> np.ndarray:
    out = np.zeros(Q7)
    lib().orc_weights7(_d(out))
    return out


def feq(rho: float, V) -> np.ndarray:
    """Eq. (17)."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    out = np.zeros(Q19)
    lib().orc_feq(rho, _d(V), _d(out))
    return out


def meq(rho: float, j, rho0: float = 1.0) -> np.ndarray:
    """Eq. (24)."""
    j = np.ascontiguousarray(j, dtype=np.float64)
    out = np.zeros(Q19)
    lib().orc_meq(rho, _d(j), rho0, _d(out))
    return out


def neq(T: float, V) -> np.ndarray:
    """Eq. (33)."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    out = np.zeros(Q7)
    lib().orc_neq(T, _d(V), _d(out))
    return out


def force(rho: float, V, G) -> np.ndarray:
    """Eq. (15)."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    G = np.ascontiguousarray(G, dtype=np.float64)
    out = np.zeros(Q19)
    lib().orc_force(rho, _d(V), _d(G), _d(out))
    return out


def lattice_from_physics(H: int, Ra: float, Pr: float, Ma: float):
    """Eq. (38): returns (nu, alpha, g*beta) in lattice units."""
    out = np.zeros(3)
    lib().orc_lattice_from_physics(int(H), Ra, Pr, Ma, _d(out))
    return float(out[0]), float(out[1]), float(out[2])


def nusselt_from_theta(theta: np.ndarray, wall: int = 0):
    """Eqs. (39)-(41) on a theta field shaped [z][y][x].
    Returns ((Nu_3D, Nu_2D, Nu_max), local[z][x])."""
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    nz, ny, nx = theta.shape
    out = np.zeros(3)
    local = np.zeros((nz, nx))
    rc = lib().orc_nusselt_from_theta(_d(theta), nx, ny, nz, wall, _d(out), _d(local))
    if rc != 0:
        raise ValueError("nusselt needs ny >= 2")
    return tuple(float(v) for v in out), local


def residual(th_now, u_now, th_prev, u_prev, K: int) -> float:
    """Reading A11 of the convergence residual."""
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (th_now, u_now, th_prev, u_prev)]
    return float(lib().orc_residual(*[_d(a) for a in arrs], arrs[0].size, int(K)))


# ---------------------------------------------------------------- stateful solver

class Oracle:
    """An FP64 cavity: populations [q][z][y][x]; wall 0 = periodic, 1..3 = Types."""

    def __init__(self, grid, wall: int, nu: float, alpha: float, gbeta: float):
        nx, ny, nz = (int(v) for v in grid)
        self.grid = (nx, ny, nz)
        self.shape = (nz, ny, nx)
        self.cells = nx * ny * nz
        self.wall = wall
        self._h = lib().orc_create(nx, ny, nz, wall, nu, alpha, gbeta)
        if not self._h:
            raise ValueError("orc_create failed")

    @classmethod
    def physical(cls, grid, wall: int, Ra: float, Pr: float = 0.71, Ma: float = 0.1):
        nu, alpha, gbeta = lattice_from_physics(grid[1], Ra, Pr, Ma)
        return cls(grid, wall, nu, alpha, gbeta)

    def close(self):
        if self._h:
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_options(self, theta_ref: float = 0.0, rho0_local: bool = False):
        lib().orc_set_options(self._h, theta_ref, int(rho0_local))

    def rates(self):
        s = np.zeros(Q19)
        q = np.zeros(Q7)
        lib().orc_get_rates(self._h, _d(s), _d(q))
        return s, q

    def set_rates(self, s, q):
        s = np.ascontiguousarray(s, dtype=np.float64)
        q = np.ascontiguousarray(q, dtype=np.float64)
        lib().orc_set_rates(self._h, _d(s), _d(q))

    def set_diffusion(self, D):
        """Eqs. (35)-(37) with a general (anisotropic) diffusion tensor D."""
        D = np.ascontiguousarray(D, dtype=np.float64).reshape(9)
        if lib().orc_set_diffusion(self._h, _d(D)) != 0:
            raise np.linalg.LinAlgError("singular relaxation matrix")

    @property
    def steps(self) -> int:
        return int(lib().orc_steps(self._h))

    def set_populations(self, f, g):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(Q19, *self.shape)
        g = np.ascontiguousarray(g, dtype=np.float64).reshape(Q7, *self.shape)
        lib().orc_set_populations(self._h, _d(f), _d(g))

    def populations(self):
        f = np.zeros((Q19,) + self.shape)
        g = np.zeros((Q7,) + self.shape)
        lib().orc_get_populations(self._h, _d(f), _d(g))
        return f, g

    def init_fields(self, rho, u, T):
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(self.shape)
        u = np.ascontiguousarray(u, dtype=np.float64).reshape((3,) + self.shape)
        T = np.ascontiguousarray(T, dtype=np.float64).reshape(self.shape)
        lib().orc_init_fields(self._h, _d(rho), _d(u), _d(T))

    def collide(self, fin, gin):
        fin = np.ascontiguousarray(fin, dtype=np.float64)
        gin = np.ascontiguousarray(gin, dtype=np.float64)
        fo = np.zeros(Q19)
        go = np.zeros(Q7)
        lib().orc_collide(self._h, _d(fin), _d(gin), _d(fo), _d(go))
        return fo, go

    def step(self, n: int = 1):
        lib().orc_step(self._h, int(n))

    def fields(self):
        """(rho[z,y,x], u[3,z,y,x], T[z,y,x]) of the pulled populations."""
        rho = np.zeros(self.shape)
        u = np.zeros((3,) + self.shape)
        T = np.zeros(self.shape)
        lib().orc_fields(self._h, _d(rho), _d(u), _d(T))
        return rho, u, T

    def nusselt_flux(self, wall: int = 0):
        """Link-flux Nusselt numbers ((Nu_3D, Nu_2D, Nu_max), local[z][x])."""
        out = np.zeros(3)
        local = np.zeros((self.shape[0], self.shape[2]))
        rc = lib().orc_nusselt_flux(self._h, wall, _d(out), _d(local))
        if rc != 0:
            raise ValueError("nusselt_flux needs walls")
        return tuple(float(v) for v in out), local

    def nusselt(self, wall: int = 0):
        """((Nu_3D, Nu_2D, Nu_max), local[z][x])."""
        out = np.zeros(3)
        local = np.zeros((self.shape[0], self.shape[2]))
        rc = lib().orc_nusselt(self._h, wall, _d(out), _d(local))
        if rc != 0:
            raise ValueError("nusselt failed")
        return tuple(float(v) for v in out), local
