"""FP64 CPU oracle of the D2Q9 lid-driven cavity method (Xiang & Shi, arXiv 2211.05009).

TEST INFRASTRUCTURE ONLY.  This package is what the CUDA library is checked against.  Only the
test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import it;
the CUDA library never does, and the two share no code.  The arithmetic lives in the plain C
file ``lbm_oracle.c`` (FP64, AoS, one node at a time, ``-ffp-contract=off``); this module
compiles it with gcc and wraps it with ctypes and numpy.

Every function follows a passage of the paper:
  feq                  Eq. 2 (Sec. 2.1)
  step / step_node     Eq. 1 streaming + Sec. 2.2 (ii) non-equilibrium extrapolation + Eq. 1 BGK
  init                 Sec. 2.2 (i)
  moments              Eq. 3
  residual             Eq. 6 (Sec. 2.2 iii)
  stream_function      the Psi values and vortex centres of Table 1 / Table 2
Test-only modes (bounce-back cavity, periodic box, NEE channel with a Guo body force) are not
in the paper; they exist so closed-form flows can pin the oracle.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liblbm_oracle.so")
_OMP_PATH = os.path.join(_HERE, "liblbm_oracle_omp.so")  # the same source with -fopenmp

CAVITY_NEE, CAVITY_BB, PERIODIC, CHANNEL_NEE = 0, 1, 2, 3


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("tau", ctypes.c_double),
        ("U", ctypes.c_double),
        ("mode", ctypes.c_int),
        ("corner_moving", ctypes.c_int),
        ("Fx", ctypes.c_double),
        ("Fy", ctypes.c_double),
    ]


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile lbm_oracle.c into liblbm_oracle.so next to it (gcc, -O2, no FMA contraction).

    openmp=True builds the same source with -fopenmp into liblbm_oracle_omp.so: the node loops of
    a time step run on all host cores, with bitwise the same result (every node's arithmetic is
    unchanged).  It exists to time the oracle on all cores; the tests check it equals the plain
    build."""
    path = _OMP_PATH if openmp else _LIB_PATH
    if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
        tmp = path + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
             "-std=c11", *(["-fopenmp"] if openmp else []), "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, path)
    return path


_lib = None
_lib_omp = None


def _L(openmp: bool = False):
    global _lib, _lib_omp
    if openmp:
        if _lib_omp is None:
            _lib_omp = _bind(ctypes.CDLL(build(openmp=True)))
        return _lib_omp
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _bind(lib):
    dp = ctypes.POINTER(ctypes.c_double)
    pp = ctypes.POINTER(_Params)
    ip = ctypes.POINTER(ctypes.c_int)
    lib.orc_feq.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
    lib.orc_step.argtypes = [pp, dp, dp]
    lib.orc_step_node.argtypes = [pp, dp, ctypes.c_int, ctypes.c_int, dp]
    lib.orc_init.argtypes = [pp, dp]
    lib.orc_init_moments.argtypes = [pp, dp, dp, dp, dp]
    lib.orc_init_moments_neq.argtypes = [pp, dp, dp, dp, dp]
    lib.orc_moments.argtypes = [pp, dp, dp, dp, dp]
    lib.orc_residual.argtypes = [ctypes.c_size_t, dp, dp, dp, dp]
    lib.orc_residual.restype = ctypes.c_double
    lib.orc_mass.argtypes = [pp, dp]
    lib.orc_mass.restype = ctypes.c_double
    lib.orc_stream_function.argtypes = [pp, dp, dp, dp, ip, ip, dp, ip, ip]
    lib.orc_run.argtypes = [pp, dp, dp, ctypes.c_long]
    lib.orc_run.restype = ctypes.c_int
    lib.orc_threads.argtypes = []
    lib.orc_threads.restype = ctypes.c_int
    return lib


def threads(openmp: bool = False) -> int:
    """Host threads the time step of the plain (1) or the OpenMP build uses."""
    return _L(openmp).orc_threads()


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class Params:
    """Problem statement: nx x ny nodes (walls included), relaxation time tau, lid speed U."""

    nx: int
    ny: int
    tau: float
    U: float = 0.1
    mode: int = CAVITY_NEE
    corner_moving: bool = False
    Fx: float = 0.0
    Fy: float = 0.0

    @staticmethod
    def from_re(nx: int, ny: int, Re: float, U: float, **kw) -> "Params":
        """Re = U L / nu with L = nx (Sec. 1) and nu = (tau - 1/2)/3 (Eq. 5, dt = dx = 1)."""
        nu = U * nx / Re
        return Params(nx, ny, 3.0 * nu + 0.5, U, **kw)

    def c(self) -> _Params:
        return _Params(self.nx, self.ny, self.tau, self.U, self.mode, int(self.corner_moving),
                       self.Fx, self.Fy)


def feq(rho: float, ux: float, uy: float) -> np.ndarray:
    out = np.zeros(9)
    _L().orc_feq(rho, ux, uy, _dp(out))
    return out


def init(p: Params) -> np.ndarray:
    """Initial post-collision field f = f^eq(1, u0) as [ny, nx, 9] (Sec. 2.2 i)."""
    f = np.zeros((p.ny, p.nx, 9))
    _L().orc_init(ctypes.byref(p.c()), _dp(f))
    return f


def init_moments(p: Params, rho, ux, uy) -> np.ndarray:
    rho, ux, uy = (np.ascontiguousarray(a, dtype=np.float64) for a in (rho, ux, uy))
    f = np.zeros((p.ny, p.nx, 9))
    _L().orc_init_moments(ctypes.byref(p.c()), _dp(rho), _dp(ux), _dp(uy), _dp(f))
    return f


def init_moments_neq(p: Params, rho, ux, uy) -> np.ndarray:
    """f^eq(rho, u) plus (1 - 1/tau) times the first-order Chapman-Enskog non-equilibrium part
    built from the velocity gradients (not in the paper; a consistent warm start)."""
    rho, ux, uy = (np.ascontiguousarray(a, dtype=np.float64) for a in (rho, ux, uy))
    f = np.zeros((p.ny, p.nx, 9))
    _L().orc_init_moments_neq(ctypes.byref(p.c()), _dp(rho), _dp(ux), _dp(uy), _dp(f))
    return f


def step(p: Params, f: np.ndarray, openmp: bool = False) -> np.ndarray:
    """One time step; returns the new post-collision field (openmp: the all-core build)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(f)
    _L(openmp).orc_step(ctypes.byref(p.c()), _dp(f), _dp(out))
    return out


def step_node(p: Params, f: np.ndarray, x: int, y: int) -> np.ndarray:
    """The value step() would store at node (x, y), computed from f alone."""
    out = np.zeros(9)
    _L().orc_step_node(ctypes.byref(p.c()), _dp(f), int(x), int(y), _dp(out))
    return out


def run(p: Params, f: np.ndarray, n: int, openmp: bool = False) -> np.ndarray:
    """n time steps from f; returns the new field (f is not modified).  openmp=True runs the
    OpenMP build of the same source (all host cores, bitwise the same result)."""
    f = np.array(f, dtype=np.float64, order="C", copy=True)
    tmp = np.empty_like(f)
    rc = _L(openmp).orc_run(ctypes.byref(p.c()), _dp(f), _dp(tmp), int(n))
    if rc:
        raise FloatingPointError("oracle: non-finite population")
    return f


def moments(p: Params, f: np.ndarray):
    """(rho, ux, uy), each [ny, nx], of a post-collision field (Eq. 3)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    rho, ux, uy = (np.zeros((p.ny, p.nx)) for _ in range(3))
    _L().orc_moments(ctypes.byref(p.c()), _dp(f), _dp(rho), _dp(ux), _dp(uy))
    return rho, ux, uy


def residual(ux1, uy1, ux0, uy0) -> float:
    """Eq. 6 between two velocity fields."""
    a = [np.ascontiguousarray(v, dtype=np.float64).ravel() for v in (ux1, uy1, ux0, uy0)]
    return _L().orc_residual(a[0].size, *(_dp(v) for v in a))


def mass(p: Params, f: np.ndarray) -> float:
    f = np.ascontiguousarray(f, dtype=np.float64)
    return _L().orc_mass(ctypes.byref(p.c()), _dp(f))


def stream_function(p: Params, ux: np.ndarray):
    """Psi [ny, nx] (u_x = dPsi/dy, Psi = 0 on the bottom wall) and its extrema.

    Returns (psi, (psi_min, i_min, j_min), (psi_max, i_max, j_max)).
    """
    ux = np.ascontiguousarray(ux, dtype=np.float64)
    psi = np.zeros((p.ny, p.nx))
    vmin, vmax = ctypes.c_double(), ctypes.c_double()
    imin, jmin, imax, jmax = (ctypes.c_int() for _ in range(4))
    _L().orc_stream_function(ctypes.byref(p.c()), _dp(ux), _dp(psi), ctypes.byref(vmin),
                             ctypes.byref(imin), ctypes.byref(jmin), ctypes.byref(vmax),
                             ctypes.byref(imax), ctypes.byref(jmax))
    return psi, (vmin.value, imin.value, jmin.value), (vmax.value, imax.value, jmax.value)


def to_soa(f: np.ndarray) -> np.ndarray:
    """[ny, nx, 9] -> [9, ny, nx] (the layout the C ABI exchanges)."""
    return np.ascontiguousarray(np.moveaxis(f, 2, 0))


def from_soa(f: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(np.moveaxis(f, 0, 2))
