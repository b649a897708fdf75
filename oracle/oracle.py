"""ctypes binding of the FP64 CPU oracle (``sgpe_oracle.c``).

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this module. The CUDA product path
never imports it and shares no code with it.

The oracle follows arXiv:2009.13507: Sec. 2 (Eqs. (1)-(2), the SO terms, the
normalisation Eq. (noma), the energy Eq. (energy)), Sec. 3 (the split-step
Crank-Nicolson modules SO, CALCNU, HERM, LU/LUX/LUY, RENORM, ENERGY) and
Appendix A (Eqs. (nu), (11), (p1), (p2), (DJ), (DJ2)). See the C source for
the per-function citations.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sgpe_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

OBS_NAMES = (
    "N+", "N0", "N-", "N", "mag", "E", "mu", "rms+", "rms0", "rms-", "rms",
    "E_kin", "E_trap", "E_int", "E_rabi", "E_so",
)

SUBSTEP = {"so": 0, "calcnu": 1, "herm": 2, "cn_x": 3, "cn_y": 4, "renorm": 5, "so_cn": 6, "so_cn_rev": 7}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, FP64, no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-std=gnu99", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
               "-fcx-fortran-rules", "-fopenmp", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double),
        ("c0", ctypes.c_double), ("c2", ctypes.c_double),
        ("so_type", ctypes.c_int),
        ("gamma", ctypes.c_double), ("omega", ctypes.c_double),
        ("wx", ctypes.c_double), ("wy", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("renorm", ctypes.c_int), ("mag", ctypes.c_double),
        ("split", ctypes.c_int), ("so_mode", ctypes.c_int),
    ]


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER(_Params)
        C = ctypes.c_void_p
        lib.orc_step.argtypes = [P, C, ctypes.c_int, ctypes.c_int, C]
        lib.orc_substep.argtypes = [P, C, ctypes.c_int, ctypes.c_int, ctypes.c_double]
        lib.orc_substep.restype = ctypes.c_int
        lib.orc_observables.argtypes = [P, C, ctypes.c_double, C]
        lib.orc_apply_hso.argtypes = [P, C, C]
        lib.orc_norms.argtypes = [P, C, C]
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_get_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def set_threads(n: int) -> int:
    """Threads for the oracle's point and line loops (n <= 0: all cores the
    process may use); results do not depend on it. Returns the count in use."""
    lib = _load()
    if n <= 0 and hasattr(os, "sched_getaffinity"):
        n = len(os.sched_getaffinity(0))
    lib.orc_set_threads(int(n))
    return int(lib.orc_get_threads())


def get_threads() -> int:
    return int(_load().orc_get_threads())


@dataclass
class Problem:
    """Grid and physical parameters (the paper's Table 2 inputs)."""
    dim: int
    nx: int
    ny: int = 1
    dx: float = 0.05
    dy: float = 0.05
    c0: float = 0.0
    c2: float = 0.0
    so_type: int = 0
    gamma: float = 0.0
    omega: float = 0.0
    wx: float = 1.0
    wy: float = 1.0
    dt: float = 1e-4
    renorm: int = 1
    mag: float = 0.0
    split: int = 0      # 0 Lie, 1 Strang
    so_mode: int = 0    # 0 explicit Euler SO, 1 Crank-Nicolson SO

    def _c(self) -> _Params:
        return _Params(self.dim, self.nx, self.ny if self.dim == 2 else 1, self.dx, self.dy,
                       self.c0, self.c2, self.so_type, self.gamma, self.omega, self.wx, self.wy,
                       self.dt, self.renorm, self.mag, self.split, self.so_mode)

    @property
    def shape(self):
        return (3, self.ny if self.dim == 2 else 1, self.nx)


def _state(prob: Problem, psi) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(psi, dtype=np.complex128).reshape(prob.shape)).copy()
    return a


def step(prob: Problem, psi, nsteps: int, imag: bool, omega_t=None) -> np.ndarray:
    """Advance ``psi`` ([3][ny][nx] complex128) by ``nsteps`` full split steps; returns a new array."""
    lib = _load()
    a = _state(prob, psi)
    p = prob._c()
    om = None
    if omega_t is not None:
        om = np.ascontiguousarray(np.asarray(omega_t, dtype=np.float64))
        assert om.size >= nsteps
    lib.orc_step(ctypes.byref(p), a.ctypes.data, int(nsteps), int(bool(imag)),
                 om.ctypes.data if om is not None else None)
    return a


def substep(prob: Problem, psi, which: str, imag: bool, omega=None) -> np.ndarray:
    """Apply one substep ('so', 'calcnu', 'herm', 'cn_x', 'cn_y', 'renorm', 'so_cn', 'so_cn_rev')."""
    lib = _load()
    a = _state(prob, psi)
    p = prob._c()
    rc = lib.orc_substep(ctypes.byref(p), a.ctypes.data, SUBSTEP[which], int(bool(imag)),
                         float(prob.omega if omega is None else omega))
    assert rc == 0
    return a


def apply_hso(prob: Problem, psi) -> np.ndarray:
    lib = _load()
    a = _state(prob, psi)
    out = np.zeros_like(a)
    lib.orc_apply_hso(ctypes.byref(prob._c()), a.ctypes.data, out.ctypes.data)
    return out


def observables(prob: Problem, psi, omega=None) -> dict:
    lib = _load()
    a = _state(prob, psi)
    out = np.zeros(16, dtype=np.float64)
    lib.orc_observables(ctypes.byref(prob._c()), a.ctypes.data,
                        float(prob.omega if omega is None else omega), out.ctypes.data)
    return dict(zip(OBS_NAMES, out.tolist()))


def observables_array(prob: Problem, psi, omega=None) -> np.ndarray:
    o = observables(prob, psi, omega)
    return np.array([o[k] for k in OBS_NAMES])
