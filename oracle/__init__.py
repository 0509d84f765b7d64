"""FP64 CPU oracle for the HDM pseudopotential lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg may import this package; the product library never does.  It
shares no code with the CUDA path.  The arithmetic lives in ``lbm_oracle.c``
(plain C, FP64, no FMA contraction); this module compiles it with gcc on first
use and marshals numpy arrays through ctypes.

Paper: Qin, Zhao, Chen, Zhang & Wen, arXiv:1712.06079.  Each wrapper names the
equation it follows.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None

EOS = {"vdw": 0, "cs": 1, "pr": 2, "rk": 3, "rks": 4, "psi": 5}
FORCE = {"sc": 0, "zc": 1}
GRAD = {"hdm": 0, "cdm": 1}

# D2Q9 ordering used by the oracle's state arrays (Eq. 2; the paper does not
# print the ordering): rest, +x, +y, -x, -y, (+,+), (-,+), (-,-), (+,-).
EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


def build(force: bool = False) -> str:
    """Compile ``lbm_oracle.c`` into ``_build/liblbm_oracle.so`` (gcc, -O2,
    OpenMP, -ffp-contract=off so no FMA contraction changes the rounding)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu99", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


class _Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("eos", ctypes.c_int),
                ("force", ctypes.c_int), ("grad", ctypes.c_int), ("walls", ctypes.c_int),
                ("a", ctypes.c_double), ("b", ctypes.c_double), ("R", ctypes.c_double),
                ("omega", ctypes.c_double), ("T", ctypes.c_double), ("Tc", ctypes.c_double),
                ("k", ctypes.c_double), ("tau", ctypes.c_double), ("G", ctypes.c_double),
                ("rho0", ctypes.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(_Params)
            D = ctypes.POINTER(ctypes.c_double)
            lib.orc_critical_point.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double, D, D]
            lib.orc_maxwell.argtypes = [P, D, D, D]
            lib.orc_p_eos.argtypes = [P, D, D, D, ctypes.c_int]
            lib.orc_feq.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, D]
            lib.orc_hdm_line.argtypes = [D, D, ctypes.c_int]
            lib.orc_hdm_grad.argtypes = [D, D, D, ctypes.c_int, ctypes.c_int]
            lib.orc_cdm_grad.argtypes = [D, D, D, ctypes.c_int, ctypes.c_int]
            lib.orc_force.argtypes = [P, D, D, D]
            lib.orc_grad.argtypes = [P, D, D, D]
            lib.orc_init.argtypes = [P, D, D, D, D]
            lib.orc_step.argtypes = [P, D, D]
            lib.orc_run.argtypes = [P, D, ctypes.c_int]
            lib.orc_moments.argtypes = [P, D, D, D, D]
            lib.orc_flat_profile.argtypes = [P, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, D, D]
            lib.orc_cs_run.argtypes = [P, D, D, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int, D, D]
            lib.orc_set_threads.argtypes = [ctypes.c_int]
            lib.orc_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def max_threads() -> int:
    return int(_load().orc_max_threads())


@dataclasses.dataclass
class Params:
    """Model parameters.  ``T`` is the absolute temperature; build it from a
    reduced temperature with :func:`params_at` (T = Tr * Tc)."""
    nx: int
    ny: int
    eos: str = "cs"
    a: float = 1.0
    b: float = 4.0
    R: float = 1.0
    omega: float = 0.0
    T: float = 0.0
    Tc: float = 0.0
    k: float = 1.0
    tau: float = 1.0
    force: str = "sc"
    grad: str = "hdm"
    G: float = 0.0       # eos "psi": interaction strength of Eq. 4
    rho0: float = 1.0    # eos "psi": reference density of the effective mass
    walls: bool = False  # no-slip walls below row 0 and above row ny-1 (Sec. 5.5); else periodic in y

    def c(self) -> _Params:
        return _Params(self.nx, self.ny, EOS[self.eos], FORCE[self.force], GRAD[self.grad], int(self.walls),
                       self.a, self.b, self.R, self.omega, self.T, self.Tc, self.k, self.tau, self.G, self.rho0)


def critical_point(eos: str, a: float, b: float, R: float = 1.0):
    """(Tc, rho_c): maximum of the spinodal temperature over rho.  PR and RKS
    use alpha = 1 (its value at Tc); RK uses alpha = 1/sqrt(T) (Eq. 27)."""
    Tc, rc = ctypes.c_double(), ctypes.c_double()
    rc_ = _load().orc_critical_point(EOS[eos], a, b, R, ctypes.byref(Tc), ctypes.byref(rc))
    if rc_ != 0:
        raise RuntimeError("critical point not found")
    return Tc.value, rc.value


def params_at(nx, ny, eos, a, b, Tr, *, R=1.0, omega=0.0, k=1.0, tau=1.0,
              force="sc", grad="hdm", walls=False) -> Params:
    Tc, _ = critical_point(eos, a, b, R)
    return Params(nx, ny, eos, a, b, R, omega, Tr * Tc, Tc, k, tau, force, grad, walls=walls)


def params_psi(nx, ny, G, *, rho0=1.0, tau=1.0, force="sc", grad="hdm") -> Params:
    """The original Shan-Chen model (Eq. 4-5): effective mass psi = 1 - exp(-rho/rho0),
    interaction strength G; no equation of state, temperature or Hu factor."""
    return Params(nx, ny, "psi", tau=tau, force=force, grad=grad, G=G, rho0=rho0)


def maxwell(p: Params):
    """Maxwell equal-area coexistence densities (rho_g, rho_l, p_sat) of the
    unscaled EOS at p.T (Sec. 5.2)."""
    g, l, s = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    if _load().orc_maxwell(ctypes.byref(p.c()), ctypes.byref(g), ctypes.byref(l), ctypes.byref(s)):
        raise RuntimeError("no van der Waals loop at this temperature")
    return g.value, l.value, s.value


def flat_profile(p: Params, kappa: float, h: float, n: int, i0: int | None = None, sub: int = 64):
    """Equilibrium density profile across a flat interface (Sec. 5.1): Eq. 26
    with the pressure tensor of Eq. 25 for the unscaled EOS at p.T, integrated
    through its first integral (kappa/2) rho'^2 = W(rho).  Returns (y, rho,
    drho/dy) at y_i = (i - i0) h, rising from rho_g to rho_l, y = 0 at the mean
    of the two Maxwell densities (i0 = n // 2 by default)."""
    i0 = n // 2 if i0 is None else int(i0)
    rho, drho = np.empty(n), np.empty(n)
    if _load().orc_flat_profile(ctypes.byref(p.c()), float(kappa), float(h), int(n), i0, int(sub),
                                _ptr(rho), _ptr(drho)):
        raise RuntimeError("no van der Waals loop at this temperature, or invalid arguments")
    return (np.arange(n) - i0) * h, rho, drho


def p_eos(p: Params, rho):
    """(p_EOS, dp_EOS/drho) at p.T, without the Hu factor k."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    out = np.empty_like(rho)
    dout = np.empty_like(rho)
    _load().orc_p_eos(ctypes.byref(p.c()), _ptr(rho.ravel()), _ptr(out.ravel()),
                      _ptr(dout.ravel()), rho.size)
    return out, dout


def feq(rho: float, ux: float, uy: float) -> np.ndarray:
    """Equilibrium distribution of Eq. 2."""
    out = np.empty(9)
    _load().orc_feq(rho, ux, uy, _ptr(out))
    return out


def hdm_line(u) -> np.ndarray:
    """Periodic HDM derivative of Eq. 20 (h = 1) by the cyclic Thomas solve."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    d = np.empty_like(u)
    _load().orc_hdm_line(_ptr(u), _ptr(d), u.size)
    return d


def hdm_grad(q):
    """(d/dx, d/dy) of a (ny, nx) field by Eq. 20 along rows and columns."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    gx, gy = np.empty_like(q), np.empty_like(q)
    _load().orc_hdm_grad(_ptr(q), _ptr(gx), _ptr(gy), q.shape[1], q.shape[0])
    return gx, gy


def cdm_grad(q):
    """(d/dx, d/dy) of a (ny, nx) field by Eq. 15 scaled by 1/c_s^2."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    gx, gy = np.empty_like(q), np.empty_like(q)
    _load().orc_cdm_grad(_ptr(q), _ptr(gx), _ptr(gy), q.shape[1], q.shape[0])
    return gx, gy


def grad(p: Params, q):
    """(d/dx, d/dy) of a (ny, nx) field as the step of p takes it: HDM (Eq. 20)
    or CDM (Eq. 15), periodic, or with p.walls the field mirrored across the
    walls (Eq. 20 on the mirrored column of period 2 ny)."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    gx, gy = np.empty_like(q), np.empty_like(q)
    _load().orc_grad(ctypes.byref(p.c()), _ptr(q), _ptr(gx), _ptr(gy))
    return gx, gy


def force(p: Params, rho):
    """Interaction force (Eq. 22 for SC, Eq. 7 for ZC) of a density field."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    Fx, Fy = np.empty_like(rho), np.empty_like(rho)
    _load().orc_force(ctypes.byref(p.c()), _ptr(rho), _ptr(Fx), _ptr(Fy))
    return Fx, Fy


def init(p: Params, rho, ux=None, uy=None) -> np.ndarray:
    """f = f^eq(rho, u), shape (9, ny, nx)."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    ux = None if ux is None else np.ascontiguousarray(ux, dtype=np.float64)
    uy = None if uy is None else np.ascontiguousarray(uy, dtype=np.float64)
    f = np.empty((9,) + rho.shape)
    _load().orc_init(ctypes.byref(p.c()), _ptr(rho), _ptr(ux), _ptr(uy), _ptr(f))
    return f


def step(p: Params, f) -> np.ndarray:
    """One time step (Eq. 1 with Eq. 10 forcing and periodic streaming)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(f)
    if _load().orc_step(ctypes.byref(p.c()), _ptr(f), _ptr(out)):
        raise MemoryError
    return out


def run(p: Params, f, nsteps: int) -> np.ndarray:
    """nsteps time steps; returns the new state (the input is not modified)."""
    g = np.array(f, dtype=np.float64, order="C", copy=True)
    if _load().orc_run(ctypes.byref(p.c()), _ptr(g), int(nsteps)):
        raise MemoryError
    return g


def moments(p: Params, f):
    """(rho, vx, vy): density (Eq. 3) and the half-step velocity of Eq. 11."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    shp = f.shape[1:]
    rho, vx, vy = np.empty(shp), np.empty(shp), np.empty(shp)
    if _load().orc_moments(ctypes.byref(p.c()), _ptr(f), _ptr(rho), _ptr(vx), _ptr(vy)):
        raise MemoryError
    return rho, vx, vy


def tangent(p: Params, rho0, nsteps: int, *, drho0=None, dTr: float = 0.0, dG: float = 0.0, h: float = 1e-30):
    """Complex-step derivative of the discrete map (Squire & Trapp 1998): the
    step run in complex arithmetic from f = f^eq(rho0 + i h drho0, 0) with
    T + i h dTr Tc and G + i h dG.  Returns (rho_T, d rho_T) where d rho_T is
    the derivative of the density after nsteps steps along the direction
    (drho0, dTr, dG), exact to rounding (no difference quotient).  dTr is a
    direction in the reduced temperature (T = Tr Tc); dG applies in psi mode."""
    rho0 = np.ascontiguousarray(rho0, dtype=np.float64)
    d0 = None if drho0 is None else np.ascontiguousarray(drho0, dtype=np.float64)
    if d0 is not None and d0.shape != rho0.shape:
        raise ValueError("drho0 must have the shape of rho0")
    rho, drho = np.empty_like(rho0), np.empty_like(rho0)
    if _load().orc_cs_run(ctypes.byref(p.c()), _ptr(rho0), _ptr(d0), float(dTr) * p.Tc, float(dG), float(h),
                          int(nsteps), _ptr(rho), _ptr(drho)):
        raise MemoryError
    return rho, drho
