"""FP64 CPU oracle of the LBGK method (test infrastructure only).

This package is the checker that the CUDA library is compared against.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import it; the library and
its Python binding never do, and this package imports nothing from the library.

The arithmetic of a time step lives in ``lbm_oracle.c`` (plain C, FP64, array-of-structures, full
populations f_i rather than deviations).  This module compiles it with gcc, loads it with ctypes,
and adds the host-side pieces written directly from the paper:

* geometry labels of the two workloads (plate and rectangular beam), Sec. 6 "Fluid-solid interaction";
* the mapping from the nondimensional frequency tau*omega to lattice (tau, omega), Sec. 6
  ("tau = mu/p = nu/theta");
* the least-squares split of the force history into the parts in phase with the body velocity and
  with its acceleration (the dissipative and inertial parts of F_f in Eq. 1), and the normalized
  damping of Eq. 20.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "lbm_oracle.c"
_BUILD = _HERE / "_build"
_LIB_PATH = _BUILD / "liblbm_oracle.so"
_lib = None

DRIVE_WALL = 0   # label-1 solid moves with U_w = u0 sin(omega t) x
DRIVE_BODY = 1   # body frame: fluid force density rho * u0 omega cos(omega t) x, walls static
COLL_BGK = 0
COLL_REG = 1
WALL_BB = 0      # bounce-back, Eq. 12
WALL_DS = 1      # diffuse scattering, Eq. 11


class _Params(ctypes.Structure):
    _fields_ = [
        ("Q", ctypes.c_int),
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("tau", ctypes.c_double),
        ("omega", ctypes.c_double),
        ("u0", ctypes.c_double),
        ("rho0", ctypes.c_double),
        ("eq_order", ctypes.c_int),
        ("collision", ctypes.c_int),
        ("drive", ctypes.c_int),
        ("label", ctypes.POINTER(ctypes.c_ubyte)),
        ("wall", ctypes.c_int),
    ]


def build(force: bool = False) -> Path:
    """Compile lbm_oracle.c into a shared library (gcc, -O2, OpenMP); returns its path."""
    _BUILD.mkdir(exist_ok=True)
    if force or not _LIB_PATH.exists() or _LIB_PATH.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _BUILD / f"liblbm_oracle.{os.getpid()}.so"
        subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", str(tmp), str(_SRC), "-lm"],
                       check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(str(build()))
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_lattice.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp, dp]
        lib.oracle_equilibrium.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, dp]
        lib.oracle_project.argtypes = [ctypes.c_int, dp, dp, dp]
        lib.oracle_source.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, dp]
        lib.oracle_collide.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, dp,
                                       ctypes.c_double, dp]
        lib.oracle_run.argtypes = [ctypes.POINTER(_Params), ctypes.c_long, ctypes.c_long, dp, dp, ctypes.c_int]
        lib.oracle_max_threads.argtypes = []
        _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def lattice(Q: int):
    """Lattice velocities c (Q x 2 int), weights w (Q,) and theta, in the oracle's own order."""
    c = (ctypes.c_int * (2 * Q))()
    w = np.zeros(Q)
    th = ctypes.c_double()
    if _load().oracle_lattice(Q, c, _dptr(w), ctypes.byref(th)):
        raise ValueError(f"no lattice with Q={Q}")
    return np.array(c[:], dtype=np.int64).reshape(Q, 2), w, th.value


def radius(Q: int) -> int:
    """Largest |c_ia| of the lattice: the stencil reach of one step."""
    c, _, _ = lattice(Q)
    return int(np.abs(c).max())


def equilibrium(Q: int, order: int, rho: float, ux: float, uy: float) -> np.ndarray:
    """f^eq of Eq. 15 (order 2) or its 4th-order Hermite continuation (order 4)."""
    out = np.zeros(Q)
    if _load().oracle_equilibrium(Q, order, rho, ux, uy, _dptr(out)):
        raise ValueError("bad lattice or order")
    return out


def project(Q: int, fadv: np.ndarray, feq: np.ndarray) -> np.ndarray:
    """Projected non-equilibrium part of Eq. 19 (plus its first Hermite moment, see lbm_oracle.c)."""
    fadv = np.ascontiguousarray(fadv, dtype=np.float64)
    feq = np.ascontiguousarray(feq, dtype=np.float64)
    out = np.zeros(Q)
    if _load().oracle_project(Q, _dptr(fadv), _dptr(feq), _dptr(out)):
        raise ValueError("bad lattice")
    return out


def source(Q: int, tau: float, ux: float, uy: float, Fx: float, Fy: float) -> np.ndarray:
    """Body-force source S_i of the time step (Guo-type, half-force velocity u; see lbm_oracle.c)."""
    out = np.zeros(Q)
    if _load().oracle_source(Q, tau, ux, uy, Fx, Fy, _dptr(out)):
        raise ValueError("bad lattice or tau")
    return out


def collide(Q: int, eq_order: int, collision: int, tau: float, fadv: np.ndarray, gx: float = 0.0) -> np.ndarray:
    """One node's collision from its advected populations, exactly as the time step does it: Eq. 16
    (half-force velocity with the body force rho gx along x), Eq. 15, then Eq. 18 + 19 (collision 1)
    or the BGK step (collision 0), plus the source."""
    fadv = np.ascontiguousarray(fadv, dtype=np.float64)
    out = np.zeros(Q)
    if _load().oracle_collide(Q, eq_order, collision, tau, _dptr(fadv), gx, _dptr(out)):
        raise ValueError("bad arguments")
    return out


def max_threads() -> int:
    return int(_load().oracle_max_threads())


# ---------------------------------------------------------------------------------------------
# geometry (labels: 0 fluid, 1 body whose force is recorded, 2 static wall)
# ---------------------------------------------------------------------------------------------

def geometry_plate(Q: int, nx: int, ny: int) -> np.ndarray:
    """Oscillating plate (Stokes' second problem, Sec. 3.1): the bottom R rows are the plate
    (label 1), the top R rows a static wall (label 2), R the lattice reach, so that no link of
    the periodic box crosses a wall without ending inside it."""
    R = radius(Q)
    lab = np.zeros((ny, nx), dtype=np.uint8)
    lab[:R, :] = 1
    lab[ny - R:, :] = 2
    return lab


def geometry_beam(nx: int, ny: int, lx: int, ly: int) -> np.ndarray:
    """Rectangular beam section, lx nodes along the motion (x) and ly across, centred in the
    periodic nx x ny box (Sec. 3: AR = Ly/Lx)."""
    lab = np.zeros((ny, nx), dtype=np.uint8)
    x0 = (nx - lx) // 2
    y0 = (ny - ly) // 2
    lab[y0:y0 + ly, x0:x0 + lx] = 1
    return lab


def rest_state(Q: int, nx: int, ny: int, rho0: float = 1.0) -> np.ndarray:
    """Fluid at rest, f_i = w_i rho0 at every node (AoS: [ny][nx][Q])."""
    _, w, _ = lattice(Q)
    return np.ascontiguousarray(np.broadcast_to(w * rho0, (ny, nx, Q)), dtype=np.float64)


def run(Q, label, tau, omega, u0, nsteps, *, rho0=1.0, eq_order=2, collision=COLL_REG, drive=DRIVE_WALL,
        f=None, n0=0, nthreads=1, wall=WALL_BB):
    """Advance the post-collision state f ([ny][nx][Q], full populations) by nsteps steps starting
    at step n0; returns (f, force) with force[k] = (Fx, Fy) on the label-1 body during step n0+k."""
    label = np.ascontiguousarray(label, dtype=np.uint8)
    ny, nx = label.shape
    if f is None:
        f = rest_state(Q, nx, ny, rho0)
    f = np.ascontiguousarray(f, dtype=np.float64).copy()
    assert f.shape == (ny, nx, Q)
    force = np.zeros((max(nsteps, 0), 2))
    p = _Params(Q, nx, ny, tau, omega, u0, rho0, eq_order, collision, drive,
                label.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), wall)
    rc = _load().oracle_run(ctypes.byref(p), n0, nsteps, _dptr(f), _dptr(force), nthreads)
    if rc:
        raise ValueError(f"oracle_run failed ({rc})")
    return f, force


# ---------------------------------------------------------------------------------------------
# parameters and post-processing
# ---------------------------------------------------------------------------------------------

def params_from_tau_omega(Q: int, tau_omega: float, delta_min: float = 4.0, p_min: int = 128):
    """Lattice (tau, omega, steps per period) for a nondimensional frequency tau*omega.

    Sec. 6 sets tau = mu/p = nu/theta; with the LBGK viscosity nu = theta (tau_LB - 1/2) the
    physical relaxation time is tau_LB - 1/2 steps, so tau*omega = (tau_LB - 1/2) omega.  The
    period P (an integer number of steps) is the larger of p_min and the one that puts delta_min
    nodes in the Stokes layer sqrt(2 nu / omega); then omega = 2 pi / P and tau_LB = 1/2 + tau*omega / omega.
    """
    _, _, th = lattice(Q)
    P = max(p_min, math.ceil(2.0 * math.pi * delta_min / math.sqrt(2.0 * th * tau_omega)))
    omega = 2.0 * math.pi / P
    return 0.5 + tau_omega / omega, omega, P


def fit_force(force_x: np.ndarray, omega: float, n0: int = 0, skip: int = 0):
    """Least squares of F_x(t_n) = A sin(omega t) + B cos(omega t) + C at t_n = n + 1/2 over the
    samples from index `skip` on; returns (A, B, C)."""
    n = np.arange(n0, n0 + len(force_x)) + 0.5
    t = n[skip:]
    M = np.stack([np.sin(omega * t), np.cos(omega * t), np.ones_like(t)], axis=1)
    coef, *_ = np.linalg.lstsq(M, np.asarray(force_x)[skip:], rcond=None)
    return float(coef[0]), float(coef[1]), float(coef[2])


def body_velocity_sign(drive: int) -> float:
    """Body velocity is V(t) = s u0 sin(omega t): s = +1 for the moving wall; s = -1 in the body
    frame, where the fluid force g = u0 omega cos(omega t) equals -dV/dt."""
    return 1.0 if drive == DRIVE_WALL else -1.0


def in_phase_quadrature(force_x, omega, drive, n0=0, skip=0):
    """(F_in, F_q): force parts along the body velocity V/u0 and along dV/dt/(u0 omega)."""
    A, B, _ = fit_force(force_x, omega, n0, skip)
    s = body_velocity_sign(drive)
    return s * A, s * B


def gamma_bar(F_in: float, u0: float, rho0: float, theta: float, perimeter: float) -> float:
    """Normalized damping of Eq. 20 per unit length: gamma_f m_o = -F_in/u0 and S/m_o -> wetted
    perimeter / m_o, so gamma_bar = -F_in / (u0 rho0 sqrt(theta/2) perimeter)."""
    return -F_in / (u0 * rho0 * math.sqrt(theta / 2.0) * perimeter)
