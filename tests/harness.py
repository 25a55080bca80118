"""Shared helpers of the parity tests: run the CUDA library and the oracle on the same inputs and
bring both states to one layout ((Q, ny, nx) deviations g = f - w rho0, library direction order)."""
from __future__ import annotations

import numpy as np

import oracle as orc
from paper_0904_4504_gb300 import lbm as L


def perm_lib_to_oracle(Q: int) -> np.ndarray:
    """p with oracle_c[p[i]] == library_c[i] (a permutation; the two sides order velocities differently)."""
    c_lib, w_lib, th_lib = L.lbm_lattice_velocities(Q)
    c_or, w_or, th_or = orc.lattice(Q)
    p = np.array([int(np.flatnonzero((c_or == c).all(1))[0]) for c in c_lib])
    assert sorted(p.tolist()) == list(range(Q))
    return p


def oracle_state_to_g(Q: int, f: np.ndarray, rho0: float = 1.0) -> np.ndarray:
    """Oracle AoS f [ny][nx][Q] -> library-order deviations (Q, ny, nx)."""
    p = perm_lib_to_oracle(Q)
    _, w_or, _ = orc.lattice(Q)
    g = f - w_or * rho0
    return np.ascontiguousarray(np.transpose(g[:, :, p], (2, 0, 1)))


def g_to_oracle_state(Q: int, g: np.ndarray, rho0: float = 1.0) -> np.ndarray:
    p = perm_lib_to_oracle(Q)
    _, w_or, _ = orc.lattice(Q)
    f = np.empty((g.shape[1], g.shape[2], Q))
    f[:, :, p] = np.transpose(g, (1, 2, 0))
    return f + w_or * rho0


def oracle_labels(kind: int, Q: int, nx: int, ny: int, lx: int = 0, ly: int = 0, mask=None) -> np.ndarray:
    if kind == L.LBM_GEOM_PLATE:
        return orc.geometry_plate(Q, nx, ny)
    if kind == L.LBM_GEOM_BEAM:
        return orc.geometry_beam(nx, ny, lx, ly)
    if kind == L.LBM_GEOM_MASK:
        return np.asarray(mask, np.uint8)
    return np.zeros((ny, nx), np.uint8)


def scaled(Q: int, g: np.ndarray) -> np.ndarray:
    """h = g / w: every direction on the same footing."""
    _, w, _ = L.lbm_lattice_velocities(Q)
    return g / w[:, None, None]


def stream_offset_magnitude(Q: int, u0: float, omega: float, n: int, eq_order: int, rho0: float = 1.0) -> np.ndarray:
    """|H_i| of the 16-bit body-frame storage convention (include/lbm.h): the scaled equilibrium
    deviation of the uniform stream U(n) = sum_{k<n} u0 omega cos(omega (k + 1/2)); 16-bit storage
    rounds h - H, so its rounding error is bounded relative to |h| + |H|.  Tolerances only."""
    c, w, th = L.lbm_lattice_velocities(Q)
    U = sum(u0 * omega * np.cos(omega * (k + 0.5)) for k in range(n))
    a = c[:, 0] * U / th
    b = U * U / th
    poly = a + 0.5 * (a * a - b)
    if eq_order >= 4:
        poly = poly + (a ** 3 - 3 * a * b) / 6.0 + (a ** 4 - 6 * a * a * b + 3 * b * b) / 24.0
    return np.abs(rho0 * poly / u0)
