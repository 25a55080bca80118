"""Seeded synthetic workloads shaped like the paper's cases (no LBGK arithmetic here).

The paper's simulations are 2-D cross-sections of resonators: an oscillating plate (the quartz
thickness-shear disk, AR = 0) and rectangular beams (AR = Ly/Lx = 1, 10, 26 in Table 1), over
0.001 <= tau*omega <= 10 (Sec. 6).  Its experimental data and figures are not available, so every
input here is generated: workload descriptions (lattice, grid, geometry, tau*omega, drive, number
of periods) and, for parity tests, random masks and random initial deviations.  Both the CUDA
library and the oracle are fed from these descriptions; each side maps tau*omega to its own lattice
parameters.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

PLATE, BEAM, MASK, NONE = 0, 1, 2, 3
DRIVE_WALL, DRIVE_BODY = 0, 1
BGK, REG = 0, 1
F64, F32, BF16, F16 = 0, 1, 2, 3

SWEEP_SEED = 20090424
SERVE_SEED = 4504


@dataclass
class Workload:
    name: str
    lattice: int
    nx: int
    ny: int
    tau_omega: float | None       # nondimensional frequency (None: tau/omega given directly)
    geometry: int
    lx: int = 0
    ly: int = 0
    drive: int = DRIVE_WALL
    u0: float = 1e-3
    eq_order: int = 2
    collision: int = REG
    storage: int = F32
    periods: float = 30.0
    tau: float | None = None      # only for workloads that fix tau and omega themselves
    omega: float | None = None
    extra: dict = field(default_factory=dict)


def plate_d2q9_fp64() -> Workload:
    """Thickness-shear limit: infinite plate oscillating tangentially, D2Q9 plain BGK in FP64, 4 x 256
    periodic in x, U0 = 1e-3, tau = 0.8, tau*omega = 0.1 (with tau*omega = (tau - 1/2) omega this
    gives omega = 1/3), 20 periods."""
    return Workload("plate-d2q9-bgk-fp64-4x256", 9, 4, 256, None, PLATE, drive=DRIVE_WALL, u0=1e-3, eq_order=2,
                    collision=BGK, storage=F64, periods=20.0, tau=0.8, omega=0.1 / 0.3)


def beam_d2q37_h4(tau_omega: float, n: int = 1024, storage: int = F32, side: int = 32) -> Workload:
    """Rectangular beam 32 x 32 centred in an n x n periodic box, D2Q37 with the 4th-order
    equilibrium, regularized collision, body frame with force rho U0 omega cos(omega t), 30 periods."""
    return Workload(f"beam-d2q37-h4-{n}x{n}-to{tau_omega:g}", 37, n, n, tau_omega, BEAM, lx=side, ly=side,
                    drive=DRIVE_BODY, u0=1e-3, eq_order=4, collision=REG, storage=storage, periods=30.0)


BEAM_TAU_OMEGAS = (0.01, 1.0, 10.0)
PRECISION_TAU_OMEGAS = (0.1, 1.0, 10.0)


def sweep_d2q37(seed: int = SWEEP_SEED) -> list[Workload]:
    """64 instances: 16 log-spaced tau*omega in [1e-2, 1e2] x AR in {0.25, 0.5, 1, 2} (Lx = 32,
    Ly = 32 AR), square sides drawn uniformly from {256, 512, 768, 1024}, U0 ~ U[5e-4, 2e-3]."""
    rng = np.random.default_rng(seed)
    out = []
    for to in np.logspace(-2, 2, 16):
        for ar in (0.25, 0.5, 1.0, 2.0):
            n = int(rng.choice([256, 512, 768, 1024]))
            u0 = float(rng.uniform(5e-4, 2e-3))
            out.append(Workload(f"sweep-to{to:.3g}-ar{ar:g}-n{n}", 37, n, n, float(to), BEAM, lx=32, ly=int(32 * ar),
                                drive=DRIVE_BODY, u0=u0, eq_order=4, collision=REG, storage=F32, periods=30.0))
    return out


@dataclass
class Request:
    arrival_s: float
    workload: Workload


def serving_requests(n: int = 2000, rate_per_s: float = 50.0, seed: int = SERVE_SEED) -> list[Request]:
    """Poisson arrivals (mean rate 50/s); plate or beam 50/50 (beam AR ~ U[0.25, 4], Lx = 32);
    tau*omega log-uniform on [1e-3, 1e3]; square side ~ U[128, 2048] rounded to 32; periods ~ U{10..50};
    D2Q9 or D2Q37 50/50."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, n))
    out = []
    for k in range(n):
        lattice = 9 if rng.random() < 0.5 else 37
        plate = rng.random() < 0.5
        side = int(round(rng.uniform(128, 2048) / 32.0) * 32)
        to = float(10 ** rng.uniform(-3, 3))
        periods = int(rng.integers(10, 51))
        ar = float(rng.uniform(0.25, 4.0))
        if plate:
            w = Workload(f"req{k}", lattice, side, side, to, PLATE, drive=DRIVE_WALL, u0=1e-3,
                         eq_order=2 if lattice == 9 else 4, collision=REG, storage=F32, periods=periods)
        else:
            ly = max(8, min(side - 16, int(round(32 * ar))))
            w = Workload(f"req{k}", lattice, side, side, to, BEAM, lx=32, ly=ly, drive=DRIVE_BODY, u0=1e-3,
                         eq_order=2 if lattice == 9 else 4, collision=REG, storage=F32, periods=periods)
        out.append(Request(float(t[k]), w))
    return out


# ------------------------------------------------------------------------------------------------
# inputs for parity tests
# ------------------------------------------------------------------------------------------------

def random_mask(nx: int, ny: int, reach: int, seed: int, n_blocks: int = 3) -> np.ndarray:
    """Labels (0 fluid, 1 body, 2 static wall): a few axis-aligned solid blocks at least `reach`
    nodes thick and `reach` nodes apart (so no link tunnels through a solid or between two)."""
    rng = np.random.default_rng(seed)
    lab = np.zeros((ny, nx), np.uint8)
    placed = 0
    for _ in range(200):
        if placed == n_blocks:
            break
        w = int(rng.integers(reach, max(reach + 1, nx // 3)))
        h = int(rng.integers(reach, max(reach + 1, ny // 3)))
        x0 = int(rng.integers(0, nx))
        y0 = int(rng.integers(0, ny))
        ys = (np.arange(y0 - reach, y0 + h + reach) % ny)[:, None]
        xs = (np.arange(x0 - reach, x0 + w + reach) % nx)[None, :]
        if lab[ys, xs].any():
            continue
        lab[(np.arange(y0, y0 + h) % ny)[:, None], (np.arange(x0, x0 + w) % nx)[None, :]] = 1 if placed == 0 else 2
        placed += 1
    return lab


def random_scaled_state(Q: int, nx: int, ny: int, exponent: int, seed: int) -> np.ndarray:
    """Random initial state in storage units h = k * 2**exponent with |k| <= 255, shape (Q, ny, nx).

    Eight significant bits make every value exact in BF16, FP16 (for exponents >= -14), FP32 and
    FP64, so the library and the oracle start from the same numbers whatever the storage type."""
    rng = np.random.default_rng(seed)
    k = np.clip(np.rint(64.0 * rng.standard_normal((Q, ny, nx))), -255, 255)
    return k * 2.0 ** exponent
