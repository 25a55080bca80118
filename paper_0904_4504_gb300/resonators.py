"""Quality factor of the paper's resonators in nitrogen from simulated normalized damping.

Eq. 20 normalizes the fluid damping: gamma_f = rho sqrt(theta/2) (S/m_o) gamma_bar(tau*omega, AR),
and Eq. 21 (Sec. 6) gives Q = Q_o / (1 + gamma_f / gamma_o) with gamma_o = omega_o / Q_o.  For a gas at pressure p: theta = c_s^2, rho = p / theta and
tau = mu / p, so tau*omega = mu omega_o / p.  gamma_bar comes from simulations (a tau*omega sweep of
the device's cross-section, `damping_sweep`), interpolated in log(tau*omega).

Device data: Table 1 (omega_o / 2 pi, Q_o, S / m_o, AR; Sec. 6 takes AR = 0 for the quartz disk and
1, 10, 26 for the beams); gas: nitrogen at room temperature, c_s ~ 298 m/s and
mu ~ 1.78e-5 kg/(m s) (Sec. 3).  Pressures of the experiments: 0.1 to 1000 Torr (Sec. 2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

C_S_N2 = 298.0          # m/s
MU_N2 = 1.78e-5         # kg/(m s)
TORR = 133.322368       # Pa


@dataclass(frozen=True)
class Resonator:
    name: str
    f0_hz: float          # omega_o / 2 pi
    q0: float
    s_over_m: float       # m^2/kg
    aspect_ratio: float   # AR = Ly / Lx


TABLE1 = (
    Resonator("cantilever beam", 0.078e6, 8320, 688, 26),
    Resonator("cantilever beam, first harmonic", 1.97e6, 3520, 405, 10),
    Resonator("doubly-clamped beam", 24.2e6, 415, 8380, 1),
    Resonator("quartz crystal disk", 32.7e6, 40755, 6.29, 0),
)


def tau_omega(dev: Resonator, p_pa, mu=MU_N2):
    """tau*omega = mu omega_o / p."""
    return mu * 2.0 * math.pi * dev.f0_hz / np.asarray(p_pa, dtype=float)


def fluid_damping(dev: Resonator, p_pa, gamma_bar, c_s=C_S_N2):
    """gamma_f = rho sqrt(theta/2) (S/m_o) gamma_bar with theta = c_s^2, rho = p / theta."""
    theta = c_s * c_s
    rho = np.asarray(p_pa, dtype=float) / theta
    return rho * math.sqrt(theta / 2.0) * dev.s_over_m * np.asarray(gamma_bar, dtype=float)


def quality_factor(dev: Resonator, p_pa, gamma_bar_of_tau_omega, mu=MU_N2, c_s=C_S_N2):
    """Q(p) of Eq. 21, Q_o / (1 + gamma_f / gamma_o); gamma_bar_of_tau_omega maps tau*omega to gamma_bar."""
    to = tau_omega(dev, p_pa, mu)
    gf = fluid_damping(dev, p_pa, gamma_bar_of_tau_omega(to), c_s)
    gamma_o = 2.0 * math.pi * dev.f0_hz / dev.q0
    return dev.q0 / (1.0 + gf / gamma_o)


def interpolated(tau_omegas, gamma_bars):
    """gamma_bar(tau*omega) from sweep points: linear in log(tau*omega) between them, held at the
    last value above them (gamma_bar saturates as tau*omega -> infinity, Sec. 6), and continued as
    sqrt(tau*omega) below them (the Newtonian Stokes-layer scaling, Eq. 4)."""
    x = np.log(np.asarray(tau_omegas, dtype=float))
    y = np.asarray(gamma_bars, dtype=float)
    order = np.argsort(x)
    x, y = x[order], y[order]

    def gamma_bar(to):
        lt = np.log(np.asarray(to, dtype=float))
        return np.where(lt < x[0], y[0] * np.exp(0.5 * (lt - x[0])), np.interp(lt, x, y))
    return gamma_bar


def beam_section(aspect_ratio: float, ly_max: int = 208, lx_max: int = 32):
    """(lx, ly) in lattice nodes of a beam section with ly / lx = AR: the thickest section at most
    lx_max thick along the motion and ly_max across."""
    lx = min(lx_max, max(1, int(round(ly_max / aspect_ratio))))
    return lx, max(1, int(round(aspect_ratio * lx)))


def sweep_period(tau_omega, length, box, theta, p_res, acoustic=0.25, mfp_fraction=0.25):
    """Steps per period of one sweep point.  gamma_bar depends on tau*omega and AR alone (Sec. 6)
    while the section is small against the acoustic wavelength (omega L / c_s <= `acoustic`; the
    devices sit near 0.1) and the box is large against the mean free path c_s tau (<= `mfp_fraction`
    of the box, else molecules bounced off the body come back through the periodic images without
    meeting the gas).  With tau = tau*omega / omega and omega = 2 pi / P the first asks for a long
    period and the second for a short one at large tau*omega; the period is the acoustic one capped by
    the mean-free-path one, and never below p_res (the resolution rule of lbm_params_from_tau_omega)."""
    c_s = math.sqrt(theta)
    p_ac = 2.0 * math.pi * length / (acoustic * c_s) if length > 0 else 0.0
    p_mfp = 2.0 * math.pi * mfp_fraction * box / (c_s * tau_omega)
    return max(p_res, int(math.ceil(min(p_ac, p_mfp))))


def damping_sweep(tau_omegas, aspect_ratio, *, lattice=37, side=1024, plate_ny=4096, periods=12, u0=1e-3,
                  eq_order=4, storage=None, wall_scheme=0, lx_max=32, ly_max=208, acoustic=0.25,
                  mfp_fraction=0.25):
    """gamma_bar at each tau*omega for one aspect ratio, from GPU runs batched in one lbm_batch
    (streams mode).  AR = 0 is the oscillating plate (32 x plate_ny box, wall drive, one face);
    AR > 0 a beam_section() centred in a side x side periodic box, body-frame drive.  The period of
    each point is sweep_period(); U_0 is capped at omega / 10 (displacement below a tenth of a node,
    and U_0 < omega as Sec. 6 requires).  Each run lasts `periods` periods and the fit skips the
    first half.  Returns one record per point: gamma_bar, period, tau, omega, u0, omega_L_over_cs
    (the acoustic compactness reached) and mfp_over_box.  Needs the CUDA library."""
    from . import lbm as L

    storage = L.LBM_STORE_F32 if storage is None else storage
    _, _, theta = L.lbm_lattice_velocities(lattice)
    c_s = math.sqrt(theta)
    b = L.lbm_batch_create(lattice, storage, L.LBM_COLL_REGULARIZED)
    try:
        runs = []
        for to in tau_omegas:
            if aspect_ratio == 0:
                nx, ny, perim, length, box = 32, plate_ny, 32.0, 0, plate_ny
                geo = dict(kind=L.LBM_GEOM_PLATE, drive=L.LBM_DRIVE_WALL)
            else:
                lx, ly = beam_section(aspect_ratio, ly_max, lx_max)
                nx, ny, perim, length, box = side, side, 2.0 * (lx + ly), max(lx, ly), side
                geo = dict(kind=L.LBM_GEOM_BEAM, lx=lx, ly=ly, drive=L.LBM_DRIVE_BODYFORCE)
            _, _, p_res = L.lbm_params_from_tau_omega(lattice, to)
            P = sweep_period(to, length, box, theta, p_res, acoustic, mfp_fraction)
            tau, omega, P = L.lbm_params_from_tau_omega(lattice, to, p_min=P)
            u = min(u0, 0.1 * omega)
            d = L.make_instance(lattice, nx, ny, tau, omega, int(periods * P), u0=u, eq_order=eq_order,
                                storage=storage, wall_scheme=wall_scheme, **geo)
            rec = {"tau_omega": to, "period": P, "tau": tau, "omega": omega, "u0": u,
                   "omega_L_over_cs": omega * length / c_s, "mfp_over_box": c_s * (tau - 0.5) / box}
            runs.append((L.lbm_batch_add(b, d), d.nsteps, perim, rec))
        L.lbm_batch_run(b, max(n for _, n, _, _ in runs))
        L.lbm_batch_synchronize(b)
        out = []
        for s, _, perim, rec in runs:
            sim = L.lbm_batch_instance(b, s)
            f_in, _, _ = L.lbm_fit(sim, periods / 2.0)
            rec["gamma_bar"] = L.lbm_gamma_bar(sim, f_in, perim)
            out.append(rec)
        return out
    finally:
        L.lbm_batch_destroy(b)


def quality_curves(tau_omegas=None, pressures_torr=None, devices=TABLE1, **sweep):
    """Q/Q_o over pressure for each device: one damping_sweep per distinct AR, then Eq. 21.
    Returns {"tau_omega": [...], "pressure_torr": [...], "devices": [{name, aspect_ratio,
    gamma_bar: [...], points: [damping_sweep records], q_over_q0: [...]}]}."""
    tau_omegas = list(np.logspace(-3, 1, 9) if tau_omegas is None else tau_omegas)
    p_torr = np.logspace(-1, 3, 13) if pressures_torr is None else np.asarray(pressures_torr, dtype=float)
    sweeps = {}
    out = {"tau_omega": tau_omegas, "pressure_torr": p_torr.tolist(), "devices": []}
    for dev in devices:
        ar = dev.aspect_ratio
        if ar not in sweeps:
            sweeps[ar] = damping_sweep(tau_omegas, ar, **sweep)
        gbs = [r["gamma_bar"] for r in sweeps[ar]]
        q = quality_factor(dev, p_torr * TORR, interpolated(tau_omegas, gbs)) / dev.q0
        out["devices"].append({"name": dev.name, "aspect_ratio": ar, "gamma_bar": gbs, "points": sweeps[ar],
                               "q_over_q0": q.tolist()})
    return out


if __name__ == "__main__":
    import argparse
    import json

    ap = argparse.ArgumentParser(description="Q/Q_o(p) of the Table 1 resonators from simulated damping")
    ap.add_argument("--side", type=int, default=1024)
    ap.add_argument("--periods", type=int, default=12)
    ap.add_argument("--points", type=int, default=9, help="tau*omega points, log-spaced in [1e-3, 10]")
    ap.add_argument("--wall", choices=["bb", "ds"], default="bb")
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    res = quality_curves(np.logspace(-3, 1, a.points).tolist(), side=a.side, periods=a.periods,
                         wall_scheme=1 if a.wall == "ds" else 0)
    text = json.dumps(res, indent=1)
    if a.out:
        with open(a.out, "w") as fh:
            fh.write(text)
    print(text)
