"""Q(p) post-processing (Sec. 6 "Quality factor", Eq. 20, Table 1): checks against closed forms
and the scalings the paper states (Sec. 7: Q ~ omega for tau*omega > 1 against Q ~ sqrt(omega) in
the Newtonian regime)."""
import math

import numpy as np
import pytest

from paper_0904_4504_gb300 import resonators as R


def test_table1_values():
    quartz = R.TABLE1[3]
    assert quartz.f0_hz == 32.7e6 and quartz.q0 == 40755 and quartz.s_over_m == 6.29 and quartz.aspect_ratio == 0
    assert [d.aspect_ratio for d in R.TABLE1] == [26, 10, 1, 0]


def test_vacuum_limit_and_monotone_damping():
    dev = R.TABLE1[2]
    p = np.logspace(-3, 5, 30)
    q = R.quality_factor(dev, p, lambda to: np.ones_like(to))
    assert abs(q[0] / dev.q0 - 1) < 1e-6
    assert np.all(np.diff(q) < 0)


def test_newtonian_plate_scaling():
    """gamma_bar = sqrt(tau*omega) (Stokes plate, Eq. 4): gamma_f ~ sqrt(p) and, with the fluid
    dominating, Q ~ sqrt(omega_o) at fixed p."""
    dev = R.TABLE1[3]
    p = np.array([1e4, 4e4])
    gf = R.fluid_damping(dev, p, np.sqrt(R.tau_omega(dev, p)))
    assert abs(math.log(gf[1] / gf[0]) / math.log(4.0) - 0.5) < 1e-12
    # textbook Stokes layer: in-phase drag per unit area sqrt(rho mu omega / 2) per unit velocity,
    # rho = p / c_s^2, so gamma_f = (S/m) sqrt(rho mu omega_o / 2)
    om = 2 * math.pi * dev.f0_hz
    rho = p[0] / R.C_S_N2 ** 2
    assert abs(gf[0] / (dev.s_over_m * math.sqrt(rho * R.MU_N2 * om / 2.0)) - 1) < 1e-12
    hi = R.Resonator("x", 4 * dev.f0_hz, 1e18, dev.s_over_m, 0)
    lo = R.Resonator("x", dev.f0_hz, 1e18, dev.s_over_m, 0)
    g = lambda to: np.sqrt(to)
    ratio = R.quality_factor(hi, 1e5, g) / R.quality_factor(lo, 1e5, g)
    assert abs(ratio - 2.0) < 1e-6


def test_free_molecular_scaling():
    """gamma_bar -> const for tau*omega -> infinity: gamma_f ~ p and Q ~ omega_o."""
    dev = R.TABLE1[0]
    hi = R.Resonator("x", 4 * dev.f0_hz, 1e18, dev.s_over_m, 26)
    lo = R.Resonator("x", dev.f0_hz, 1e18, dev.s_over_m, 26)
    g = lambda to: 0.9 * np.ones_like(to)
    assert abs(R.quality_factor(hi, 10.0, g) / R.quality_factor(lo, 10.0, g) - 4.0) < 1e-6
    gf = R.fluid_damping(dev, np.array([1.0, 3.0]), [0.9, 0.9])
    assert abs(gf[1] / gf[0] - 3.0) < 1e-12


def test_interpolation_is_log_linear_saturates_and_continues_as_sqrt():
    f = R.interpolated([0.01, 1.0, 100.0], [0.1, 1.0, 2.0])
    assert abs(f(0.1) - 0.55) < 1e-12 and abs(f(1e6) - 2.0) < 1e-12
    assert abs(f(1e-6) - 0.1 * math.sqrt(1e-4)) < 1e-15


def test_beam_sections_have_the_table_aspect_ratios():
    assert R.beam_section(1) == (32, 32)
    for ar in (10, 26):
        lx, ly = R.beam_section(ar)
        assert abs(ly / lx - ar) / ar < 0.05 and ly <= 210


def test_quality_curves_vacuum_to_atmosphere(monkeypatch):
    """With a saturating damping curve, Q/Q_o -> 1 at low pressure and falls with p for every device."""
    monkeypatch.setattr(R, "damping_sweep", lambda tos, ar, **kw: [{"gamma_bar": 0.9 * t / (1 + t) + 0.1 * math.sqrt(t)}
                                                                   for t in tos])
    res = R.quality_curves(pressures_torr=[1e-4, 1.0, 1e3])
    for d in res["devices"]:
        q = d["q_over_q0"]
        assert q[0] > 0.99 and q[0] > q[1] > q[2] > 0


def test_sweep_period_balances_compactness_and_mean_free_path():
    th = 1 / 1.19697977039307 ** 2
    c_s = math.sqrt(th)
    # small tau*omega: the acoustic period (omega L / c_s = 1/4) wins
    P = R.sweep_period(1e-3, 208, 1024, th, 128)
    assert abs(2 * math.pi / P * 208 / c_s - 0.25) < 1e-3
    # large tau*omega: capped so that c_s tau <= box / 4, never below the resolution rule
    P = R.sweep_period(1.0, 208, 1024, th, 128)
    tau = 1.0 * P / (2 * math.pi)
    assert c_s * tau <= 1024 / 4 + c_s and P > 128
    assert R.sweep_period(100.0, 208, 1024, th, 128) == 128
    # the plate has no length: resolution and mean free path only
    assert R.sweep_period(1e-3, 0, 4096, th, 673) == 673
