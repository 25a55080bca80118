"""Precision study (GPU): in-phase and quadrature force of the D2Q37-H4 beam, every storage type,
against the FP64 oracle on the 256 x 256 downscale, body frame (tests/golden/precision_beam256.json)
and lab frame with moving walls (precision_beam256_lab.json).

Error metric: err_c = |F_c(gpu) - F_c(oracle)| / sqrt(F_in^2 + F_q^2)(oracle), c in {in, q}
(normalizing by the amplitude keeps the metric finite when one component vanishes).
Bounds: FP64 storage agrees with the oracle to rounding (1e-9); FP32 and FP16 storage (scaled by
U0, FP32 arithmetic, FP64 force) meet the 1e-4 target; BF16 storage does not (each stored value
is rounded to 8 significant bits, 2^-8 relative, every step) and is held to 1e-2.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_0904_4504_gb300 import inputs as I
from paper_0904_4504_gb300 import lbm as L

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

GOLDEN = {frame: os.path.join(os.path.dirname(__file__), "golden", name)
          for frame, name in (("body", "precision_beam256.json"), ("lab", "precision_beam256_lab.json"))}
BOUND = {L.LBM_STORE_F64: 1e-9, L.LBM_STORE_F32: 1e-4, L.LBM_STORE_F16: 1e-4, L.LBM_STORE_BF16: 1e-2}


def gpu_fit(case, storage, n=256, drive=None):
    w = I.beam_d2q37_h4(case["tau_omega"], n=n, storage=storage)
    geom = L.make_geometry(kind=w.geometry, lx=w.lx, ly=w.ly, drive=w.drive if drive is None else drive, u0=w.u0,
                           eq_order=w.eq_order, collision=w.collision, storage=storage)
    h = L.lbm_create(37, n, n, case["tau"], case["omega"], geom)
    try:
        L.lbm_step(h, case["steps"])
        F = L.lbm_force_history(h)
        f_in, f_q, _ = L.lbm_fit(h, 15.0)
    finally:
        L.lbm_destroy(h)
    return f_in, f_q, F


@pytest.mark.parametrize("frame", ["body", "lab"])
@pytest.mark.parametrize("storage", [L.LBM_STORE_F64, L.LBM_STORE_F32, L.LBM_STORE_F16, L.LBM_STORE_BF16])
def test_force_error_against_oracle(storage, frame):
    gold = json.load(open(GOLDEN[frame]))
    drive = L.LBM_DRIVE_WALL if frame == "lab" else L.LBM_DRIVE_BODYFORCE
    for case in gold["cases"]:
        f_in, f_q, F = gpu_fit(case, storage, drive=drive)
        amp = math.hypot(case["F_in"], case["F_q"])
        e_in = abs(f_in - case["F_in"]) / amp
        e_q = abs(f_q - case["F_q"]) / amp
        # every 64th force sample as well (max norm over the history, relative to the amplitude)
        e_hist = np.abs(F[::gold["cases"][0]["sample_every"], 0] - np.array(case["Fx_samples"])).max() / amp
        print(f"{frame} frame, storage {storage} tau*omega {case['tau_omega']}: err_in {e_in:.2e} err_q {e_q:.2e} "
              f"hist {e_hist:.2e}")
        assert e_in <= BOUND[storage] and e_q <= BOUND[storage], (e_in, e_q)


@pytest.mark.parametrize("storage", [L.LBM_STORE_F32, L.LBM_STORE_F16])
def test_lab_and_body_frames_agree_at_full_size(storage):
    """The 1024 x 1024 beam of the headline workload driven both ways: the body-frame force history
    is the lab-frame one half a step later, so (F_in, F_q) of the body frame rotated by omega/2
    matches the lab frame (the same Galilean equivalence the oracle is pinned to, here at the full
    size with 1e-3 blockage).  16-bit storage reaches it through two different number paths: the
    stream offset in the body frame, plain scaled deviations in the lab frame."""
    for to in (0.1, 1.0, 10.0):
        w = I.beam_d2q37_h4(to, n=1024, storage=storage)
        tau, omega, P = L.lbm_params_from_tau_omega(37, to)
        fits = {}
        for drive in (L.LBM_DRIVE_WALL, L.LBM_DRIVE_BODYFORCE):
            geom = L.make_geometry(kind=w.geometry, lx=w.lx, ly=w.ly, drive=drive, u0=w.u0, eq_order=w.eq_order,
                                   collision=w.collision, storage=storage)
            h = L.lbm_create(37, 1024, 1024, tau, omega, geom)
            try:
                L.lbm_step(h, 8 * P)
                fits[drive] = L.lbm_fit(h, 4.0)[:2]
            finally:
                L.lbm_destroy(h)
        li, lq = fits[L.LBM_DRIVE_WALL]
        bi, bq = fits[L.LBM_DRIVE_BODYFORCE]
        amp = math.hypot(li, lq)
        c, s = math.cos(omega / 2), math.sin(omega / 2)
        d_in, d_q = (li - (bi * c - bq * s)) / amp, (lq - (bq * c + bi * s)) / amp
        print(f"storage {storage} tau*omega {to}: lab ({li:.6e}, {lq:.6e}) body ({bi:.6e}, {bq:.6e}) "
              f"shifted diff ({d_in:.2e}, {d_q:.2e})")
        assert abs(lq - bq) > 1e-2 * amp
        assert abs(d_in) < 3e-4 and abs(d_q) < 3e-4
