"""Write tests/golden/precision_beam256.json: FP64 oracle fits of the downscaled precision-study beam.

The workload is the D2Q37 beam of the precision study (32 x 32 section, 4th-order equilibrium,
regularized collision, body-frame drive U0 = 1e-3) in a 256 x 256 box instead of 2048 x 2048, at
tau*omega = 0.1, 1, 10, for 30 periods.  For each one it stores the in-phase and quadrature force
(fit after the first 15 periods) and every 64th force sample.  Only the oracle runs here.
With --lab the beam is driven as a moving wall instead (lab frame, Sec. 6), written to
precision_beam256_lab.json.

    python tests/golden/make_precision_beam256.py [--lab]     # ~minutes on a few cores
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle as orc  # noqa: E402
from paper_0904_4504_gb300 import inputs as I  # noqa: E402

N, PERIODS, SKIP = 256, 30, 15


def main(lab_frame=False):
    drive = orc.DRIVE_WALL if lab_frame else orc.DRIVE_BODY
    frame = "lab-frame moving-wall" if lab_frame else "body-frame"
    out = {"workload": f"D2Q37-H4 regularized beam 32x32 in {N}x{N}, {frame} drive, U0=1e-3, rho0=1",
           "periods": PERIODS, "skip_periods": SKIP, "cases": []}
    for to in I.PRECISION_TAU_OMEGAS:
        w = I.beam_d2q37_h4(to, n=N)
        tau, omega, P = orc.params_from_tau_omega(37, to)
        lab = orc.geometry_beam(N, N, w.lx, w.ly)
        steps = PERIODS * P
        t0 = time.time()
        _, F = orc.run(37, lab, tau, omega, w.u0, steps, eq_order=4, collision=orc.COLL_REG, drive=drive,
                       nthreads=orc.max_threads())
        Fin, Fq = orc.in_phase_quadrature(F[:, 0], omega, drive, skip=SKIP * P)
        out["cases"].append({"tau_omega": to, "tau": tau, "omega": omega, "period": P, "steps": steps,
                             "F_in": Fin, "F_q": Fq, "sample_every": 64,
                             "Fx_samples": F[::64, 0].tolist(), "Fy_samples": F[::64, 1].tolist()})
        print(f"tau*omega={to}: {steps} steps in {time.time() - t0:.0f} s, F_in={Fin:.6e} F_q={Fq:.6e}", flush=True)
    name = "precision_beam256_lab.json" if lab_frame else "precision_beam256.json"
    with open(os.path.join(HERE, name), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main(lab_frame="--lab" in sys.argv[1:])
