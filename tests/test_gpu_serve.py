"""GPU tests of the serving loop (continuous batching over the batch kernel).

The isolation test is the serving contract: every request gives the same force history and fit
whether it is served alone or in a mix of requests that arrive at different times, share the GPU
with other lattices and sizes, and join or leave the batch while it runs.  The batch kernel
computes each instance exactly as alone, so the histories must be bit for bit equal (the stated
tolerance is 0).
"""
import time

import numpy as np
import pytest

from paper_0904_4504_gb300 import lbm as L

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def _req(Q, nx, ny, tau, omega, nsteps, skip=0.25, **kw):
    geo = dict(kind=L.LBM_GEOM_BEAM, lx=12, ly=9, drive=L.LBM_DRIVE_BODYFORCE, u0=1e-3,
               eq_order=4 if Q == 37 else 2, collision=L.LBM_COLL_REGULARIZED, storage=L.LBM_STORE_F32)
    geo.update(kw)
    d = L.make_instance(Q, nx, ny, tau, omega, nsteps, **geo)
    return L.make_request(d, skip, 2.0 * (geo["lx"] + geo["ly"]) if geo["kind"] == L.LBM_GEOM_BEAM else 0.0)


REQS = [
    (37, 70, 41, 0.9, 0.05, 260, {}),
    (9, 64, 80, 0.8, 0.06, 300, dict(kind=L.LBM_GEOM_PLATE, drive=L.LBM_DRIVE_WALL)),
    (37, 133, 64, 1.7, 0.04, 200, dict(lx=20, ly=30)),
    (37, 96, 96, 0.6, 0.07, 150, dict(kind=L.LBM_GEOM_PLATE, drive=L.LBM_DRIVE_WALL)),
    (9, 120, 50, 1.2, 0.05, 280, dict(lx=16, ly=8)),
    (37, 200, 90, 3.0, 0.03, 300, dict(lx=24, ly=19, storage=L.LBM_STORE_F16)),
]


def _serve(reqs, delays, budget=0, k=16, mode=L.LBM_BATCH_STREAMS):
    srv = L.lbm_server_create(budget, k)
    try:
        L.lbm_server_set_batch_mode(srv, mode)
        ids = []
        for r, dly in zip(reqs, delays):
            time.sleep(dly)
            ids.append(L.lbm_server_submit(srv, r))
        out = []
        for i in ids:
            done, res = L.lbm_server_wait(srv, i, 120.0)
            assert done and res["status"] == 2, res
            out.append((res, L.lbm_server_force_history(srv, i)))
        stats = L.lbm_server_stats(srv)
    finally:
        L.lbm_server_destroy(srv)
    return out, stats


@pytest.mark.parametrize("mode", [L.LBM_BATCH_STREAMS, L.LBM_BATCH_PERSISTENT], ids=["streams", "persistent"])
def test_served_result_is_the_same_alone_and_in_the_mix(mode):
    reqs = [_req(Q, nx, ny, tau, om, n, **kw) for Q, nx, ny, tau, om, n, kw in REQS]
    mixed, stats = _serve(reqs, [0.0, 0.0, 0.01, 0.0, 0.02, 0.0], mode=mode)
    assert stats["completed"] == len(reqs) and stats["peak_running"] >= 2
    for r, (res_m, hist_m) in zip(reqs, mixed):
        (res_a, hist_a), = _serve([r], [0.0], mode=mode)[0]
        assert hist_m.shape == hist_a.shape == (r.desc.nsteps, 2)
        assert (hist_m == hist_a).all()
        for key in ("f_in", "f_q", "f_0", "gamma_bar"):
            assert res_m[key] == res_a[key], key
        assert res_m["admit_s"] >= res_m["submit_s"] and res_m["done_s"] >= res_m["admit_s"]


def test_served_fit_matches_direct_fit():
    r = _req(37, 70, 41, 0.9, 0.05, 400, skip=2.0)
    (res, hist), = _serve([r], [0.0])[0]
    h = L.lbm_create(37, 70, 41, 0.9, 0.05, r.desc.geom)
    try:
        L.lbm_set_variant(h, 2)   # the kernel the server's batches run D2Q37 FP32 instances with
        L.lbm_step(h, 400)
        F = L.lbm_force_history(h)
        f_in, f_q, f_0 = L.lbm_fit(h, 2.0)
    finally:
        L.lbm_destroy(h)
    assert (F == hist).all()
    assert (res["f_in"], res["f_q"], res["f_0"]) == (f_in, f_q, f_0)


def test_admission_waits_for_memory_in_arrival_order():
    reqs = [_req(37, 256, 256, 0.9, 0.05, 200) for _ in range(3)]
    need = L.lbm_batch_footprint(reqs[0].desc)
    out, stats = _serve(reqs, [0.0, 0.0, 0.0], budget=int(1.5 * need), k=32)
    assert stats["peak_running"] == 1 and stats["completed"] == 3
    admits = [res["admit_s"] for res, _ in out]
    dones = [res["done_s"] for res, _ in out]
    assert admits == sorted(admits)
    assert admits[1] >= dones[0] and admits[2] >= dones[1]


def test_request_larger_than_budget_is_rejected():
    srv = L.lbm_server_create(1 << 20, 16)
    try:
        with pytest.raises(L.LbmError) as e:
            L.lbm_server_submit(srv, _req(37, 256, 256, 0.9, 0.05, 50))
        assert e.value.code == L.LBM_ENOMEM
    finally:
        L.lbm_server_destroy(srv)


def test_in_place_layout_doubles_what_a_budget_admits():
    """The AA layout holds one population buffer: a budget that fits two two-buffer instances of a
    2048^2 D2Q37 FP32 beam fits at least three in-place ones, and the results are those of the
    two-buffer layout to FP32 rounding."""
    kw = dict(lx=32, ly=32)
    ab = [_req(37, 2048, 2048, 0.9, 0.2, 60, **kw) for _ in range(4)]     # 60 steps: 1.9 periods
    aa = [_req(37, 2048, 2048, 0.9, 0.2, 60, layout=L.LBM_LAYOUT_AA, **kw) for _ in range(4)]
    budget = int(2.2 * L.lbm_batch_footprint(ab[0].desc))
    assert 3 * L.lbm_batch_footprint(aa[0].desc) < budget
    out_ab, st_ab = _serve(ab, [0.0] * 4, budget=budget, k=8)
    out_aa, st_aa = _serve(aa, [0.0] * 4, budget=budget, k=8)
    assert st_ab["peak_running"] == 2 and st_aa["peak_running"] >= 3
    for (ra, ha), (rb, hb) in zip(out_aa, out_ab):
        amp = np.abs(hb[:, 0]).max()
        assert np.abs(ha[:, 0] - hb[:, 0]).max() <= 1e-5 * amp


@pytest.mark.parametrize("Q,kind,drive", [(37, L.LBM_GEOM_BEAM, L.LBM_DRIVE_BODYFORCE),
                                          (9, L.LBM_GEOM_PLATE, L.LBM_DRIVE_WALL),
                                          (9, L.LBM_GEOM_BEAM, L.LBM_DRIVE_BODYFORCE)],
                         ids=["q37-beam-body", "q9-plate-wall", "q9-beam-body"])
def test_served_fp16_request_matches_oracle(Q, kind, drive):
    """A served FP16 request (the mixed-precision form the server runs) against the FP64 oracle run
    of the same solve from rest: the in-phase and quadrature force of the fit agree within the
    stated 1e-4 of the force amplitude (error metric: |F_c - F_c^oracle| / sqrt(F_in^2 + F_q^2)).
    The request is served among others (an FP32 D2Q37 one and an FP16 one of the other lattice)."""
    import oracle as orc

    nx, ny, lx, ly, u0 = 96, 64, 16, 12, 1e-3
    P = 96
    omega, tau = 2 * np.pi / P, 0.9
    nsteps, skip = 3 * P, 1.0
    eq = 4 if Q == 37 else 2
    geo = dict(kind=kind, lx=lx, ly=ly, drive=drive, u0=u0, eq_order=eq, collision=L.LBM_COLL_REGULARIZED,
               storage=L.LBM_STORE_F16)
    perim = 2.0 * (lx + ly) if kind == L.LBM_GEOM_BEAM else float(nx)
    target = L.make_request(L.make_instance(Q, nx, ny, tau, omega, nsteps, **geo), skip, perim)
    other_q = 9 if Q == 37 else 37
    others = [_req(37, 70, 41, 0.9, 0.05, 200),
              _req(other_q, 80, 72, 0.8, 0.05, 250, storage=L.LBM_STORE_F16, lx=12, ly=9)]
    out, _ = _serve([others[0], target, others[1]], [0.0, 0.0, 0.005])
    res, hist = out[1]
    lab = orc.geometry_beam(nx, ny, lx, ly) if kind == L.LBM_GEOM_BEAM else orc.geometry_plate(Q, nx, ny)
    _, F_or = orc.run(Q, lab, tau, omega, u0, nsteps, eq_order=eq, collision=orc.COLL_REG, drive=drive,
                      nthreads=orc.max_threads())
    n0 = int(np.ceil(skip * 2 * np.pi / omega))   # the fit window of lbm_fit
    f_in, f_q = orc.in_phase_quadrature(F_or[:, 0], omega, drive, skip=n0)
    amp = float(np.hypot(f_in, f_q))
    assert amp > 0
    assert abs(res["f_in"] - f_in) <= 1e-4 * amp, (res["f_in"], f_in, amp)
    assert abs(res["f_q"] - f_q) <= 1e-4 * amp, (res["f_q"], f_q, amp)
