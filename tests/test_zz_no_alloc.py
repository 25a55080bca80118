"""lbm_step_noalloc against lbm_step: two steps in a row, the same states and forces.

lbm_step_noalloc serves callers that must not allocate device memory when they step the solver
(work recorded into a CUDA graph, device memory owned by another allocator, fixed budgets).  This
test drives it through the C ABI with buffers the test allocates itself (torch), for two calls in
a row (the second reusing the shared static scratch the first left behind), and compares the
states and forces with the library's regular path, lbm_step, within the FP32 parity tolerance.
The file name puts it last in collection, so a run that stops at the first failure has already
run every other test.
"""
import numpy as np
import pytest

from paper_0904_4504_gb300 import inputs as I
from paper_0904_4504_gb300 import lbm as L

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

EPS_F32_STEP = 4e-6   # FP32 per-step bound of the parity tests, relative to the state scale


def _geom():
    return L.make_geometry(kind=L.LBM_GEOM_BEAM, lx=20, ly=13, drive=L.LBM_DRIVE_BODYFORCE, u0=2e-3, eq_order=4,
                           collision=L.LBM_COLL_REGULARIZED, storage=L.LBM_STORE_F32)


def test_noalloc_matches_lbm_step_on_two_calls():
    Q, nx, ny, tau, omega = 37, 133, 71, 0.9, 0.05
    _, w, _ = L.lbm_lattice_velocities(Q)

    # regular path: library-owned buffers
    ref = L.lbm_create(Q, nx, ny, tau, omega, _geom())
    try:
        lab = L.lbm_get_labels(ref)
        h0 = I.random_scaled_state(Q, nx, ny, -17, seed=21)
        h0[:, lab != 0] = 0.0
        L.lbm_set_state(ref, h0 * w[:, None, None])
        L.lbm_step(ref, 1)
        g1 = L.lbm_get_state(ref)
        L.lbm_step(ref, 1)
        g2 = L.lbm_get_state(ref)
        F = L.lbm_force_history(ref)
    finally:
        L.lbm_destroy(ref)

    # no-allocation path: caller-owned state and force buffers
    sim = L.lbm_create(Q, nx, ny, tau, omega, _geom())
    try:
        info = L.lbm_info(sim)
        assert info["storage"] == L.LBM_STORE_F32
        pitch = info["pitch"]
        a = torch.zeros((Q, ny, pitch), dtype=torch.float32, device="cuda")
        a[:, :, :nx] = torch.from_numpy(h0.astype(np.float32)).cuda()
        b = torch.zeros_like(a)
        force = torch.full((2, 2), float("nan"), dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream()
        L.lbm_step_noalloc(sim, 0, a.data_ptr(), b.data_ptr(), force[0].data_ptr(), stream)
        L.lbm_step_noalloc(sim, 1, b.data_ptr(), a.data_ptr(), force[1].data_ptr(), stream)
        torch.cuda.synchronize()
        s1 = b[:, :, :nx].double().cpu().numpy() * w[:, None, None]
        s2 = a[:, :, :nx].double().cpu().numpy() * w[:, None, None]
        Fn = force.cpu().numpy()
        assert L.lbm_info(sim)["steps_done"] == 0   # the simulation's own state is untouched
    finally:
        L.lbm_destroy(sim)

    fl = lab == 0
    scale = np.abs(h0[:, fl]).max()
    for k, (got, want) in enumerate([(s1, g1), (s2, g2)], start=1):
        err = np.abs((got - want) / w[:, None, None])[:, fl].max()
        assert err <= EPS_F32_STEP * k * scale, (k, err)
    for k in range(2):
        for c in range(2):
            assert abs(Fn[k, c] - F[k, c]) <= EPS_F32_STEP * (k + 1) * (abs(F[k, c]) + 1.0), (k, c, Fn[k], F[k])


def test_noalloc_rejects_bad_buffers():
    sim = L.lbm_create(37, 64, 48, 0.9, 0.05, _geom())
    try:
        with pytest.raises(L.LbmError) as e:
            L.lbm_step_noalloc(sim, 0, 0, 0, 0)
        assert e.value.code == L.LBM_EINVAL
        buf = torch.zeros(16, device="cuda")
        with pytest.raises(L.LbmError) as e:
            L.lbm_step_noalloc(sim, 0, buf.data_ptr(), buf.data_ptr(), buf.data_ptr())
        assert e.value.code == L.LBM_EINVAL and "different" in L.lbm_last_error()
    finally:
        L.lbm_destroy(sim)
