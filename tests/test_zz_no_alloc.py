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


def _geom(storage=L.LBM_STORE_F32, lx=20, ly=13):
    return L.make_geometry(kind=L.LBM_GEOM_BEAM, lx=lx, ly=ly, drive=L.LBM_DRIVE_BODYFORCE, u0=2e-3, eq_order=4,
                           collision=L.LBM_COLL_REGULARIZED, storage=storage)


@pytest.mark.parametrize("variant", [None, 26])
def test_noalloc_matches_lbm_step_on_two_calls(variant):
    """variant 26: the simulation's tile is 64 x 3 (the staged kernel's), so the tile slots the
    static scratch holds are those of that shape; lbm_step runs the staged kernel, the
    no-allocation step the plain kernel on the same tiles."""
    Q, nx, ny, tau, omega = 37, 133, 71, 0.9, 0.05
    _, w, _ = L.lbm_lattice_velocities(Q)

    # regular path: library-owned buffers
    ref = L.lbm_create(Q, nx, ny, tau, omega, _geom())
    try:
        if variant is not None:
            L.lbm_set_variant(ref, variant)
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
        if variant is not None:
            L.lbm_set_variant(sim, variant)
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


def test_noalloc_fp16_body_force_against_oracle():
    """16-bit storage with the body-force drive: lbm_step stores the populations relative to the
    uniform stream, the no-allocation step plain scaled deviations.  Two calls from a 16-bit-exact
    state; after each, one FP64 oracle step from the state the call started from, rounded once to
    FP16, is what the call must give (bound of the parity tests: 2^-11 of each value plus the FP32
    part), and the forces agree to the same bound."""
    import oracle as orc
    from harness import g_to_oracle_state, oracle_state_to_g, scaled

    Q, nx, ny, tau, omega, u0 = 37, 133, 71, 0.9, 0.05, 2e-3
    _, w, _ = L.lbm_lattice_velocities(Q)
    sim = L.lbm_create(Q, nx, ny, tau, omega, _geom(L.LBM_STORE_F16))
    try:
        lab = L.lbm_get_labels(sim)
        pitch = L.lbm_info(sim)["pitch"]
        h0 = I.random_scaled_state(Q, nx, ny, -7, seed=31)
        h0[:, lab != 0] = 0.0
        a = torch.zeros((Q, ny, pitch), dtype=torch.float16, device="cuda")
        a[:, :, :nx] = torch.from_numpy(h0.astype(np.float16)).cuda()
        b = torch.zeros_like(a)
        force = torch.full((2, 2), float("nan"), dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream()
        L.lbm_step_noalloc(sim, 4, a.data_ptr(), b.data_ptr(), force[0].data_ptr(), stream)
        torch.cuda.synchronize()
        h1 = b[:, :, :nx].double().cpu().numpy()
        L.lbm_step_noalloc(sim, 5, b.data_ptr(), a.data_ptr(), force[1].data_ptr(), stream)
        torch.cuda.synchronize()
        h2 = a[:, :, :nx].double().cpu().numpy()
        Fn = force.cpu().numpy()
    finally:
        L.lbm_destroy(sim)
    fl = lab == 0
    for k, (hin, hout) in enumerate([(h0, h1), (h1, h2)]):
        g_in = hin * w[:, None, None] * u0
        f, F_or = orc.run(Q, lab, tau, omega, u0, 1, eq_order=4, collision=orc.COLL_REG, drive=orc.DRIVE_BODY,
                          f=g_to_oracle_state(Q, g_in), n0=4 + k, nthreads=orc.max_threads())
        want = scaled(Q, oracle_state_to_g(Q, f))[:, fl] / u0
        got = hout[:, fl]
        scale = max(np.abs(want).max(), np.abs(hin[:, fl]).max())
        err = np.abs(got - want)
        bound = EPS_F32_STEP * scale + 2.0 ** -11 * np.abs(want) + 1e-12 * scale
        assert (err <= bound).all(), (k, err.max(), (err / bound).max())
        c, wo, _ = orc.lattice(Q)
        link_scale = 2.0 * np.abs(c).sum(1).dot(wo) * int((lab == 1).sum())
        for comp in range(2):
            tol = (EPS_F32_STEP + 2.0 ** -11) * (link_scale + abs(F_or[0, comp]))
            assert abs(Fn[k, comp] - F_or[0, comp]) <= tol, (k, comp, Fn[k], F_or[0])


def test_noalloc_rejects_geometries_beyond_the_scratch():
    """A tall beam on 32 x 1 tiles: two tiles of every row along its sides hold body links, more
    than LBM_NOALLOC_MAX_SLOTS in all, so the step is refused with LBM_ERANGE (nothing runs)."""
    sim = L.lbm_create(37, 64, 4200, 0.9, 0.05, _geom(lx=16, ly=4100))
    try:
        L.lbm_set_tile(sim, 32, 1)
        buf = torch.zeros(16, device="cuda")
        out = torch.zeros(16, device="cuda")
        with pytest.raises(L.LbmError) as e:
            L.lbm_step_noalloc(sim, 0, buf.data_ptr(), out.data_ptr(), out.data_ptr())
        assert e.value.code == L.LBM_ERANGE and "scratch" in L.lbm_last_error()
    finally:
        L.lbm_destroy(sim)


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
