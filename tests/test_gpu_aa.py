"""In-place streaming (LBM_LAYOUT_AA): one population buffer, even steps pull and push, odd steps
stay at the node.  Parity against the FP64 oracle with the tolerances of test_gpu_parity (the
arithmetic of a step is the same; only where values are read and written changes), chunked runs
with odd chunk lengths (each launch alternates the two kernels), the forces of both kinds of step,
and the calls that the layout rejects."""
import math

import numpy as np
import pytest

import oracle as orc
from paper_0904_4504_gb300 import inputs as I
from paper_0904_4504_gb300 import lbm as L

from harness import scaled, stream_offset_magnitude
from test_gpu_parity import EPS_STEP, ROUND16, assert_force_close, assert_state_close, run_both

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

AA = L.LBM_LAYOUT_AA

CASES = [
    # id, Q, nx, ny, kind, lx, ly, drive, eq, coll, storage, steps, tile
    ("q9-bgk-plate-f64", 9, 45, 37, L.LBM_GEOM_PLATE, 0, 0, L.LBM_DRIVE_WALL, 2, L.LBM_COLL_BGK, L.LBM_STORE_F64, 40,
     None),
    ("q9-reg-beam-body-f64", 9, 45, 37, L.LBM_GEOM_BEAM, 9, 7, L.LBM_DRIVE_BODYFORCE, 2, L.LBM_COLL_REGULARIZED,
     L.LBM_STORE_F64, 40, (64, 2)),
    ("q37-reg-h4-beam-body-f64", 37, 70, 41, L.LBM_GEOM_BEAM, 12, 9, L.LBM_DRIVE_BODYFORCE, 4,
     L.LBM_COLL_REGULARIZED, L.LBM_STORE_F64, 34, (32, 4)),
    ("q37-reg-h4-beam-lab-f64", 37, 70, 41, L.LBM_GEOM_BEAM, 12, 9, L.LBM_DRIVE_WALL, 4,
     L.LBM_COLL_REGULARIZED, L.LBM_STORE_F64, 34, None),
    ("q37-bgk-h4-mask-wall-f64", 37, 67, 53, L.LBM_GEOM_MASK, 0, 0, L.LBM_DRIVE_WALL, 4, L.LBM_COLL_BGK,
     L.LBM_STORE_F64, 28, (128, 2)),
    ("q37-reg-h2-plate-f32", 37, 45, 50, L.LBM_GEOM_PLATE, 0, 0, L.LBM_DRIVE_WALL, 2,
     L.LBM_COLL_REGULARIZED, L.LBM_STORE_F32, 34, None),
    ("q37-reg-h4-beam-body-f32", 37, 70, 41, L.LBM_GEOM_BEAM, 12, 9, L.LBM_DRIVE_BODYFORCE, 4,
     L.LBM_COLL_REGULARIZED, L.LBM_STORE_F32, 34, None),
    ("q37-bgk-h4-mask-wall-f32", 37, 67, 53, L.LBM_GEOM_MASK, 0, 0, L.LBM_DRIVE_WALL, 4, L.LBM_COLL_BGK,
     L.LBM_STORE_F32, 28, (64, 4)),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_aa_parity(case):
    """Random exact start, run in 3 chunks of odd and even length (both kernels start chunks)."""
    name, Q, nx, ny, kind, lx, ly, drive, eq, coll, st, steps, tile = case
    mask = I.random_mask(nx, ny, 3 if Q == 37 else 1, seed=7) if kind == L.LBM_GEOM_MASK else None
    g_gpu, g_or, F_gpu, F_or, lab, g0 = run_both(Q, nx, ny, 0.83, 0.05, kind, steps, lx=lx, ly=ly, mask=mask,
                                                 drive=drive, u0=2e-3, eq_order=eq, collision=coll, storage=st,
                                                 init_exp=-17, seed=11, tile=tile, n0_chunks=3, layout=AA)
    assert steps % 2 == 0 and (steps // 3) % 2 == 1  # chunks of odd length
    assert_state_close(Q, g_gpu, g_or, lab, st, steps, g0)
    assert_force_close(F_gpu, F_or, Q, lab, st, steps)


@pytest.mark.parametrize("drive", [L.LBM_DRIVE_BODYFORCE, L.LBM_DRIVE_WALL])
@pytest.mark.parametrize("st", [L.LBM_STORE_BF16, L.LBM_STORE_F16])
def test_aa_parity_16bit_two_steps(st, drive):
    """Two steps from a 16-bit-exact state (one pull-push and one local kernel), body frame with the
    stream offset and lab frame without.  Each value is rounded once per step; the first rounding
    reaches the second step through the collision, whose output depends on all 37 inputs with
    weights summing to a few units, so 8 half-ulps of the state scale are allowed on top."""
    Q, nx, ny, u0 = 37, 70, 41, 2e-3
    g_gpu, g_or, F_gpu, F_or, lab, g0 = run_both(Q, nx, ny, 0.9, 0.05, L.LBM_GEOM_BEAM, 2, lx=12, ly=9,
                                                 drive=drive, u0=u0, eq_order=4, storage=st, init_exp=-7, seed=5,
                                                 layout=AA)
    fl = lab == 0
    hg, ho = scaled(Q, g_gpu)[:, fl], scaled(Q, g_or)[:, fl]
    scale = max(np.abs(ho).max(), np.abs(scaled(Q, g0)[:, fl]).max())
    mag = np.abs(ho)
    if drive == L.LBM_DRIVE_BODYFORCE:
        mag = mag + (u0 * stream_offset_magnitude(Q, u0, 0.05, 2, 4))[:, None]
    bound = EPS_STEP[st] * 2 * scale + ROUND16[st] * (mag + 8 * scale)
    err = np.abs(hg - ho)
    assert (err <= bound).all(), (err.max(), (err / bound).max())
    assert_force_close(F_gpu, F_or, Q, lab, st, 2)


@pytest.mark.parametrize("storage", [L.LBM_STORE_F32, L.LBM_STORE_F16])
def test_aa_matches_two_buffers_at_full_size(storage):
    """The headline beam (D2Q37-H4, 32 x 32 in 1024^2, body frame, tau*omega = 1) for 8 periods in
    both layouts: force histories agree to the FP32 (16-bit) rounding of the state, and so do the
    in-phase and quadrature fits."""
    w = I.beam_d2q37_h4(1.0, n=1024, storage=storage)
    tau, omega, P = L.lbm_params_from_tau_omega(37, 1.0)
    out = {}
    for layout in (L.LBM_LAYOUT_AB, AA):
        geom = L.make_geometry(kind=w.geometry, lx=w.lx, ly=w.ly, drive=w.drive, u0=w.u0, eq_order=w.eq_order,
                               collision=w.collision, storage=storage, layout=layout)
        h = L.lbm_create(37, 1024, 1024, tau, omega, geom)
        try:
            info = L.lbm_info(h)
            assert info["layout"] == layout
            L.lbm_step(h, 8 * P)
            out[layout] = (L.lbm_force_history(h), L.lbm_fit(h, 4.0), info["device_bytes"])
        finally:
            L.lbm_destroy(h)
    (Fa, fit_a, bytes_a), (Fb, fit_b, bytes_b) = out[AA], out[L.LBM_LAYOUT_AB]
    amp = math.hypot(fit_b[0], fit_b[1])
    tol = 1e-5 if storage == L.LBM_STORE_F32 else 1e-3
    assert np.abs(Fa[:, 0] - Fb[:, 0]).max() <= tol * amp
    assert abs(fit_a[0] - fit_b[0]) <= tol * amp and abs(fit_a[1] - fit_b[1]) <= tol * amp
    pop = 37 * 1024 * 1024 * L.STORAGE_BYTES[storage]
    assert bytes_b - bytes_a >= pop  # one population buffer fewer


def test_aa_rejections():
    geom = L.make_geometry(kind=L.LBM_GEOM_BEAM, lx=12, ly=9, drive=L.LBM_DRIVE_BODYFORCE, u0=1e-3, eq_order=4,
                           storage=L.LBM_STORE_F16, layout=AA)
    h = L.lbm_create(37, 70, 41, 0.9, 0.05, geom)
    try:
        with pytest.raises(L.LbmError) as e:
            L.lbm_set_variant(h, 11)
        assert e.value.code == L.LBM_EINVAL
        L.lbm_step(h, 3)
        with pytest.raises(L.LbmError) as e:
            L.lbm_get_state(h)
        assert e.value.code == L.LBM_ERANGE
        L.lbm_step(h, 1)
        assert L.lbm_get_state(h).shape == (37, 41, 70)
        assert L.lbm_force_history(h).shape == (4, 2)
    finally:
        L.lbm_destroy(h)
    ds = L.make_geometry(kind=L.LBM_GEOM_BEAM, lx=12, ly=9, drive=L.LBM_DRIVE_WALL, u0=1e-3, storage=L.LBM_STORE_F32,
                         wall_scheme=L.LBM_SCHEME_DIFFUSE, layout=AA)
    with pytest.raises(L.LbmError) as e:
        L.lbm_create(37, 70, 41, 0.9, 0.05, ds)
    assert e.value.code == L.LBM_EINVAL
    b = L.lbm_batch_create(37, L.LBM_STORE_F32, L.LBM_COLL_REGULARIZED)
    try:
        L.lbm_batch_set_mode(b, L.LBM_BATCH_PERSISTENT)
        d = L.make_instance(37, 70, 41, 0.9, 0.05, 10, kind=L.LBM_GEOM_BEAM, lx=12, ly=9, u0=1e-3,
                            storage=L.LBM_STORE_F32, layout=AA)
        with pytest.raises(L.LbmError) as e:
            L.lbm_batch_add(b, d)
        assert e.value.code == L.LBM_EINVAL
    finally:
        L.lbm_batch_destroy(b)


def test_aa_in_a_streams_batch_is_bitwise_standalone():
    """Instances of the streams batch run the same kernels on their own streams: bitwise the same
    force history as the instance alone."""
    Q = 37
    tau, omega, P = L.lbm_params_from_tau_omega(Q, 1.0)
    descs = [L.make_instance(Q, n, n, tau, omega, 3 * P + k, kind=L.LBM_GEOM_BEAM, lx=16, ly=8 * (k + 1),
                             drive=L.LBM_DRIVE_BODYFORCE, u0=1e-3, eq_order=4, storage=L.LBM_STORE_F16, layout=AA)
             for k, n in enumerate((128, 192, 256))]
    b = L.lbm_batch_create(Q, L.LBM_STORE_F16, L.LBM_COLL_REGULARIZED)
    try:
        slots = [L.lbm_batch_add(b, d) for d in descs]
        L.lbm_batch_run(b, max(d.nsteps for d in descs))
        L.lbm_batch_synchronize(b)
        batched = [L.lbm_force_history(L.lbm_batch_instance(b, s)) for s in slots]
    finally:
        L.lbm_batch_destroy(b)
    for d, Fb in zip(descs, batched):
        h = L.lbm_create(Q, d.nx, d.ny, d.tau, d.omega, d.geom)
        try:
            L.lbm_set_tile(h, 32, 4)
            L.lbm_step(h, d.nsteps)
            Fs = L.lbm_force_history(h)
        finally:
            L.lbm_destroy(h)
        assert Fb.shape == Fs.shape and np.array_equal(Fb, Fs)
