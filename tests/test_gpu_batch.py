"""GPU tests of the batched path: one persistent cooperative kernel over many uneven instances.

An instance's arithmetic in a batch is exactly that of lbm_step on the same instance (same kernel
body, same tile shape, same fixed-order force reduction), so batch results must equal standalone
results bit for bit, whatever else shares the launch; and one batch instance is checked against
the oracle as well.
"""
import math

import numpy as np
import pytest

import oracle as orc
from paper_0904_4504_gb300 import inputs as I
from paper_0904_4504_gb300 import lbm as L

from harness import oracle_state_to_g, scaled

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def _desc(Q, nx, ny, tau, omega, nsteps, storage=L.LBM_STORE_F32, coll=L.LBM_COLL_REGULARIZED, **kw):
    geo = dict(kind=L.LBM_GEOM_BEAM, lx=12, ly=9, drive=L.LBM_DRIVE_BODYFORCE, u0=1e-3, eq_order=4 if Q == 37 else 2,
               collision=coll, storage=storage)
    geo.update(kw)
    return L.make_instance(Q, nx, ny, tau, omega, nsteps, **geo)


def batch_kernel_variant(d, mode=L.LBM_BATCH_STREAMS):
    """The single-instance kernel that computes an instance as the batch does by default: in the
    streams mode the kernel the batch launches (lbm_batch_set_variant); in the persistent mode the
    kernel whose tile code and tile shape the persistent kernel runs (staged 64 x 3 tiles, variant
    27, with 16-bit storage; plain 32 x 4 tiles otherwise, variant 2 where built)."""
    g = d.geom
    if g.layout != L.LBM_LAYOUT_AB or g.wall_scheme != L.LBM_SCHEME_BOUNCEBACK:
        return 0
    half = g.storage in (L.LBM_STORE_BF16, L.LBM_STORE_F16)
    if mode == L.LBM_BATCH_PERSISTENT:
        if half:
            return 27
        return 2 if (d.lattice == 37 and g.storage != L.LBM_STORE_F64) else 0
    if half:
        return 27 if d.lattice == 37 else 30
    return 2 if (d.lattice == 37 and g.storage == L.LBM_STORE_F32) else 0


def _alone(d, mode=L.LBM_BATCH_STREAMS):
    """Run an instance description through the single-instance path, with the batch's kernel and
    tile shape (the tile shape fixes the order in which the FP64 force partials are summed)."""
    g = d.geom
    h = L.lbm_create(d.lattice, d.nx, d.ny, d.tau, d.omega, g)
    try:
        v = batch_kernel_variant(d, mode)
        if v:
            L.lbm_set_variant(h, v)
        else:
            L.lbm_set_tile(h, 32, 4)
        L.lbm_step(h, d.nsteps)
        return L.lbm_get_state(h), L.lbm_force_history(h)
    finally:
        L.lbm_destroy(h)


MIX = [  # uneven sizes, parameters, geometries and lengths
    (70, 41, 0.9, 0.05, 37, {}),
    (133, 64, 1.7, 0.04, 23, dict(lx=20, ly=30)),
    (96, 96, 0.6, 0.07, 41, dict(kind=L.LBM_GEOM_PLATE, drive=L.LBM_DRIVE_WALL)),
    (45, 200, 3.0, 0.03, 16, dict(lx=8, ly=40, eq_order=2)),
    (257, 33, 0.75, 0.06, 30, dict(kind=L.LBM_GEOM_NONE)),
]


MODES = [L.LBM_BATCH_STREAMS, L.LBM_BATCH_PERSISTENT]


@pytest.mark.parametrize("Q,st", [(37, L.LBM_STORE_F32), (37, L.LBM_STORE_F16), (37, L.LBM_STORE_BF16),
                                  (9, L.LBM_STORE_F16), (9, L.LBM_STORE_F32)],
                         ids=["q37-f32", "q37-f16", "q37-bf16", "q9-f16", "q9-f32"])
@pytest.mark.parametrize("mode", MODES, ids=["streams", "persistent"])
def test_batch_equals_standalone_bitwise(mode, Q, st):
    """Uneven instances (sizes, tau, omega, geometries, lengths, body-frame and lab-frame drives,
    with 16-bit storage the stream offset on) in one batch give exactly the states and forces of
    the same instances run alone with the kernel whose tile code the batch runs."""
    descs = [_desc(Q, nx, ny, tau, om, n, storage=st, **kw) for nx, ny, tau, om, n, kw in MIX]
    b = L.lbm_batch_create(Q, st, L.LBM_COLL_REGULARIZED)
    try:
        L.lbm_batch_set_mode(b, mode)
        slots = [L.lbm_batch_add(b, d) for d in descs]
        # uneven chunks; the longest instance needs 41 steps
        for k in (5, 1, 17, 3, 20):
            L.lbm_batch_run(b, k)
        L.lbm_batch_synchronize(b)
        info = L.lbm_batch_info(b)
        assert info["running"] == 0 and info["live"] == len(descs)
        for d, s in zip(descs, slots):
            done, total = L.lbm_batch_status(b, s)
            assert done == total == d.nsteps
            sim = L.lbm_batch_instance(b, s)
            g_b, F_b = L.lbm_get_state(sim), L.lbm_force_history(sim)
            g_a, F_a = _alone(d, mode)
            assert (g_b == g_a).all(), d.nx
            assert (F_b == F_a).all(), d.nx
    finally:
        L.lbm_batch_destroy(b)


@pytest.mark.parametrize("strip", [1, 3, 64])
@pytest.mark.parametrize("Q,st", [(37, L.LBM_STORE_F16), (37, L.LBM_STORE_F32), (9, L.LBM_STORE_F16)],
                         ids=["q37-f16", "q37-f32", "q9-f16"])
def test_persistent_strip_lengths_bitwise(Q, st, strip):
    """The persistent kernel's work items are strips of `strip` tile rows: one tile row per strip,
    a ragged last band, and strips longer than every instance (a single band, which is its own
    neighbour across the periodic seam) all give the standalone results bit for bit.  The mix adds
    the smallest grid a lattice allows (2R + 1 rows), whose bands of one tile row are shorter than
    the reach on the last row."""
    R = 3 if Q == 37 else 1
    mix = MIX + [(40, 2 * R + 1, 0.8, 0.05, 19, dict(kind=L.LBM_GEOM_NONE))]
    descs = [_desc(Q, nx, ny, tau, om, n, storage=st, **kw) for nx, ny, tau, om, n, kw in mix]
    b = L.lbm_batch_create(Q, st, L.LBM_COLL_REGULARIZED)
    try:
        L.lbm_batch_set_mode(b, L.LBM_BATCH_PERSISTENT)
        L.lbm_batch_set_segment(b, strip)
        slots = [L.lbm_batch_add(b, d) for d in descs]
        for k in (7, 2, 33):
            L.lbm_batch_run(b, k)
        L.lbm_batch_synchronize(b)
        for d, s in zip(descs, slots):
            sim = L.lbm_batch_instance(b, s)
            g_a, F_a = _alone(d, L.LBM_BATCH_PERSISTENT)
            assert (L.lbm_get_state(sim) == g_a).all(), (d.nx, d.ny)
            assert (L.lbm_force_history(sim) == F_a).all(), (d.nx, d.ny)
        with pytest.raises(L.LbmError):
            L.lbm_batch_set_segment(b, strip + 1)  # fixed once the persistent kernel has run
    finally:
        L.lbm_batch_destroy(b)


@pytest.mark.parametrize("mode", MODES)
def test_instances_joining_and_leaving_mid_run(mode):
    """An instance added after others ran, and another removed while others continue, do not change
    anyone's result."""
    d1 = _desc(37, 70, 41, 0.9, 0.05, 30)
    d2 = _desc(37, 96, 50, 1.3, 0.04, 25, lx=16, ly=16)
    d3 = _desc(37, 64, 64, 0.7, 0.06, 12, kind=L.LBM_GEOM_PLATE, drive=L.LBM_DRIVE_WALL)
    b = L.lbm_batch_create(37, L.LBM_STORE_F32, L.LBM_COLL_REGULARIZED)
    try:
        L.lbm_batch_set_mode(b, mode)
        s1 = L.lbm_batch_add(b, d1)
        s3 = L.lbm_batch_add(b, d3)
        L.lbm_batch_run(b, 7)
        s2 = L.lbm_batch_add(b, d2)        # joins at batch step 7
        L.lbm_batch_run(b, 6)
        L.lbm_batch_run(b, 9)              # d3 finishes at 12 inside this run
        L.lbm_batch_synchronize(b)
        g3 = L.lbm_get_state(L.lbm_batch_instance(b, s3))
        L.lbm_batch_remove(b, s3)
        L.lbm_batch_run(b, 40)
        L.lbm_batch_synchronize(b)
        for d, s, g_done in ((d1, s1, None), (d2, s2, None), (d3, None, g3)):
            g_a, F_a = _alone(d, mode)
            if s is None:
                assert (g_done == g_a).all()
                continue
            sim = L.lbm_batch_instance(b, s)
            assert (L.lbm_get_state(sim) == g_a).all()
            assert (L.lbm_force_history(sim) == F_a).all()
    finally:
        L.lbm_batch_destroy(b)


@pytest.mark.parametrize("mode", MODES)
def test_batch_instance_matches_oracle(mode):
    Q, nx, ny, tau, omega, n = 37, 70, 41, 0.9, 0.05, 20
    b = L.lbm_batch_create(Q, L.LBM_STORE_F64, L.LBM_COLL_REGULARIZED)
    try:
        L.lbm_batch_set_mode(b, mode)
        s = L.lbm_batch_add(b, _desc(Q, nx, ny, tau, omega, n, storage=L.LBM_STORE_F64))
        L.lbm_batch_add(b, _desc(Q, 64, 64, 0.7, 0.06, 9, storage=L.LBM_STORE_F64))
        L.lbm_batch_run(b, n)
        L.lbm_batch_synchronize(b)
        sim = L.lbm_batch_instance(b, s)
        g, F = L.lbm_get_state(sim), L.lbm_force_history(sim)
    finally:
        L.lbm_batch_destroy(b)
    lab = orc.geometry_beam(nx, ny, 12, 9)
    f, F_or = orc.run(Q, lab, tau, omega, 1e-3, n, eq_order=4, collision=orc.COLL_REG, drive=orc.DRIVE_BODY,
                      nthreads=orc.max_threads())
    g_or = oracle_state_to_g(Q, f)
    fl = lab == 0
    err = np.abs(scaled(Q, g)[:, fl] - scaled(Q, g_or)[:, fl]).max()
    assert err <= 2e-13 * n * np.abs(scaled(Q, g_or)[:, fl]).max() + n * 2e-15
    assert np.abs(F[:, 0] - F_or[:, 0]).max() <= 1e-11 * np.abs(F_or[:, 0]).max()


def test_barrier_timeout_is_reported_not_hung():
    """A barrier wait that runs out (limit 0: give up at once) ends the kernel and is reported."""
    b = L.lbm_batch_create(37, L.LBM_STORE_F32, L.LBM_COLL_REGULARIZED)
    try:
        L.lbm_batch_set_mode(b, L.LBM_BATCH_PERSISTENT)
        for k in range(3):
            L.lbm_batch_add(b, _desc(37, 256, 256, 0.9, 0.05, 10))
        assert L.lbm_batch_info(b)["max_blocks"] > 1
        L.lbm_batch_set_barrier_limit(b, 0)
        L.lbm_batch_run(b, 4)
        with pytest.raises(L.LbmError) as e:
            L.lbm_batch_synchronize(b)
        assert e.value.code == L.LBM_ETIMEOUT
    finally:
        L.lbm_batch_destroy(b)
    # the context is still usable afterwards
    h = L.lbm_create(37, 64, 48, 0.9, 0.05, L.make_geometry(kind=L.LBM_GEOM_NONE))
    L.lbm_step(h, 2)
    L.lbm_synchronize(h)
    L.lbm_destroy(h)


def test_admission_by_footprint():
    d = _desc(37, 512, 512, 0.9, 0.05, 100)
    need = L.lbm_batch_footprint(d)
    assert need >= 2 * 37 * 512 * 512 * 4
    b = L.lbm_batch_create(37, L.LBM_STORE_F32, L.LBM_COLL_REGULARIZED, int(1.5 * need))
    try:
        L.lbm_batch_add(b, d)
        with pytest.raises(L.LbmError) as e:
            L.lbm_batch_add(b, d)
        assert e.value.code == L.LBM_ENOMEM
        assert L.lbm_batch_info(b)["live"] == 1
    finally:
        L.lbm_batch_destroy(b)


@pytest.mark.parametrize("mode", MODES)
def test_batch_sweep_shapes_run(mode):
    """The 64-instance sweep (sizes 256..1024, AR 0.25..2) fits and runs a few steps."""
    b = L.lbm_batch_create(37, L.LBM_STORE_F32, L.LBM_COLL_REGULARIZED)
    try:
        L.lbm_batch_set_mode(b, mode)
        for w in I.sweep_d2q37():
            tau, omega, P = orc.params_from_tau_omega(37, w.tau_omega)
            L.lbm_batch_add(b, L.make_instance(37, w.nx, w.ny, tau, omega, int(w.periods * P), kind=w.geometry,
                                               lx=w.lx, ly=w.ly, drive=w.drive, u0=w.u0, eq_order=4,
                                               collision=w.collision, storage=w.storage))
        L.lbm_batch_run(b, 3)
        L.lbm_batch_synchronize(b)
        info = L.lbm_batch_info(b)
        assert info["live"] == 64 and info["running"] == 64 and info["mode"] == mode
    finally:
        L.lbm_batch_destroy(b)


def test_damping_sweep_matches_direct_fit():
    """The Q(p) sweep driver gives the gamma_bar of a direct run of the same instance."""
    from paper_0904_4504_gb300 import resonators as R
    rec = R.damping_sweep([1.0], 1.0, side=128, periods=4, lx_max=16, ly_max=16)[0]
    P = rec["period"]
    tau, omega, P = L.lbm_params_from_tau_omega(37, 1.0, p_min=P)
    assert (tau, omega) == (rec["tau"], rec["omega"]) and rec["u0"] == 1e-3
    geom = L.make_geometry(kind=L.LBM_GEOM_BEAM, lx=16, ly=16, drive=L.LBM_DRIVE_BODYFORCE, u0=1e-3, eq_order=4,
                           storage=L.LBM_STORE_F32)
    h = L.lbm_create(37, 128, 128, tau, omega, geom)
    try:
        L.lbm_set_variant(h, 2)   # the batch's default kernel for D2Q37 FP32
        L.lbm_step(h, 4 * P)
        f_in, _, _ = L.lbm_fit(h, 2.0)
        direct = L.lbm_gamma_bar(h, f_in, 64.0)
    finally:
        L.lbm_destroy(h)
    assert rec["gamma_bar"] == direct and direct > 0


@pytest.mark.parametrize("Q", [37, 9])
@pytest.mark.parametrize("st", [L.LBM_STORE_BF16, L.LBM_STORE_F16], ids=["bf16", "f16"])
@pytest.mark.parametrize("mode", MODES, ids=["streams", "persistent"])
def test_batch_16bit_instances_match_oracle_step(mode, st, Q):
    """16-bit storage in a batch (the mixed-precision form): after 9 batch steps, each instance's
    10th step against one oracle step from the state it reached, with the bound of the 16-bit
    parity tests (the exact step rounded once to the storage type, relative to |h| plus the stream
    offset in the body frame).  Instances: a body-frame beam with interior (staged) tiles, a
    lab-frame beam and a plate with its moving wall, of uneven sizes."""
    from harness import g_to_oracle_state, stream_offset_magnitude
    from test_gpu_parity import assert_force_close, assert_state_close

    u0 = 2e-3
    eq = 4 if Q == 37 else 2
    cases = [(393, 90, 0.9, 0.05, dict(lx=23, ly=19)),
             (140, 75, 1.3, 0.04, dict(lx=16, ly=24, drive=L.LBM_DRIVE_WALL)),
             (96, 64, 0.7, 0.06, dict(kind=L.LBM_GEOM_PLATE, drive=L.LBM_DRIVE_WALL))]
    b = L.lbm_batch_create(Q, st, L.LBM_COLL_REGULARIZED)
    try:
        L.lbm_batch_set_mode(b, mode)
        descs = [_desc(Q, nx, ny, tau, om, 40, storage=st, u0=u0, **kw) for nx, ny, tau, om, kw in cases]
        slots = [L.lbm_batch_add(b, d) for d in descs]
        L.lbm_batch_run(b, 4)
        L.lbm_batch_run(b, 5)
        L.lbm_batch_synchronize(b)
        g9 = [L.lbm_get_state(L.lbm_batch_instance(b, s)) for s in slots]
        L.lbm_batch_run(b, 1)
        L.lbm_batch_synchronize(b)
        g10 = [L.lbm_get_state(L.lbm_batch_instance(b, s)) for s in slots]
        F = [L.lbm_force_history(L.lbm_batch_instance(b, s)) for s in slots]
    finally:
        L.lbm_batch_destroy(b)
    for d, a, z, Fh in zip(descs, g9, g10, F):
        g = d.geom
        lab = (orc.geometry_beam(d.nx, d.ny, g.lx, g.ly) if g.kind == L.LBM_GEOM_BEAM
               else orc.geometry_plate(Q, d.nx, d.ny))
        f, F_or = orc.run(Q, lab, d.tau, d.omega, u0, 1, eq_order=eq, collision=orc.COLL_REG, drive=g.drive,
                          f=g_to_oracle_state(Q, a), n0=9, nthreads=orc.max_threads())
        off = u0 * stream_offset_magnitude(Q, u0, d.omega, 10, eq) if g.drive == L.LBM_DRIVE_BODYFORCE else None
        assert_state_close(Q, z, oracle_state_to_g(Q, f), lab, st, 1, a, off)
        assert_force_close(Fh[9:10], F_or, Q, lab, st, 1)
