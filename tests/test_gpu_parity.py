"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle, element by element.

Every case starts both sides from the same state: either rest, or a random state whose values are
exact in every storage type (k * 2^e, |k| <= 255).  States are compared as h = g / w (each
direction on the same scale) at fluid nodes; forces per component.

Tolerances, from the arithmetic:
  * FP64 storage and arithmetic: every output is a short FP64 expression of ~40 inputs, so one step
    differs by at most ~1000 units of 2^-53 of the state scale: 2e-13 per step.
  * FP32 arithmetic (FP32/BF16/FP16 storage): the moments sum 37 terms (relative rounding
    37 * 2^-24 ~ 2.2e-6 of the largest term) and the collision adds a few more roundings, so one
    step differs by <= 4e-6 of the state scale; over n steps the rounding errors are damped by the
    collision but add, and we allow 4e-6 * n.
  * BF16/FP16 storage: one step ends with a rounding to 8 (11) significant bits, so each output
    differs from the exact step by at most half a unit in the last place, 2^-8 (2^-11) of itself,
    plus the FP32 part.
The state scale is the largest |h| of the initial and the final state (rounding errors are made
while the values are large; a decaying field must not shrink the bound).
The D2Q37 weights as printed (Appendix A) sum to 1 - 1.2e-15.  The oracle stores full f and
rebuilds rho from them, so each collision scales its mass by about that sum; the library stores
deviations from w_i rho0 and does not.  That drift, |1 - sum w| rho0 per step in h units, is added
to the bound.  For the same reason the oracle's own rounding is relative to rho0, not to the
deviations: each step evaluates its outputs from O(rho0) values in a few dozen operations, so up
to 64 units of 2^-53 of rho0 per step are added as well (they are damped by the collision unless
tau is large, and matter only for FP64 storage).
The wall force sums link terms of size ~ w rho0; it is compared against the same per-dtype bounds
times the sum of the absolute link momenta (the constant part |F_const| plus max |F|).
"""
import math

import numpy as np
import pytest

import oracle as orc
from paper_0904_4504_gb300 import inputs as I
from paper_0904_4504_gb300 import lbm as L

from harness import g_to_oracle_state, oracle_labels, oracle_state_to_g, scaled, stream_offset_magnitude

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

EPS_STEP = {L.LBM_STORE_F64: 2e-13, L.LBM_STORE_F32: 4e-6, L.LBM_STORE_BF16: 4e-6, L.LBM_STORE_F16: 4e-6}
ROUND16 = {L.LBM_STORE_BF16: 2.0 ** -8, L.LBM_STORE_F16: 2.0 ** -11}


def run_both(Q, nx, ny, tau, omega, kind, steps, *, lx=0, ly=0, mask=None, drive=L.LBM_DRIVE_WALL, u0=1e-3,
             eq_order=2, collision=L.LBM_COLL_REGULARIZED, storage=L.LBM_STORE_F64, init_exp=None, seed=0,
             tile=None, n0_chunks=1, wall=L.LBM_SCHEME_BOUNCEBACK, layout=L.LBM_LAYOUT_AB, variant=None):
    """Run `steps` steps on the GPU and on the oracle; returns (g_gpu, g_or, F_gpu, F_or, labels, g0)."""
    geom = L.make_geometry(kind=kind, lx=lx, ly=ly, drive=drive, u0=u0, mask=mask, eq_order=eq_order,
                           collision=collision, storage=storage, wall_scheme=wall, layout=layout)
    lab_or = oracle_labels(kind, Q, nx, ny, lx, ly, mask)
    s = 1.0 if L.STORAGE_BYTES[storage] > 2 else u0
    _, w, _ = L.lbm_lattice_velocities(Q)
    g0 = None
    if init_exp is not None:
        h0 = I.random_scaled_state(Q, nx, ny, init_exp, seed)
        h0[:, lab_or != 0] = 0.0
        g0 = h0 * w[:, None, None] * s
    h = L.lbm_create(Q, nx, ny, tau, omega, geom)
    try:
        assert (L.lbm_get_labels(h) == lab_or).all()
        if tile:
            L.lbm_set_tile(h, *tile)
        if variant is not None:
            L.lbm_set_variant(h, variant)
            assert L.lbm_info(h)["variant"] == variant
        if g0 is not None:
            L.lbm_set_state(h, g0)
        chunk = steps // n0_chunks
        done = 0
        while done < steps:
            k = min(chunk, steps - done)
            L.lbm_step(h, k)
            done += k
        g_gpu = L.lbm_get_state(h)
        F_gpu = L.lbm_force_history(h)
    finally:
        L.lbm_destroy(h)
    f0 = g_to_oracle_state(Q, g0) if g0 is not None else None
    f, F_or = orc.run(Q, lab_or, tau, omega, u0, steps, eq_order=eq_order, collision=collision, drive=drive, f=f0,
                      nthreads=orc.max_threads(), wall=wall)
    return g_gpu, oracle_state_to_g(Q, f), F_gpu, F_or, lab_or, g0


def assert_state_close(Q, g_gpu, g_or, lab, storage, steps, g0=None, offset=None):
    """offset: s |H_i| (in g/w units) of the 16-bit body-frame stream offset, if the run used it:
    16-bit storage rounds h - H, so the rounding bound is relative to |h| + |H|."""
    fl = lab == 0
    hg, ho = scaled(Q, g_gpu)[:, fl], scaled(Q, g_or)[:, fl]
    scale = max(np.abs(ho).max(), 1e-300)
    if g0 is not None:
        scale = max(scale, np.abs(scaled(Q, g0)[:, fl]).max())
    err = np.abs(hg - ho)
    _, w_or, _ = orc.lattice(Q)
    drift = steps * (abs(1.0 - w_or.sum()) + 64 * 2.0 ** -53)
    mag = np.abs(ho)
    if offset is not None and storage in ROUND16:
        mag = mag + np.asarray(offset)[:, None]
    bound = EPS_STEP[storage] * steps * scale + ROUND16.get(storage, 0.0) * mag + drift
    assert (err <= bound).all(), f"max err {err.max():.3e} (scale {scale:.3e}), worst ratio {(err / bound).max():.3f}"


def assert_force_close(F_gpu, F_or, Q, lab, storage, steps, rho0=1.0):
    assert F_gpu.shape == F_or.shape
    c, w, _ = orc.lattice(Q)
    link_scale = 2.0 * rho0 * np.abs(c).sum(1).dot(w) * max(1, int((lab == 1).sum()))
    for comp in (0, 1):
        scale = link_scale + np.abs(F_or[:, comp]).max()
        err = np.abs(F_gpu[:, comp] - F_or[:, comp]).max()
        tol = (EPS_STEP[storage] * steps + ROUND16.get(storage, 0.0)) * scale
        assert err <= tol, f"force[{comp}] err {err:.3e} > {tol:.3e}"


# -------------------------------------------------------------------------------------------------
# small grids spanning several tiles with ragged tails, every lattice/collision/drive/storage
# -------------------------------------------------------------------------------------------------

CASES = [
    # id, Q, nx, ny, kind, lx, ly, drive, eq, coll, storage, steps, init_exp, tile
    ("q9-bgk-plate-f64", 9, 45, 37, L.LBM_GEOM_PLATE, 0, 0, L.LBM_DRIVE_WALL, 2, L.LBM_COLL_BGK, L.LBM_STORE_F64, 40,
     -17, None),
    ("q9-reg-beam-body-f64", 9, 45, 37, L.LBM_GEOM_BEAM, 9, 7, L.LBM_DRIVE_BODYFORCE, 2, L.LBM_COLL_REGULARIZED,
     L.LBM_STORE_F64, 40, -17, (64, 2)),
    ("q37-reg-h2-plate-f64", 37, 45, 50, L.LBM_GEOM_PLATE, 0, 0, L.LBM_DRIVE_WALL, 2,
     L.LBM_COLL_REGULARIZED, L.LBM_STORE_F64, 30, -17, None),
    ("q37-reg-h4-beam-body-f64", 37, 70, 41, L.LBM_GEOM_BEAM, 12, 9, L.LBM_DRIVE_BODYFORCE, 4,
     L.LBM_COLL_REGULARIZED, L.LBM_STORE_F64, 30, -17, (32, 4)),
    ("q37-bgk-h4-mask-wall-f64", 37, 67, 53, L.LBM_GEOM_MASK, 0, 0, L.LBM_DRIVE_WALL, 4, L.LBM_COLL_BGK,
     L.LBM_STORE_F64, 25, -17, (128, 2)),
    ("q37-bgk-h2-open-f64", 37, 37, 29, L.LBM_GEOM_NONE, 0, 0, L.LBM_DRIVE_WALL, 2, L.LBM_COLL_BGK,
     L.LBM_STORE_F64, 20, -17, None),
    ("q9-bgk-plate-f32", 9, 45, 37, L.LBM_GEOM_PLATE, 0, 0, L.LBM_DRIVE_WALL, 2, L.LBM_COLL_BGK, L.LBM_STORE_F32, 40,
     -17, None),
    ("q37-reg-h4-beam-body-f32", 37, 70, 41, L.LBM_GEOM_BEAM, 12, 9, L.LBM_DRIVE_BODYFORCE, 4,
     L.LBM_COLL_REGULARIZED, L.LBM_STORE_F32, 30, -17, None),
    ("q37-bgk-h4-mask-wall-f32", 37, 67, 53, L.LBM_GEOM_MASK, 0, 0, L.LBM_DRIVE_WALL, 4, L.LBM_COLL_BGK,
     L.LBM_STORE_F32, 25, -17, (64, 4)),
    # lab frame: the beam's walls move (Sec. 6), no body force
    ("q9-reg-beam-lab-f64", 9, 45, 37, L.LBM_GEOM_BEAM, 9, 7, L.LBM_DRIVE_WALL, 2, L.LBM_COLL_REGULARIZED,
     L.LBM_STORE_F64, 40, -17, None),
    ("q37-reg-h4-beam-lab-f64", 37, 70, 41, L.LBM_GEOM_BEAM, 12, 9, L.LBM_DRIVE_WALL, 4,
     L.LBM_COLL_REGULARIZED, L.LBM_STORE_F64, 30, -17, (32, 4)),
    ("q37-reg-h4-beam-lab-f32", 37, 70, 41, L.LBM_GEOM_BEAM, 12, 9, L.LBM_DRIVE_WALL, 4,
     L.LBM_COLL_REGULARIZED, L.LBM_STORE_F32, 30, -17, (64, 2)),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_parity_small(case):
    name, Q, nx, ny, kind, lx, ly, drive, eq, coll, st, steps, e, tile = case
    mask = I.random_mask(nx, ny, 3 if Q == 37 else 1, seed=7) if kind == L.LBM_GEOM_MASK else None
    tau, omega = 0.83, 0.05
    g_gpu, g_or, F_gpu, F_or, lab, g0 = run_both(Q, nx, ny, tau, omega, kind, steps, lx=lx, ly=ly, mask=mask,
                                                 drive=drive, u0=2e-3, eq_order=eq, collision=coll, storage=st,
                                                 init_exp=e, seed=11, tile=tile, n0_chunks=3)
    assert_state_close(Q, g_gpu, g_or, lab, st, steps, g0)
    assert_force_close(F_gpu, F_or, Q, lab, st, steps)


@pytest.mark.parametrize("st", [L.LBM_STORE_BF16, L.LBM_STORE_F16])
@pytest.mark.parametrize("coll", [L.LBM_COLL_REGULARIZED, L.LBM_COLL_BGK])
def test_parity_16bit_one_step(st, coll):
    """One step from a 16-bit-exact state: each output is the exact step rounded once to 16 bits."""
    Q, nx, ny = 37, 70, 41
    g_gpu, g_or, F_gpu, F_or, lab, g0 = run_both(Q, nx, ny, 0.9, 0.05, L.LBM_GEOM_BEAM, 1, lx=12, ly=9,
                                                 drive=L.LBM_DRIVE_BODYFORCE, u0=2e-3, eq_order=4, collision=coll,
                                                 storage=st, init_exp=-7, seed=5)
    assert_state_close(Q, g_gpu, g_or, lab, st, 1, g0, 2e-3 * stream_offset_magnitude(Q, 2e-3, 0.05, 1, 4))
    assert_force_close(F_gpu, F_or, Q, lab, st, 1)


@pytest.mark.parametrize("st", [L.LBM_STORE_BF16, L.LBM_STORE_F16])
def test_parity_16bit_one_step_lab_frame(st):
    """Moving-wall beam in 16-bit storage: no stream offset (the far fluid is at rest), so each
    output is the exact step rounded once, relative to its own magnitude."""
    Q, nx, ny = 37, 70, 41
    g_gpu, g_or, F_gpu, F_or, lab, g0 = run_both(Q, nx, ny, 0.9, 0.05, L.LBM_GEOM_BEAM, 1, lx=12, ly=9,
                                                 drive=L.LBM_DRIVE_WALL, u0=2e-3, eq_order=4, storage=st,
                                                 init_exp=-7, seed=6)
    assert_state_close(Q, g_gpu, g_or, lab, st, 1, g0)
    assert_force_close(F_gpu, F_or, Q, lab, st, 1)


def test_parity_plate_d2q9_fp64_full_config():
    """The D2Q9 plate workload itself (4 x 256, tau = 0.8, omega = 1/3, U0 = 1e-3, 20 periods) from rest."""
    w = I.plate_d2q9_fp64()
    steps = int(round(w.periods * 2 * math.pi / w.omega))
    g_gpu, g_or, F_gpu, F_or, lab, _ = run_both(w.lattice, w.nx, w.ny, w.tau, w.omega, w.geometry, steps,
                                                drive=w.drive, u0=w.u0, eq_order=w.eq_order, collision=w.collision,
                                                storage=w.storage)
    assert_state_close(9, g_gpu, g_or, lab, w.storage, steps)
    # the force history, stamped at t = n + 1/2, agrees to FP64 rounding
    scale = np.abs(F_or[:, 0]).max()
    assert np.abs(F_gpu[:, 0] - F_or[:, 0]).max() <= 1e-10 * scale
    assert np.abs(F_gpu[:, 1] - F_or[:, 1]).max() <= 1e-12 * np.abs(F_or[:, 1]).max()


@pytest.mark.parametrize("storage", [L.LBM_STORE_F32, L.LBM_STORE_F16])
def test_kernel_variants_and_tiles_do_not_change_results(storage):
    """Tile shape and kernel variant (plain or TMA-staged) compute the same step: the states agree
    to FP32 rounding (the compiler may contract the same source into different FMAs in different
    kernels, and with 16-bit storage two nearby FP32 values can round to neighbouring 16-bit
    values: one 16-bit ulp, two half-ulps, is allowed on top), the forces to the FP64 reduction order.  The grid has interior (staged)
    tiles."""
    Q, nx, ny = 37, 200, 90
    outs = []
    configs = [("tile", (32, 8)), ("tile", (64, 4)), ("tile", (128, 1)), ("tile", (32, 16)),
               ("variant", 1), ("variant", 2), ("variant", 3), ("variant", 4), ("variant", 10), ("variant", 11),
               ("variant", 12), ("variant", 13),
               ("variant", 18), ("variant", 23), ("variant", 24), ("variant", 25), ("variant", 26), ("variant", 27),
               ("variant", 28)]
    for kind, arg in configs:
        geom = L.make_geometry(kind=L.LBM_GEOM_BEAM, lx=24, ly=19, drive=L.LBM_DRIVE_BODYFORCE, u0=1e-3, eq_order=4,
                               storage=storage)
        h = L.lbm_create(Q, nx, ny, 0.9, 0.05, geom)
        if kind == "tile":
            L.lbm_set_tile(h, *arg)
        else:
            L.lbm_set_variant(h, arg)
            assert L.lbm_info(h)["variant"] == arg
        L.lbm_step(h, 15)
        outs.append((L.lbm_get_state(h), L.lbm_force_history(h)))
        L.lbm_destroy(h)
    h_ref = scaled(Q, outs[0][0])
    scale = np.abs(h_ref).max()
    offset = (1e-3 * stream_offset_magnitude(Q, 1e-3, 0.05, 15, 4))[:, None, None] if storage in ROUND16 else 0.0
    for (kind, arg), (g, F) in zip(configs[1:], outs[1:]):
        h = scaled(Q, g)
        err = np.abs(h - h_ref)
        bound = EPS_STEP[storage] * scale + 2.0 * ROUND16.get(storage, 0.0) * (np.maximum(np.abs(h_ref), np.abs(h))
                                                                               + offset)
        assert (err <= bound).all(), (kind, arg, err.max())
        Ftol = (EPS_STEP[storage] + ROUND16.get(storage, 0.0)) * (np.abs(outs[0][1]).max() + 1.0)
        assert np.abs(F - outs[0][1]).max() <= Ftol, (kind, arg)


@pytest.mark.parametrize("variant", [1, 2, 3, 4, 10, 11, 12, 13, 18, 23, 24, 25, 26, 27, 28])
def test_parity_staged_variants(variant):
    """The occupancy-floor (1, 2) and TMA-staged kernels against the oracle on a grid with interior
    tiles, FP32."""
    Q, nx, ny, steps = 37, 200, 90, 12
    geom = L.make_geometry(kind=L.LBM_GEOM_BEAM, lx=24, ly=19, drive=L.LBM_DRIVE_BODYFORCE, u0=2e-3, eq_order=4,
                           storage=L.LBM_STORE_F32)
    lab = orc.geometry_beam(nx, ny, 24, 19)
    _, w, _ = L.lbm_lattice_velocities(Q)
    h0 = I.random_scaled_state(Q, nx, ny, -17, 9)
    h0[:, lab != 0] = 0.0
    g0 = h0 * w[:, None, None]
    h = L.lbm_create(Q, nx, ny, 0.9, 0.05, geom)
    try:
        L.lbm_set_variant(h, variant)
        L.lbm_set_state(h, g0)
        L.lbm_step(h, steps)
        g, F = L.lbm_get_state(h), L.lbm_force_history(h)
    finally:
        L.lbm_destroy(h)
    f, F_or = orc.run(Q, lab, 0.9, 0.05, 2e-3, steps, eq_order=4, collision=orc.COLL_REG, drive=orc.DRIVE_BODY,
                      f=g_to_oracle_state(Q, g0), nthreads=orc.max_threads())
    assert_state_close(Q, g, oracle_state_to_g(Q, f), lab, L.LBM_STORE_F32, steps, g0)
    assert_force_close(F, F_or, Q, lab, L.LBM_STORE_F32, steps)


# The multi-row staged kernels in 16-bit storage (the batch runs 27) against the oracle on 393 x 90:
# staged interior tiles, an odd width (a ragged last tile on the plain path) and a 23-wide beam, so
# that interior tiles hold solid and boundary nodes.
STAGED16 = [18, 26, 27, 28]


@pytest.mark.parametrize("st", [L.LBM_STORE_BF16, L.LBM_STORE_F16])
@pytest.mark.parametrize("variant", STAGED16)
def test_parity_16bit_staged_variants_one_step(st, variant):
    """One step from a 16-bit-exact state, body-force frame (stream offset on): each output is the
    exact step rounded once to 16 bits."""
    Q, nx, ny = 37, 393, 90
    g_gpu, g_or, F_gpu, F_or, lab, g0 = run_both(Q, nx, ny, 0.9, 0.05, L.LBM_GEOM_BEAM, 1, lx=23, ly=19,
                                                 drive=L.LBM_DRIVE_BODYFORCE, u0=2e-3, eq_order=4, storage=st,
                                                 init_exp=-7, seed=21, variant=variant)
    assert_state_close(Q, g_gpu, g_or, lab, st, 1, g0, 2e-3 * stream_offset_magnitude(Q, 2e-3, 0.05, 1, 4))
    assert_force_close(F_gpu, F_or, Q, lab, st, 1)


@pytest.mark.parametrize("variant", STAGED16)
def test_parity_16bit_staged_variants_chained(variant):
    """Eleven chained FP16 steps (moving wall, lab frame; two launches, so consecutive grids chain),
    then the twelfth against one oracle step from the state the GPU reached: each output is that
    exact step rounded once to 16 bits."""
    Q, nx, ny, lx, ly, u0 = 37, 393, 90, 23, 19, 2e-3
    geom = L.make_geometry(kind=L.LBM_GEOM_BEAM, lx=lx, ly=ly, drive=L.LBM_DRIVE_WALL, u0=u0, eq_order=4,
                           storage=L.LBM_STORE_F16)
    _, wts, _ = L.lbm_lattice_velocities(Q)
    lab = orc.geometry_beam(nx, ny, lx, ly)
    h0 = I.random_scaled_state(Q, nx, ny, -9, seed=22)
    h0[:, lab != 0] = 0.0
    h = L.lbm_create(Q, nx, ny, 0.9, 0.05, geom)
    try:
        L.lbm_set_variant(h, variant)
        L.lbm_set_state(h, h0 * wts[:, None, None] * u0)
        L.lbm_step(h, 5)
        L.lbm_step(h, 6)
        g11 = L.lbm_get_state(h)
        L.lbm_step(h, 1)
        g12 = L.lbm_get_state(h)
        F = L.lbm_force_history(h)
    finally:
        L.lbm_destroy(h)
    f, F_or = orc.run(Q, lab, 0.9, 0.05, u0, 1, eq_order=4, collision=orc.COLL_REG, drive=orc.DRIVE_WALL,
                      f=g_to_oracle_state(Q, g11), n0=11, nthreads=orc.max_threads())
    assert_state_close(Q, g12, oracle_state_to_g(Q, f), lab, L.LBM_STORE_F16, 1, g11)
    assert_force_close(F[11:12], F_or, Q, lab, L.LBM_STORE_F16, 1)


def test_repeat_runs_are_bitwise_identical():
    Q = 37
    res = []
    for _ in range(2):
        geom = L.make_geometry(kind=L.LBM_GEOM_BEAM, lx=12, ly=9, drive=L.LBM_DRIVE_BODYFORCE, u0=1e-3, eq_order=4,
                               storage=L.LBM_STORE_F32)
        h = L.lbm_create(Q, 70, 41, 0.9, 0.05, geom)
        L.lbm_step(h, 20)
        res.append((L.lbm_get_state(h), L.lbm_force_history(h)))
        L.lbm_destroy(h)
    assert (res[0][0] == res[1][0]).all() and (res[0][1] == res[1][1]).all()


# -------------------------------------------------------------------------------------------------
# full-size workloads, in the launch configuration the benchmark times: one oracle step from the
# GPU's own state at step n, compared at every node with the GPU's step n + 1
# -------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("n,storage,to,variant", [(1024, L.LBM_STORE_F32, 0.01, None),
                                                  (1024, L.LBM_STORE_F32, 10.0, None),
                                                  (1024, L.LBM_STORE_F32, 1.0, 2),
                                                  (2048, L.LBM_STORE_F16, 1.0, None),
                                                  (2048, L.LBM_STORE_BF16, 0.1, None),
                                                  (1024, L.LBM_STORE_F16, 1.0, 27),
                                                  (1024, L.LBM_STORE_BF16, 10.0, 27)])
def test_full_size_one_step(n, storage, to, variant):
    """variant: the kernel the batch's streams mode runs (2 for FP32, 27 for 16-bit storage) on the
    largest instance of the 64-instance sweep; None: the default of lbm_create."""
    w = I.beam_d2q37_h4(to, n=n, storage=storage)
    tau, omega, _ = orc.params_from_tau_omega(37, to)
    geom = L.make_geometry(kind=w.geometry, lx=w.lx, ly=w.ly, drive=w.drive, u0=w.u0, eq_order=w.eq_order,
                           collision=w.collision, storage=storage)
    s = 1.0 if L.STORAGE_BYTES[storage] > 2 else w.u0
    _, wts, _ = L.lbm_lattice_velocities(37)
    lab = orc.geometry_beam(n, n, w.lx, w.ly)
    h0 = I.random_scaled_state(37, n, n, -17 if s == 1.0 else -7, seed=3)
    h0[:, lab != 0] = 0.0
    h = L.lbm_create(37, n, n, tau, omega, geom)
    try:
        if variant is not None:
            L.lbm_set_variant(h, variant)
        L.lbm_set_state(h, h0 * wts[:, None, None] * s)
        L.lbm_step(h, 7)                       # n0 = 7: the drive phase is not at zero
        g7 = L.lbm_get_state(h)
        L.lbm_step(h, 1)
        g8 = L.lbm_get_state(h)
        F = L.lbm_force_history(h)
    finally:
        L.lbm_destroy(h)
    f, F_or = orc.run(37, lab, tau, omega, w.u0, 1, eq_order=4, collision=w.collision, drive=w.drive,
                      f=g_to_oracle_state(37, g7), n0=7, nthreads=orc.max_threads())
    off = s * stream_offset_magnitude(37, w.u0, omega, 8, 4) if s != 1.0 else None
    assert_state_close(37, g8, oracle_state_to_g(37, f), lab, storage, 1, g7, off)
    assert_force_close(F[7:8], F_or, 37, lab, storage, 1)


def test_full_size_momentum_balance_fp32():
    """At 1024^2, FP32: P_fluid(n+1) - P_fluid(n) = M g(n + 1/2) - F_n holds to FP32 rounding.

    Each node's output momentum is rho * (1/rho) * (j + F/2) + F/2 in FP32, a few roundings of j,
    so the total momentum P carries a relative error of a few 2^-24 per step: the bound is
    4e-7 |P| (about 7 units of 2^-24) plus FP32 rounding of the force itself."""
    to = 1.0
    w = I.beam_d2q37_h4(to)
    tau, omega, _ = orc.params_from_tau_omega(37, to)
    geom = L.make_geometry(kind=w.geometry, lx=w.lx, ly=w.ly, drive=w.drive, u0=w.u0, eq_order=4,
                           collision=w.collision, storage=L.LBM_STORE_F32)
    c, _, _ = L.lbm_lattice_velocities(37)
    h = L.lbm_create(37, w.nx, w.ny, tau, omega, geom)
    try:
        L.lbm_step(h, 10)
        P = []
        for k in range(3):
            g = L.lbm_get_state(h)
            P.append((np.einsum("iyx,i->", g, c[:, 0].astype(float)), g.sum()))
            L.lbm_step(h, 1)
        F = L.lbm_force_history(h)
    finally:
        L.lbm_destroy(h)
    lab = orc.geometry_beam(w.nx, w.ny, w.lx, w.ly)
    M = float((lab == 0).sum())   # rho0 = 1 per fluid node (+ sum g, negligible at 1e-3 * 1e-... )
    for k in range(2):
        n = 10 + k
        gx = w.u0 * omega * math.cos(omega * (n + 0.5))
        lhs = P[k + 1][0] - P[k][0]
        rhs = (M + P[k][1]) * gx - F[n, 0]
        bound = 4e-7 * max(abs(P[k][0]), abs(P[k + 1][0])) + 1e-5 * abs(F[n, 0])
        assert abs(lhs - rhs) <= bound, (lhs, rhs, bound)


# -------------------------------------------------------------------------------------------------
# diffuse-scattering walls (Eq. 11)
# -------------------------------------------------------------------------------------------------

DS_CASES = [
    ("q37-reg-h4-beam-body-f64", 37, 70, 41, L.LBM_GEOM_BEAM, 12, 9, L.LBM_DRIVE_BODYFORCE, 4,
     L.LBM_COLL_REGULARIZED, L.LBM_STORE_F64, 25),
    ("q37-reg-h2-plate-wall-f64", 37, 45, 50, L.LBM_GEOM_PLATE, 0, 0, L.LBM_DRIVE_WALL, 2, L.LBM_COLL_REGULARIZED,
     L.LBM_STORE_F64, 25),
    ("q9-bgk-plate-wall-f64", 9, 45, 37, L.LBM_GEOM_PLATE, 0, 0, L.LBM_DRIVE_WALL, 2, L.LBM_COLL_BGK,
     L.LBM_STORE_F64, 30),
    ("q37-reg-h4-mask-wall-f32", 37, 67, 53, L.LBM_GEOM_MASK, 0, 0, L.LBM_DRIVE_WALL, 4, L.LBM_COLL_REGULARIZED,
     L.LBM_STORE_F32, 25),
    ("q37-bgk-h4-beam-body-f32", 37, 70, 41, L.LBM_GEOM_BEAM, 12, 9, L.LBM_DRIVE_BODYFORCE, 4, L.LBM_COLL_BGK,
     L.LBM_STORE_F32, 25),
]


@pytest.mark.parametrize("case", DS_CASES, ids=[c[0] for c in DS_CASES])
def test_parity_diffuse_walls(case):
    name, Q, nx, ny, kind, lx, ly, drive, eq, coll, st, steps = case
    mask = I.random_mask(nx, ny, 3 if Q == 37 else 1, seed=7) if kind == L.LBM_GEOM_MASK else None
    g_gpu, g_or, F_gpu, F_or, lab, g0 = run_both(Q, nx, ny, 0.83, 0.05, kind, steps, lx=lx, ly=ly, mask=mask,
                                                 drive=drive, u0=2e-3, eq_order=eq, collision=coll, storage=st,
                                                 init_exp=-17, seed=13, n0_chunks=2, wall=L.LBM_SCHEME_DIFFUSE)
    assert_state_close(Q, g_gpu, g_or, lab, st, steps, g0)
    assert_force_close(F_gpu, F_or, Q, lab, st, steps)


@pytest.mark.parametrize("st", [L.LBM_STORE_F16, L.LBM_STORE_BF16])
def test_parity_diffuse_16bit_one_step(st):
    Q, nx, ny = 37, 70, 41
    g_gpu, g_or, F_gpu, F_or, lab, g0 = run_both(Q, nx, ny, 0.9, 0.05, L.LBM_GEOM_BEAM, 1, lx=12, ly=9,
                                                 drive=L.LBM_DRIVE_BODYFORCE, u0=2e-3, eq_order=4,
                                                 collision=L.LBM_COLL_REGULARIZED, storage=st, init_exp=-7, seed=5,
                                                 wall=L.LBM_SCHEME_DIFFUSE)
    assert_state_close(Q, g_gpu, g_or, lab, st, 1, g0, 2e-3 * stream_offset_magnitude(Q, 2e-3, 0.05, 1, 4))
    assert_force_close(F_gpu, F_or, Q, lab, st, 1)


def test_diffuse_rejected_by_staged_variants():
    geom = L.make_geometry(kind=L.LBM_GEOM_BEAM, lx=12, ly=9, drive=L.LBM_DRIVE_BODYFORCE, u0=1e-3, eq_order=4,
                           storage=L.LBM_STORE_F32, wall_scheme=L.LBM_SCHEME_DIFFUSE)
    h = L.lbm_create(37, 200, 90, 0.9, 0.05, geom)
    try:
        with pytest.raises(L.LbmError):
            L.lbm_set_variant(h, 11)
        L.lbm_step(h, 3)
        L.lbm_synchronize(h)
    finally:
        L.lbm_destroy(h)
