"""GPU parity of the D2Q9 kernels with 16-bit storage (BF16, FP16) against the FP64 oracle.

The served mixed-precision stream runs D2Q9 instances in FP16 (plates and beams), so every D2Q9
kernel built for 16-bit storage is checked here: the plain kernel (variant 0), the staged kernel
(variant 10, TMA boxes on 32 x 4 tiles), the paired kernel (variant 20, two neighbouring nodes
per thread on 64 x 4 tiles) and the vector kernel (variant 30, four neighbouring nodes per thread
with 8-byte loads and stores on 128 x 4 tiles).  Grids are 200 x 90 / 203 x 61: interior (staged)
tiles, tiles on the periodic edges (plain loads), warps whose lanes meet the periodic seam, and a
ragged last tile (203 = 4 x 50 + 3: the per-node path of the vector kernel).

Bound (see test_gpu_parity.py): one step from a 16-bit-exact state must give the exact step
rounded once to the storage type, i.e. within 2^-8 (BF16) or 2^-11 (FP16) of each value (relative
to |h| plus the stream offset |H| when the body-frame run stores h - H), plus the FP32 part.
Chained runs: 11 steps on the GPU, then the 12th compared with one oracle step from the state the
GPU reached (the same bound), so that consecutive launches and the stream offset's step-to-step
update are exercised.
"""
import numpy as np
import pytest

import oracle as orc
from paper_0904_4504_gb300 import inputs as I
from paper_0904_4504_gb300 import lbm as L

from harness import g_to_oracle_state, oracle_labels, oracle_state_to_g, stream_offset_magnitude
from test_gpu_parity import assert_force_close, assert_state_close, run_both

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ST16 = [L.LBM_STORE_BF16, L.LBM_STORE_F16]
VARIANTS = [0, 10, 20, 30]
# (geometry, drive): the beam in the body frame (stream offset on) and the plate with its moving
# wall (the D2Q9 plate workload), and a lab-frame beam
GEOMS = [(L.LBM_GEOM_BEAM, L.LBM_DRIVE_BODYFORCE), (L.LBM_GEOM_PLATE, L.LBM_DRIVE_WALL),
         (L.LBM_GEOM_BEAM, L.LBM_DRIVE_WALL)]
U0, TAU, OMEGA = 2e-3, 0.9, 0.05


def _offset(drive, n):
    return U0 * stream_offset_magnitude(9, U0, OMEGA, n, 2) if drive == L.LBM_DRIVE_BODYFORCE else None


@pytest.mark.parametrize("geom", GEOMS, ids=["beam-body", "plate-wall", "beam-lab"])
@pytest.mark.parametrize("coll", [L.LBM_COLL_BGK, L.LBM_COLL_REGULARIZED], ids=["bgk", "reg"])
@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("st", ST16, ids=["bf16", "f16"])
def test_q9_16bit_one_step(st, variant, coll, geom):
    kind, drive = geom
    nx, ny = 200, 90
    g_gpu, g_or, F_gpu, F_or, lab, g0 = run_both(9, nx, ny, TAU, OMEGA, kind, 1, lx=23, ly=17, drive=drive, u0=U0,
                                                 eq_order=2, collision=coll, storage=st, init_exp=-7, seed=41,
                                                 variant=variant)
    assert_state_close(9, g_gpu, g_or, lab, st, 1, g0, _offset(drive, 1))
    assert_force_close(F_gpu, F_or, 9, lab, st, 1)


@pytest.mark.parametrize("geom", GEOMS[:2], ids=["beam-body", "plate-wall"])
@pytest.mark.parametrize("coll", [L.LBM_COLL_BGK, L.LBM_COLL_REGULARIZED], ids=["bgk", "reg"])
@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("st", ST16, ids=["bf16", "f16"])
def test_q9_16bit_chained(st, variant, coll, geom):
    kind, drive = geom
    Q, nx, ny, lx, ly = 9, 203, 61, 23, 17
    g = L.make_geometry(kind=kind, lx=lx, ly=ly, drive=drive, u0=U0, eq_order=2, collision=coll, storage=st)
    _, wts, _ = L.lbm_lattice_velocities(Q)
    lab = oracle_labels(kind, Q, nx, ny, lx, ly)
    h0 = I.random_scaled_state(Q, nx, ny, -9, seed=42)
    h0[:, lab != 0] = 0.0
    h = L.lbm_create(Q, nx, ny, TAU, OMEGA, g)
    try:
        L.lbm_set_variant(h, variant)
        assert L.lbm_info(h)["variant"] == variant
        L.lbm_set_state(h, h0 * wts[:, None, None] * U0)
        L.lbm_step(h, 5)
        L.lbm_step(h, 6)
        g11 = L.lbm_get_state(h)
        L.lbm_step(h, 1)
        g12 = L.lbm_get_state(h)
        F = L.lbm_force_history(h)
    finally:
        L.lbm_destroy(h)
    f, F_or = orc.run(Q, lab, TAU, OMEGA, U0, 1, eq_order=2, collision=coll, drive=drive,
                      f=g_to_oracle_state(Q, g11), n0=11, nthreads=orc.max_threads())
    assert_state_close(Q, g12, oracle_state_to_g(Q, f), lab, st, 1, g11, _offset(drive, 12))
    assert_force_close(F[11:12], F_or, Q, lab, st, 1)


@pytest.mark.parametrize("geom", GEOMS[:2], ids=["beam-body", "plate-wall"])
@pytest.mark.parametrize("st", ST16, ids=["bf16", "f16"])
def test_q9_16bit_diffuse_walls_one_step(st, geom):
    """Diffuse-scattering walls (Eq. 11) run the plain kernel only."""
    kind, drive = geom
    g_gpu, g_or, F_gpu, F_or, lab, g0 = run_both(9, 120, 64, TAU, OMEGA, kind, 1, lx=19, ly=11, drive=drive, u0=U0,
                                                 eq_order=2, collision=L.LBM_COLL_REGULARIZED, storage=st,
                                                 init_exp=-7, seed=43, wall=L.LBM_SCHEME_DIFFUSE)
    assert_state_close(9, g_gpu, g_or, lab, st, 1, g0, _offset(drive, 1))
    assert_force_close(F_gpu, F_or, 9, lab, st, 1)


@pytest.mark.parametrize("variant", VARIANTS)
def test_q9_16bit_full_size_one_step(variant):
    """The largest D2Q9 request shape of the served stream (a 2048^2 plate, regularized, FP16) in
    each kernel: one oracle step from the GPU's own state at step 7, compared at every node."""
    Q, n, st = 9, 2048, L.LBM_STORE_F16
    lab = orc.geometry_plate(Q, n, n)
    g = L.make_geometry(kind=L.LBM_GEOM_PLATE, drive=L.LBM_DRIVE_WALL, u0=1e-3, eq_order=2,
                        collision=L.LBM_COLL_REGULARIZED, storage=st)
    _, wts, _ = L.lbm_lattice_velocities(Q)
    tau, omega, _ = orc.params_from_tau_omega(Q, 0.3)
    h0 = I.random_scaled_state(Q, n, n, -7, seed=44)
    h0[:, lab != 0] = 0.0
    h = L.lbm_create(Q, n, n, tau, omega, g)
    try:
        L.lbm_set_variant(h, variant)
        L.lbm_set_state(h, h0 * wts[:, None, None] * 1e-3)
        L.lbm_step(h, 7)
        g7 = L.lbm_get_state(h)
        L.lbm_step(h, 1)
        g8 = L.lbm_get_state(h)
        F = L.lbm_force_history(h)
    finally:
        L.lbm_destroy(h)
    f, F_or = orc.run(Q, lab, tau, omega, 1e-3, 1, eq_order=2, collision=orc.COLL_REG, drive=orc.DRIVE_WALL,
                      f=g_to_oracle_state(Q, g7), n0=7, nthreads=orc.max_threads())
    assert_state_close(Q, g8, oracle_state_to_g(Q, f), lab, st, 1, g7)
    assert_force_close(F[7:8], F_or, Q, lab, st, 1)
