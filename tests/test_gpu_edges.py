"""Degenerate cases against the FP64 oracle: the smallest grids the lattice reach allows (every
pull wraps around the periodic box), a plate box with a single fluid row, no drive at all, a single
fluid node closed in by the body, a box with no fluid, and relaxation times at both ends
(tau -> 1/2 and tau -> infinity, the collisionless limit)."""
import numpy as np
import pytest

import oracle as orc
from paper_0904_4504_gb300 import lbm as L

from test_gpu_parity import assert_force_close, assert_state_close, run_both

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

REG, BGK = L.LBM_COLL_REGULARIZED, L.LBM_COLL_BGK
F64, F32 = L.LBM_STORE_F64, L.LBM_STORE_F32


@pytest.mark.parametrize("Q,n,eq,coll", [(37, 7, 4, REG), (37, 7, 2, BGK), (9, 3, 2, REG), (9, 3, 2, BGK)])
@pytest.mark.parametrize("layout", [L.LBM_LAYOUT_AB, L.LBM_LAYOUT_AA])
def test_smallest_periodic_box(Q, n, eq, coll, layout):
    """n = 2R + 1 nodes per side: links of length 3 (D2Q37) reach past the whole box and wrap."""
    g_gpu, g_or, F_gpu, F_or, lab, g0 = run_both(Q, n, n, 0.8, 0.05, L.LBM_GEOM_NONE, 12, u0=1e-3, eq_order=eq,
                                                 collision=coll, storage=F64, init_exp=-17, seed=3, n0_chunks=3,
                                                 layout=layout)
    assert_state_close(Q, g_gpu, g_or, lab, F64, 12, g0)


@pytest.mark.parametrize("Q", [37, 9])
def test_plate_with_one_fluid_row(Q):
    """ny = 2R + 1: R rows of plate, R rows of static wall and one fluid row between them."""
    R = 3 if Q == 37 else 1
    g_gpu, g_or, F_gpu, F_or, lab, g0 = run_both(Q, 40, 2 * R + 1, 0.9, 0.05, L.LBM_GEOM_PLATE, 20, u0=2e-3,
                                                 eq_order=2, collision=REG, storage=F64, init_exp=-17, seed=4)
    assert (lab == 0).sum() == 40
    assert_state_close(Q, g_gpu, g_or, lab, F64, 20, g0)
    assert_force_close(F_gpu, F_or, Q, lab, F64, 20)


@pytest.mark.parametrize("drive", [L.LBM_DRIVE_WALL, L.LBM_DRIVE_BODYFORCE])
@pytest.mark.parametrize("st", [F64, F32])
def test_no_drive_keeps_the_rest_state_exactly(drive, st):
    """u0 = 0: every stored deviation stays exactly zero and the force is the geometry-only part."""
    geom = L.make_geometry(kind=L.LBM_GEOM_BEAM, lx=12, ly=9, drive=drive, u0=0.0, eq_order=4, storage=st)
    h = L.lbm_create(37, 70, 41, 0.9, 0.05, geom)
    try:
        L.lbm_step(h, 50)
        g = L.lbm_get_state(h)
        F = L.lbm_force_history(h)
    finally:
        L.lbm_destroy(h)
    assert not g.any()
    assert (F == F[0]).all()
    _, F_or = orc.run(37, orc.geometry_beam(70, 41, 12, 9), 0.9, 0.05, 0.0, 3, eq_order=4, drive=drive)
    assert np.abs(F[:3] - F_or).max() < 1e-12


@pytest.mark.parametrize("drive", [L.LBM_DRIVE_WALL, L.LBM_DRIVE_BODYFORCE])
def test_single_fluid_node_inside_the_body(drive):
    """Every link of the only fluid node is blocked: all of its populations come back each step."""
    nx, ny = 40, 33
    mask = np.ones((ny, nx), dtype=np.uint8)
    mask[16, 20] = 0
    g_gpu, g_or, F_gpu, F_or, lab, g0 = run_both(37, nx, ny, 0.9, 0.05, L.LBM_GEOM_MASK, 16, mask=mask, drive=drive,
                                                 u0=2e-3, eq_order=4, collision=REG, storage=F64, init_exp=-17,
                                                 seed=6)
    assert_state_close(37, g_gpu, g_or, lab, F64, 16, g0)
    assert_force_close(F_gpu, F_or, 37, lab, F64, 16)


def test_box_without_fluid():
    mask = np.ones((30, 40), dtype=np.uint8)
    mask[:10] = 2
    geom = L.make_geometry(kind=L.LBM_GEOM_MASK, mask=mask, u0=1e-3, storage=F32)
    h = L.lbm_create(37, 40, 30, 0.9, 0.05, geom)
    try:
        assert L.lbm_info(h)["n_fluid"] == 0
        L.lbm_step(h, 5)
        assert not L.lbm_get_state(h).any()
        assert not L.lbm_force_history(h).any()
    finally:
        L.lbm_destroy(h)
    _, F_or = orc.run(37, mask, 0.9, 0.05, 1e-3, 5)
    assert not F_or.any()


@pytest.mark.parametrize("tau", [0.5 + 1e-6, 1e6])
@pytest.mark.parametrize("st", [F64, F32])
def test_relaxation_time_extremes(tau, st):
    """tau -> 1/2 (the collision reflects the non-equilibrium part) and tau -> infinity (no
    collisions: free streaming and wall reflections only)."""
    g_gpu, g_or, F_gpu, F_or, lab, g0 = run_both(37, 70, 41, tau, 0.05, L.LBM_GEOM_BEAM, 10, lx=12, ly=9,
                                                 drive=L.LBM_DRIVE_BODYFORCE, u0=2e-3, eq_order=4, collision=REG,
                                                 storage=st, init_exp=-17, seed=8)
    assert_state_close(37, g_gpu, g_or, lab, st, 10, g0)
    assert_force_close(F_gpu, F_or, 37, lab, st, 10)
