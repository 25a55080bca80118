"""Host-side checks of the C ABI (no GPU): the library loads, exports every declared symbol, its
tables and parameter mapping agree with the oracle's, and bad arguments are rejected."""
import ctypes
import math

import numpy as np
import pytest

import oracle as orc
from paper_0904_4504_gb300 import builder as B
from paper_0904_4504_gb300 import lbm as L


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def test_library_exports_every_declared_symbol():
    names = L.header_functions()
    assert len(names) >= 16
    lib = ctypes.CDLL(str(B.LIB))
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


@pytest.mark.parametrize("Q", [9, 37])
def test_velocity_table_matches_oracle(Q):
    c, w, th = L.lbm_lattice_velocities(Q)
    co, wo, tho = orc.lattice(Q)
    assert th == pytest.approx(tho, rel=0, abs=1e-16)
    lib_set = sorted((int(a), int(b), float(x)) for (a, b), x in zip(c, w))
    or_set = sorted((int(a), int(b), float(x)) for (a, b), x in zip(co, wo))
    assert lib_set == or_set
    # pair order: 0 rest, (1+2k, 2+2k) = (+c, -c)
    assert tuple(c[0]) == (0, 0)
    for k in range((Q - 1) // 2):
        assert (c[1 + 2 * k] == -c[2 + 2 * k]).all() and w[1 + 2 * k] == w[2 + 2 * k]


@pytest.mark.parametrize("Q", [9, 37])
@pytest.mark.parametrize("to", [1e-3, 0.01, 0.1, 1.0, 10.0, 1e3])
def test_params_mapping_matches_oracle(Q, to):
    assert L.lbm_params_from_tau_omega(Q, to) == pytest.approx(orc.params_from_tau_omega(Q, to), rel=1e-15)


def test_params_mapping_rejects_bad_input():
    with pytest.raises(L.LbmError) as e:
        L.lbm_params_from_tau_omega(37, 0.0)
    assert e.value.code == L.LBM_EINVAL


@pytest.mark.parametrize("args,msg", [
    (dict(lattice=37, nx=64, ny=64, tau=0.5, omega=0.1), "tau"),
    (dict(lattice=37, nx=64, ny=64, tau=0.8, omega=0.0), "omega"),
    (dict(lattice=37, nx=6, ny=64, tau=0.8, omega=0.1), "grid"),
    (dict(lattice=11, nx=64, ny=64, tau=0.8, omega=0.1), "lattice"),
    (dict(lattice=37, nx=64, ny=64, tau=0.8, omega=0.1, u0=0.2), "u0"),
    (dict(lattice=9, nx=64, ny=64, tau=0.8, omega=0.1, eq_order=4), "D2Q9"),
    (dict(lattice=37, nx=64, ny=64, tau=0.8, omega=0.1, storage=7), "storage"),
    (dict(lattice=37, nx=64, ny=64, tau=0.8, omega=0.1, storage=L.LBM_STORE_F16, u0=0.0), "16-bit"),
])
def test_create_rejects_bad_arguments(args, msg):
    a = dict(args)
    geom = L.make_geometry(kind=L.LBM_GEOM_NONE, u0=a.pop("u0", 1e-3), eq_order=a.pop("eq_order", 2),
                           storage=a.pop("storage", L.LBM_STORE_F32))
    with pytest.raises(L.LbmError) as e:
        L.lbm_create(a["lattice"], a["nx"], a["ny"], a["tau"], a["omega"], geom)
    assert e.value.code == L.LBM_EINVAL
    assert msg in L.lbm_last_error()


def test_null_handles_are_rejected():
    assert L.lib().lbm_step(None, 1) == L.LBM_EINVAL
    assert L.lib().lbm_synchronize(None) == L.LBM_EINVAL
    L.lib().lbm_destroy(None)  # NULL-safe


def test_batch_footprint_counts_both_population_buffers():
    d = L.make_instance(37, 1024, 1024, 0.9, 0.05, 3840, kind=L.LBM_GEOM_BEAM, lx=32, ly=32,
                        storage=L.LBM_STORE_F32)
    n = L.lbm_batch_footprint(d)
    assert 2 * 37 * 1024 * 1024 * 4 < n < 2 * 37 * 1024 * 1024 * 4 + 40 * 1024 * 1024


def test_batch_footprint_of_the_in_place_layout_holds_one_buffer():
    kw = dict(kind=L.LBM_GEOM_BEAM, lx=32, ly=32, storage=L.LBM_STORE_F16)
    ab = L.lbm_batch_footprint(L.make_instance(37, 2048, 2048, 0.9, 0.05, 3840, **kw))
    aa = L.lbm_batch_footprint(L.make_instance(37, 2048, 2048, 0.9, 0.05, 3840, layout=L.LBM_LAYOUT_AA, **kw))
    assert ab - aa == 37 * 2048 * 2048 * 2


def test_create_rejects_bad_layout_and_diffuse_in_place():
    for kw in (dict(layout=7), dict(layout=L.LBM_LAYOUT_AA, wall_scheme=L.LBM_SCHEME_DIFFUSE)):
        geom = L.make_geometry(kind=L.LBM_GEOM_NONE, u0=1e-3, **kw)
        with pytest.raises(L.LbmError) as e:
            L.lbm_create(37, 64, 64, 0.8, 0.1, geom)
        assert e.value.code == L.LBM_EINVAL


def test_batch_create_rejects_bad_arguments():
    with pytest.raises(L.LbmError) as e:
        L.lbm_batch_create(11, L.LBM_STORE_F32, L.LBM_COLL_REGULARIZED)
    assert e.value.code == L.LBM_EINVAL
    assert L.lib().lbm_batch_run(None, 1) == L.LBM_EINVAL
    L.lib().lbm_batch_destroy(None)


def test_create_rejects_bad_wall_scheme():
    geom = L.make_geometry(kind=L.LBM_GEOM_NONE, u0=1e-3, wall_scheme=5)
    with pytest.raises(L.LbmError) as e:
        L.lbm_create(37, 64, 64, 0.8, 0.1, geom)
    assert e.value.code == L.LBM_EINVAL and "wall scheme" in L.lbm_last_error()


def _links_brute(Q, lab):
    """Eq. 12's blocked links as lbm_create applies them (node-return bounce-back), written out per
    node and direction: link i of fluid node x is blocked when x - c_i, or a lattice node strictly
    between, is solid; the first solid met walking back from x decides body (label 1) or wall."""
    c, _, _ = L.lbm_lattice_velocities(Q)
    ny, nx = lab.shape
    cls = np.zeros((ny, nx), dtype=np.uint8)
    body = np.zeros((ny, nx), dtype=np.uint64)
    wall = np.zeros((ny, nx), dtype=np.uint64)
    for y in range(ny):
        for x in range(nx):
            if lab[y, x]:
                cls[y, x] = 1
                continue
            b = w = 0
            for i in range(1, Q):
                cx, cy = int(c[i, 0]), int(c[i, 1])
                g = math.gcd(abs(cx), abs(cy))
                for k in range(1, g + 1):
                    l = lab[(y - k * cy // g) % ny, (x - k * cx // g) % nx]
                    if l:
                        if l == L.LBM_BODY:
                            b |= 1 << i
                        else:
                            w |= 1 << i
                        break
            body[y, x], wall[y, x] = b, w
            if b or w:
                cls[y, x] = 2
    return cls, body, wall


@pytest.mark.parametrize("case", ["beam37", "plate37", "mask37", "mask9", "small37", "wide37"])
def test_geometry_links_match_the_wall_rule(case):
    """The host geometry of lbm_create (classes and link masks, computed only near the solids)
    against the rule written out node by node, on grids whose solids reach the periodic edges."""
    rng = np.random.default_rng(7)
    if case == "beam37":
        Q, nx, ny, geom = 37, 45, 31, L.make_geometry(kind=L.LBM_GEOM_BEAM, lx=9, ly=5)
    elif case == "plate37":
        Q, nx, ny, geom = 37, 12, 23, L.make_geometry(kind=L.LBM_GEOM_PLATE)
    elif case in ("mask37", "mask9"):
        Q, nx, ny = (37, 41, 29) if case == "mask37" else (9, 33, 19)
        m = np.where(rng.random((ny, nx)) < 0.04, rng.integers(1, 3, (ny, nx)), 0).astype(np.uint8)
        geom = L.make_geometry(kind=L.LBM_GEOM_MASK, mask=m)
    elif case == "small37":
        m = np.zeros((7, 7), dtype=np.uint8)
        m[3, 3] = L.LBM_BODY
        Q, nx, ny, geom = 37, 7, 7, L.make_geometry(kind=L.LBM_GEOM_MASK, mask=m)
    else:
        m = np.zeros((7, 60), dtype=np.uint8)
        m[0, 10:14] = L.LBM_WALL
        m[6, 50] = L.LBM_BODY
        Q, nx, ny, geom = 37, 60, 7, L.make_geometry(kind=L.LBM_GEOM_MASK, mask=m)
    cls, body, wall, nf, nb = L.lbm_geometry_links(Q, nx, ny, geom)
    if case == "beam37":
        lab = orc.geometry_beam(nx, ny, 9, 5)
    elif case == "plate37":
        lab = orc.geometry_plate(Q, nx, ny)
    else:
        lab = np.asarray(geom._mask_ref)
    c_ref, b_ref, w_ref = _links_brute(Q, lab)
    assert (cls == c_ref).all()
    assert (body == b_ref).all() and (wall == w_ref).all()
    assert nf == int((lab == 0).sum()) and nb == int((c_ref == 2).sum())


def test_geometry_links_rejects_bad_input():
    geom = L.make_geometry(kind=L.LBM_GEOM_BEAM, lx=4, ly=4)
    with pytest.raises(L.LbmError):
        L.lbm_geometry_links(37, 6, 20, geom)       # below 2R + 1 nodes per side
    with pytest.raises(L.LbmError):
        L.lbm_geometry_links(11, 20, 20, geom)      # no such lattice
