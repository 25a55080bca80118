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
