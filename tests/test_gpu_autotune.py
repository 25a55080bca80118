"""GPU tests of the kernel autotuner: lbm_tune times every built candidate on a clone (the
simulation itself is not advanced), lbm_autotune applies the fastest, and the JSON cache applies a
stored choice without timing again; for batches, lbm_batch_tune times the candidates on clones of
the instance mix in the batch's mode, and a batch set up from the cache computes its instances
exactly as the single-instance kernel of the chosen variant does."""
import pytest

from paper_0904_4504_gb300 import autotune as A
from paper_0904_4504_gb300 import lbm as L

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def _sim(storage):
    geom = L.make_geometry(kind=L.LBM_GEOM_BEAM, lx=32, ly=32, drive=L.LBM_DRIVE_BODYFORCE, u0=1e-3, eq_order=4,
                           storage=storage)
    return L.lbm_create(37, 512, 384, 0.9, 0.05, geom)


@pytest.mark.parametrize("storage", [L.LBM_STORE_F32, L.LBM_STORE_F16])
def test_tune_times_candidates_without_advancing(storage):
    h = _sim(storage)
    try:
        L.lbm_step(h, 3)
        before = L.lbm_get_state(h)
        table = L.lbm_tune(h, 5)
        assert L.lbm_info(h)["steps_done"] == 3
        assert (L.lbm_get_state(h) == before).all()
        variants = {e["variant"] for e in table}
        assert 0 in variants and {10, 11, 12} <= variants
        assert all(e["us_per_step"] > 0 for e in table)
        best = L.lbm_autotune(h, 5)
        info = L.lbm_info(h)
        assert info["variant"] == best["variant"]
        assert (info["block_x"], info["block_y"]) == (best["block_x"], best["block_y"])
        L.lbm_step(h, 2)
        L.lbm_synchronize(h)
    finally:
        L.lbm_destroy(h)


def test_json_cache_reuses_choice(tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    h = _sim(L.LBM_STORE_F16)
    try:
        first = A.tune(h, path, steps=3)
    finally:
        L.lbm_destroy(h)
    assert path.exists()
    calls = []
    monkeypatch.setattr(L, "lbm_tune", lambda *a, **k: calls.append(1) or [])
    h = _sim(L.LBM_STORE_F16)
    try:
        second = A.tune(h, path)
        assert second == first and not calls
        assert L.lbm_info(h)["variant"] == first["variant"]
    finally:
        L.lbm_destroy(h)


def _descs(Q, storage, n=4):
    out = []
    for k in range(n):
        side = 160 + 48 * k
        out.append(L.make_instance(Q, side, side - 16, 0.8 + 0.2 * k, 0.05, 12, kind=L.LBM_GEOM_BEAM, lx=16,
                                   ly=12 + 4 * k, drive=L.LBM_DRIVE_BODYFORCE, u0=1e-3,
                                   eq_order=4 if Q == 37 else 2, collision=L.LBM_COLL_REGULARIZED, storage=storage))
    return out


def _standalone(d, variant):
    h = L.lbm_create(d.lattice, d.nx, d.ny, d.tau, d.omega, d.geom)
    try:
        if variant:
            L.lbm_set_variant(h, variant)
        else:
            L.lbm_set_tile(h, 32, 4)
        L.lbm_step(h, d.nsteps)
        return L.lbm_get_state(h), L.lbm_force_history(h)
    finally:
        L.lbm_destroy(h)


@pytest.mark.parametrize("Q,storage", [(37, L.LBM_STORE_F16), (9, L.LBM_STORE_F16), (37, L.LBM_STORE_F32)])
@pytest.mark.parametrize("mode", [L.LBM_BATCH_STREAMS, L.LBM_BATCH_PERSISTENT], ids=["streams", "persistent"])
def test_batch_uses_cached_choice_bitwise(tmp_path, monkeypatch, mode, Q, storage):
    path = tmp_path / "tune.json"
    descs = _descs(Q, storage)
    b = L.lbm_batch_create(Q, storage, L.LBM_COLL_REGULARIZED)
    try:
        L.lbm_batch_set_mode(b, mode)
        first = A.tune_batch(b, descs, path, steps=4)
    finally:
        L.lbm_batch_destroy(b)
    assert path.exists() and first["us_per_step"] > 0
    calls = []
    monkeypatch.setattr(L, "lbm_batch_tune", lambda *a, **k: calls.append(1) or [])
    b = L.lbm_batch_create(Q, storage, L.LBM_COLL_REGULARIZED)
    try:
        L.lbm_batch_set_mode(b, mode)
        second = A.tune_batch(b, descs, path)
        assert second == first and not calls
        slots = [L.lbm_batch_add(b, d) for d in descs]
        L.lbm_batch_run(b, 5)
        L.lbm_batch_run(b, 7)
        L.lbm_batch_synchronize(b)
        for d, sl in zip(descs, slots):
            sim = L.lbm_batch_instance(b, sl)
            v = L.lbm_info(sim)["variant"]
            if mode == L.LBM_BATCH_STREAMS:
                assert v == first["variant"]
            g, F = L.lbm_get_state(sim), L.lbm_force_history(sim)
            g_a, F_a = _standalone(d, v)
            assert (g == g_a).all() and (F == F_a).all()
    finally:
        L.lbm_batch_destroy(b)

