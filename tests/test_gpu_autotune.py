"""GPU tests of the kernel autotuner: lbm_tune times every built candidate on a clone (the
simulation itself is not advanced), lbm_autotune applies the fastest, and the JSON cache applies a
stored choice without timing again."""
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
