"""Kernel choice with a JSON cache: time the step-kernel candidates once per problem class with
lbm_tune (one simulation: lattice, storage type, collision, equilibrium order, grid) or lbm_batch_tune
(a batch: lattice, storage type, collision, batch mode, and the size of its instance mix), keep the
result in a JSON file, and apply the cached choice to later simulations or batches of the class."""
from __future__ import annotations

import json
import os
from pathlib import Path

from . import lbm as L

DEFAULT_CACHE = Path(os.environ.get("XDG_CACHE_HOME", Path.home() / ".cache")) / "lbm_gb300_tune.json"


def problem_key(sim: int) -> str:
    i = L.lbm_info(sim)
    return f"Q{i['lattice']}-st{i['storage']}-coll{i['collision']}-eq{i['eq_order']}-{i['nx']}x{i['ny']}"


def load(path=DEFAULT_CACHE) -> dict:
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def apply(sim: int, choice: dict) -> None:
    if choice["variant"]:
        L.lbm_set_variant(sim, choice["variant"])
    else:
        L.lbm_set_tile(sim, choice["block_x"], choice["block_y"])


def tune(sim: int, path=DEFAULT_CACHE, steps: int = 20, refresh: bool = False) -> dict:
    """Apply the cached kernel choice for this simulation's class, timing the candidates first if
    the class is not cached yet (or refresh is set).  Returns the choice."""
    cache = load(path)
    key = problem_key(sim)
    if refresh or key not in cache:
        table = L.lbm_tune(sim, steps)
        best = min(table, key=lambda e: e["us_per_step"])
        cache[key] = {"best": best, "candidates": table}
        Path(path).parent.mkdir(parents=True, exist_ok=True)
        tmp = Path(str(path) + f".{os.getpid()}")
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1)
        os.replace(tmp, path)
    choice = cache[key]["best"]
    apply(sim, choice)
    return choice


def batch_key(batch: int, descs) -> str:
    """Class of a batch: its lattice, storage, collision and mode, the number of instances (rounded
    up to a power of two) and their total node count (to a power of two): the kernel that wins
    depends on how many instances run concurrently and how large they are."""
    i = L.lbm_batch_info(batch)
    nodes = sum(d.nx * d.ny for d in descs)
    inst = 1 << max(0, (len(descs) - 1).bit_length())
    return (f"batch-Q{i['lattice']}-st{i['storage']}-coll{i['collision']}-mode{i['mode']}-inst{inst}-"
            f"nodes2^{max(0, nodes - 1).bit_length()}")


def tune_batch(batch: int, descs, path=DEFAULT_CACHE, steps: int = 10, refresh: bool = False) -> dict:
    """Set the cached kernel choice of this batch's class on the (still empty) batch, timing the
    candidates on clones of `descs` first if the class is not cached yet (or refresh is set).
    Returns the choice ({variant, segment, us_per_step})."""
    cache = load(path)
    key = batch_key(batch, descs)
    if refresh or key not in cache:
        table = L.lbm_batch_tune(batch, descs, steps)
        if not table:
            raise RuntimeError("no batch kernel candidate could be timed")
        best = min(table, key=lambda e: e["us_per_step"])
        cache[key] = {"best": best, "candidates": table}
        Path(path).parent.mkdir(parents=True, exist_ok=True)
        tmp = Path(str(path) + f".{os.getpid()}")
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1)
        os.replace(tmp, path)
    choice = cache[key]["best"]
    L.lbm_batch_set_variant(batch, choice["variant"])
    if L.lbm_batch_info(batch)["mode"] == L.LBM_BATCH_PERSISTENT:
        L.lbm_batch_set_segment(batch, choice["segment"])
    return choice


def tune_server(server: int, requests, path=DEFAULT_CACHE, steps: int = 10, sample: int = 16, mode=None) -> dict:
    """Choose the kernel of every (lattice, storage, collision) class among `requests` (lbm_request
    objects) with tune_batch on a sample of up to `sample` requests of the class (cached in the JSON
    file), and tell the server (lbm_server_set_class_kernel).  Returns {class: choice}."""
    mode = L.LBM_BATCH_STREAMS if mode is None else mode
    classes = {}
    for r in requests:
        d = r.desc
        classes.setdefault((d.lattice, d.geom.storage, d.geom.collision), []).append(d)
    out = {}
    for (q, st, coll), descs in classes.items():
        b = L.lbm_batch_create(q, st, coll)
        try:
            L.lbm_batch_set_mode(b, mode)
            choice = tune_batch(b, descs[:sample], path, steps)
        finally:
            L.lbm_batch_destroy(b)
        L.lbm_server_set_class_kernel(server, q, st, coll, choice["variant"], choice.get("segment", 0))
        out[(q, st, coll)] = choice
    return out

