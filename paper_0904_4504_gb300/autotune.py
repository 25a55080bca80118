"""Kernel choice with a JSON cache: time the step-kernel candidates once per problem class
(lattice, storage type, collision, equilibrium order, grid) with lbm_tune, keep the result in a JSON
file, and apply the cached choice to later simulations of the same class."""
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
