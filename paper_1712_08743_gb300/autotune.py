"""Tile-shape autotuning of the complex64 multigrid kernels, cached per shape.

The first call for a (padded grid shape, batch size) times the two tile shapes
of each grid-level multigrid kernel on the device (helm_autotune) and stores the
winners in a JSON file; later calls for the same key apply the stored choice
(helm_set_tiles) without timing. The cache is keyed on the shape only, so it is
valid for any slowness model and frequency of that grid.
"""
from __future__ import annotations

import ctypes as C
import json
import os

from . import _lib

NTILES = 48  # 24 levels x (restriction, prolongation)


def default_cache_path() -> str:
    base = os.environ.get("HELM_TUNE_CACHE")
    if base:
        return base
    return os.path.join(os.path.expanduser("~"), ".cache", "helm_gb300_tiles.json")


def cache_key(nx: int, nz: int, nrhs: int) -> str:
    return f"{nx}x{nz}:b{nrhs}:c64:shapes5"


def load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(path: str, cache: dict) -> None:
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def autotune(model, nrhs: int, omega: float, cache_path: str | None = None) -> list[int]:
    """Apply the cached tile choice for this shape, or measure and cache one."""
    path = cache_path or default_cache_path()
    key = cache_key(model.nx, model.nz, nrhs)
    cache = load_cache(path)
    lib = model.lib
    if key in cache and len(cache[key]) == NTILES:
        arr = (C.c_int * NTILES)(*cache[key])
        _lib.check(lib.helm_set_tiles(model.handle, arr), "helm_set_tiles")
        return list(cache[key])
    arr = (C.c_int * NTILES)()
    _lib.check(lib.helm_autotune(model.handle, int(nrhs), float(omega), arr), "helm_autotune")
    cache[key] = list(arr)
    save_cache(path, cache)
    return list(arr)
