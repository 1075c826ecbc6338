"""Pair-loop shape autotuning with a persistent cache.

The shapes -- active particles staged per shared-memory tile, and warps per cell (CTA) -- of the density and the
force pair loop are chosen by the library's autotuner (sph_autotune), which times every candidate on the caller's
data.  The choice depends on the GPU, the precision, the form (one periodic grid or patches) and the mean
occupancy of the cells, so it is cached under that key in a JSON file and restored with sph_view_set_tiles /
sph_view_set_warps instead of re-timed.
"""
from __future__ import annotations

import json
import math
import os

from . import sph


def default_cache_path() -> str:
    return os.environ.get("SPH_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "sph_views_gb300", "tiles.json"))


def cache_key(gpu_name: str, prec: int, form: str, mean_ppc: float) -> str:
    bucket = int(round(math.log2(max(mean_ppc, 1.0))))
    return f"{gpu_name}|{'f64' if prec == sph.SPH_F64 else 'f32'}|{form}|ppc2^{bucket}"


def tuned_tiles(view, aos_dev, n, params, key: str, cache_path: str | None = None, retune: bool = False):
    """Apply the cached tiles for `key`, or run the autotuner on these records and cache its choice.

    Returns (tile_density, tile_force, warps_density, warps_force, source) with source "cache" or "tuned".  Tuning runs one pass on the
    records, exactly as a step would."""
    path = cache_path or default_cache_path()
    cache = {}
    if os.path.exists(path):
        try:
            with open(path) as fh:
                cache = json.load(fh)
        except (OSError, ValueError):
            cache = {}
    if key in cache and not retune and len(cache[key]) == 4:
        td, tf, wd, wf = cache[key]
        sph.sph_view_set_tiles(view, td, tf)
        sph.sph_view_set_warps(view, wd, wf)
        return td, tf, wd, wf, "cache"
    sph.sph_autotune(view, aos_dev, n, params)
    td, tf, wd, wf = sph.sph_view_get_tuning(view)
    cache[key] = [td, tf, wd, wf]
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass
    return td, tf, wd, wf, "tuned"
