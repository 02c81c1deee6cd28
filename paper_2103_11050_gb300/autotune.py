"""Launch-shape autotuning with a JSON cache.

The library's mpm_autotune times every candidate launch shape of the step's kernels on a
context's own data and keeps the fastest (threads per CTA and factor staging of the local
solves, tile height of the transport kernel).  The best shape depends on the geometry (how
many subdomains of what size, how many realisations) and the GPU, so the result is cached
per (GPU, realisations, grid, decomposition, precision) in a JSON file and reused by later
contexts of the same shape without timing anything.
"""
from __future__ import annotations

import json
import os

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_cache.json")


def _runs(v):
    """Run-length form of a width list: [16, 16, 8] -> "16*2,8"."""
    out, k = [], 0
    v = [int(x) for x in v]
    while k < len(v):
        n = 1
        while k + n < len(v) and v[k + n] == v[k]:
            n += 1
        out.append(f"{v[k]}*{n}" if n > 1 else f"{v[k]}")
        k += n
    return ",".join(out)


def shape_key(R, nx, ny, col_w, row_h, prec, device_name=""):
    return f"{device_name}|R={R}|{nx}x{ny}|cols={_runs(col_w)}|rows={_runs(row_h)}|prec={prec}"


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def cached(key, names, path=CACHE):
    """The cached tuning of `key` when it holds exactly the parameters `names`, else None."""
    entry = _load(path).get(key)
    if entry is not None and set(entry["tuning"]) == set(names):
        return dict(entry["tuning"])
    return None


def tuned(ctx, key, path=CACHE, reps=5):
    """Apply the cached tuning of `key` to ctx, or (cache miss) autotune ctx, which must hold a
    stored basis, and cache the result.  Returns (tuning dict, source) with source "cache" or
    "autotune"."""
    cache = _load(path)
    if key in cache and set(cache[key]["tuning"]) == set(ctx.get_tuning()):
        ctx.set_tuning(cache[key]["tuning"])
        return cache[key]["tuning"], "cache"
    tune, ms = ctx.autotune(reps)
    cache = _load(path)  # re-read: another process may have written meanwhile
    cache[key] = {"tuning": tune, "best_ms": {"transport": ms[0], "local_solve": ms[1], "downscale_solve": ms[2],
                                              "interface_sweeps": ms[3]}}
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return tune, "autotune"
