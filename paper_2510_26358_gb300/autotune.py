"""Autotuner for the rasteriser's tile size and shared-memory batch depth.

The best (tile, batch depth) pair depends on the rig and the scene: small
tiles waste fewer fragment evaluations but multiply the instances to sort,
deep batches amortise barriers but stage Gaussians that saturated pixels no
longer need.  ``tune`` times every candidate on the caller's own data and
returns the fastest; results are cached per rig/scene signature in a JSON
file so a mapping session tunes once.  Every candidate renders the same
images (the support rule makes the output independent of the tile size), so
the choice only affects speed.
"""
from __future__ import annotations

import hashlib
import json
import os
from typing import Callable, Iterable

# tile (w, h) x batch depth, as the configuration space of the batched raster
CANDIDATES = [(tw, th, d) for (tw, th) in ((8, 8), (16, 16), (16, 32)) for d in (64, 128, 256)]

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def signature(cameras, n_gaussians: int, sh_degree: int, submap_offsets, extra: str = "") -> str:
    """Key of a tuning result: camera sizes, submap sizes, SH degree."""
    sizes = [(int(c.width), int(c.height), int(c.submap)) for c in cameras]
    subs = [int(b) - int(a) for a, b in zip(list(submap_offsets)[:-1], list(submap_offsets)[1:])]
    # Gaussian counts enter on a log scale: the optimum moves slowly with N
    bucket = [max(0, int(round(4 * __import__("math").log2(max(1, s))))) for s in subs]
    raw = json.dumps([sizes, bucket, int(sh_degree), extra])
    return hashlib.sha1(raw.encode()).hexdigest()[:16]


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune(measure: Callable[[int, int, int], float], key: str | None = None,
         candidates: Iterable = CANDIDATES, cache_path: str = CACHE, refresh: bool = False) -> dict:
    """Time ``measure(tile_w, tile_h, depth)`` (milliseconds per step) for each
    candidate and return {"tile_w", "tile_h", "batch_depth", "ms", "timings"}.
    With a ``key``, a cached result is returned unless ``refresh``."""
    cache = _load(cache_path) if key else {}
    if key and not refresh and key in cache:
        return dict(cache[key], cached=True)
    timings = {}
    for tw, th, d in candidates:
        timings[f"{tw}x{th}/{d}"] = float(measure(tw, th, d))
    best = min(timings, key=timings.get)
    tile, depth = best.split("/")
    tw, th = (int(x) for x in tile.split("x"))
    res = {"tile_w": tw, "tile_h": th, "batch_depth": int(depth), "ms": timings[best], "timings": timings}
    if key:
        cache[key] = res
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        tmp = cache_path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    return dict(res, cached=False)


def renderer_measure(cameras, submap_offsets, sh_degree, params, upstream, steps: int = 5, warmup: int = 2,
                     inst_capacity: int | None = None):
    """A ``measure`` callback that times forward + backward of a Renderer on
    the given parameters (torch CUDA tensors) and upstream gradients."""
    import torch
    from . import gsraster as G

    def measure(tw, th, d):
        cfg = G.gs_config_default(tile_w=tw, tile_h=th, batch_depth=d)
        r = G.Renderer(cameras, submap_offsets, sh_degree, config=cfg, inst_capacity=inst_capacity)
        try:
            outs = None
            grads = None

            def step():
                nonlocal outs, grads
                outs = r.forward(*params, outputs=outs)
                grads = r.backward(*params, *upstream, grads=grads)
            for _ in range(warmup):
                step()
            st = r.status()[0]
            if st != G.GS_OK:
                return float("inf")
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(steps):
                step()
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / steps
        finally:
            r.close()
    return measure
