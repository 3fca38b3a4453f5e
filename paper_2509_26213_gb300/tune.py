"""Autotuner for the render launch: ray-tile shape, lane-refill threshold and brick size.

Times every candidate with CUDA events (median of `reps` frames after `warmup`) and caches the
winner in a JSON file keyed by the GPU name and a caller-supplied workload key, so a later run
on the same GPU reuses it without timing.  Tile shape and refill threshold are render
parameters; the brick size is a volume property, so the caller supplies `make_volume(brick)`.
Only performance depends on the choice: every candidate renders the same image.
"""
from __future__ import annotations

import json
import os
import statistics

import torch

# one warp's worth of rays per tile first (the shapes that win on GB300), then larger tiles
DEFAULT_TILES = ((4, 8), (8, 4), (2, 16), (32, 1), (8, 8), (16, 16), (32, 4))
DEFAULT_REFILL = (16, 20, 28)


def _gpu_name() -> str:
    return torch.cuda.get_device_name(torch.cuda.current_device())


def _time(vol, cams, tf, params, reps, warmup, flush):
    for _ in range(warmup):
        vol.render(cams, tf, params)
    torch.cuda.synchronize()
    evs = []
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        vol.render(cams, tf, params)
        b.record()
        evs.append((a, b))
    torch.cuda.synchronize()
    return statistics.median(a.elapsed_time(b) for a, b in evs)


def autotune(make_volume, cams, tf, params: dict, key: str, bricks=(32, 64), tiles=DEFAULT_TILES,
             refills=DEFAULT_REFILL, reps: int = 5, warmup: int = 2, cache_path: str | None = None,
             flush_bytes: int = 256 << 20, timer=None, device_name: str | None = None) -> dict:
    """Returns {"brick", "tile_w", "tile_h", "refill", "ms", "timings", "cached"}.

    make_volume(brick) -> Volume (resident, ready to render); the tuner closes each volume
    it does not return, and returns the winner's volume under "volume" unless it came from the
    cache (then the caller builds it).  timer(vol, cams, tf, params) -> ms replaces the timing
    of renders with CUDA events, and device_name the GPU's name in the cache key (both for
    tests of the selection and the cache without a GPU)."""
    cache_key = f"{device_name or _gpu_name()}|{key}"
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if cache_key in cache:
            out = dict(cache[cache_key])
            out["cached"] = True
            return out
    if timer is None:
        flush = torch.empty(flush_bytes, dtype=torch.uint8, device="cuda") if flush_bytes else None

        def timer(vol, cams, tf, prm):
            return _time(vol, cams, tf, prm, reps, warmup, flush)
    timings = {}
    best = None
    best_vol = None
    for brick in bricks:
        vol = make_volume(brick)
        local_best = None
        for tw, th in tiles:
            for refill in refills:
                prm = dict(params, tile_w=tw, tile_h=th, refill=refill)
                ms = timer(vol, cams, tf, prm)
                timings[f"b{brick} t{tw}x{th} r{refill}"] = ms
                if local_best is None or ms < local_best[0]:
                    local_best = (ms, tw, th, refill)
        if best is None or local_best[0] < best["ms"]:
            if best_vol is not None:
                best_vol.close()
            best = {"brick": brick, "tile_w": local_best[1], "tile_h": local_best[2], "refill": local_best[3],
                    "ms": local_best[0]}
            best_vol = vol
        else:
            vol.close()
        if torch.cuda.is_available():
            torch.cuda.empty_cache()
    best["timings"] = timings
    if cache_path:
        cache[cache_key] = {k: v for k, v in best.items()}
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    best["cached"] = False
    best["volume"] = best_vol
    return best
