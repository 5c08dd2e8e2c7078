"""Autotuner for multi-view batches: picks the tile edge (8, 16, 32) and the
radix sort's digit width (4 to 8 bits) by timing the actual batch with CUDA
events, and caches the choice per (device, Gaussian-count bucket,
pixel-count bucket, camera count, mode).  The tile edge also fixes the block
shape of the blend and its backward (one thread per pixel: 64, 256 or 1024
threads per CTA, 8 x 4-pixel warp sub-tiles), so the 15 candidates cover
tile x threads per tile x digit width.

In the exact modes (SnugBox, AccuTile) the image does not depend on the tile
edge or on the digit width, so the choice changes speed only.
"""
from __future__ import annotations

import json
import math
import os
from pathlib import Path

import torch

from . import raster

CANDIDATES = [(t, d) for t in (8, 16, 32) for d in (0, 7, 6, 5, 4)]  # d = 0: 8-bit digits
CACHE = Path(__file__).resolve().parent / "_build" / "autotune.json"


def bucket_key(device_name: str, n, cams, mode) -> str:
    name = device_name.replace(" ", "_")
    pixels = sum(c.width * c.height for c in cams)
    return f"{name}|n2^{max(0, round(math.log2(max(n, 1))))}|px2^{max(0, round(math.log2(max(pixels, 1))))}" \
           f"|v{len(cams)}|{mode}"


def _time(renderer, scene, cams, reps):
    renderer.render(scene, cams)  # sizes the frame
    s = renderer.rast.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(2):
        renderer._launch(scene, cams)
    e0.record(s)
    for _ in range(reps):
        renderer._launch(scene, cams)
    e1.record(s)
    torch.cuda.synchronize(renderer.device)
    return e0.elapsed_time(e1) / reps


def tune(scene, cams, device=None, mode="accutile", reps=5, cache_path: Path | None = CACHE, force=False,
         timer=None, device_name: str | None = None):
    """Returns {"tile", "sort_digit_bits", "ms", "timings", "cached"} for this
    batch.  timer(tile, sort_digit_bits) -> ms replaces the CUDA-event timing
    of a BatchRenderer (and device_name the device query) where given."""
    device = torch.device(device or "cuda")
    n = int(scene.means.shape[1])
    if device_name is None:
        device_name = torch.cuda.get_device_name(device)
    key = bucket_key(device_name, n, cams, mode)
    cache = {}
    if cache_path is not None and cache_path.exists():
        try:
            cache = json.loads(cache_path.read_text())
        except Exception:
            cache = {}
    if not force and key in cache:
        return dict(cache[key], cached=True)
    if timer is None:
        def timer(tile, d):
            r = raster.BatchRenderer(device, tile=tile, mode=mode, sort_digit_bits=d)
            ms = _time(r, scene, cams, reps)
            del r
            torch.cuda.empty_cache()
            return ms
    timings = {f"{tile}/{d or 8}": float(timer(tile, d)) for tile, d in CANDIDATES}
    best = min(timings, key=timings.get)
    tile, d = (int(x) for x in best.split("/"))
    choice = {"tile": tile, "sort_digit_bits": 0 if d == 8 else d, "ms": timings[best], "timings": timings}
    if cache_path is not None:
        cache[key] = choice
        cache_path.parent.mkdir(parents=True, exist_ok=True)
        tmp = cache_path.with_suffix(f".{os.getpid()}.tmp")
        tmp.write_text(json.dumps(cache, indent=1))
        os.replace(tmp, cache_path)
    return dict(choice, cached=False)
