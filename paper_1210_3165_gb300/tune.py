"""Autotuner for the fused kernel's strip width.

For each (channels, W) it times the fused kernel with every strip width that
fits shared memory (512, 256, 128 output columns) on a synthetic page and
keeps the fastest.  The page is tall (4096 rows by default) so that, as in a
batch or a stream of pages, the W rows of warm-up at the top of each strip
segment are amortized; on short pages narrower strips win only because they
give each CTA more rows per segment.  Results are cached as JSON keyed by GPU name, so tuning is
done once per machine; batches take their per-page ``tile_w`` from the table.
"""
from __future__ import annotations

import json
import os

from . import (BNZ_SAUVOLA, BnzError, alloc_pitched, bnz_binarize_dev, bnz_tile, load)

DEFAULT_WINDOWS = (15, 25, 31, 45, 61, 75, 101)
TILE_WIDTHS = (512, 256, 128)


def cache_path(gpu_name: str | None = None) -> str:
    import torch
    name = gpu_name or torch.cuda.get_device_name()
    base = os.environ.get("BNZ_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "bnz")
    if base.endswith(".json"):
        return base
    return os.path.join(base, "tune-" + "".join(c if c.isalnum() else "_" for c in name) + ".json")


def _time_one(src, out, W, tile, reps):
    import torch
    for _ in range(2):
        bnz_binarize_dev(src, W, BNZ_SAUVOLA, 0.5, 128.0, out, tile=tile)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    for _ in range(reps):
        start.record()
        bnz_binarize_dev(src, W, BNZ_SAUVOLA, 0.5, 128.0, out, tile=tile)
        end.record()
        end.synchronize()
        times.append(start.elapsed_time(end))
    times.sort()
    return times[len(times) // 2]


def tune(windows=DEFAULT_WINDOWS, channels=(1, 3), shape=(4096, 4096), reps: int = 7, seed: int = 4,
         save: bool = True) -> dict:
    """Return {"1": {"15": 512, ...}, "3": {...}} and cache it unless save=False."""
    import torch
    import synth
    from . import to_device_pitched
    load()
    table: dict = {"gpu": torch.cuda.get_device_name(), "shape": list(shape)}
    for ch in channels:
        page = synth.page(shape[0], shape[1], seed, synth.STAINS if ch == 3 else synth.DOC, ch)
        src = to_device_pitched(page)
        out = alloc_pitched(shape[0], shape[1])
        best = {}
        for W in windows:
            timings = {}
            for tw in TILE_WIDTHS:
                try:
                    timings[tw] = _time_one(src, out, W, bnz_tile(tw, 0, 0, 0), reps)
                except BnzError:
                    continue  # does not fit shared memory
            best[str(W)] = min(timings, key=timings.get)
        table[str(ch)] = best
    if save:
        path = cache_path()
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as f:
            json.dump(table, f, indent=1)
    return table


def load_table(path: str | None = None) -> dict | None:
    try:
        with open(path or cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return None


def tile_for(table: dict | None, channels: int, W: int) -> int:
    """Tuned strip width for the nearest tuned W (0 = let the library choose)."""
    if not table or str(channels) not in table:
        return 0
    entries = {int(k): v for k, v in table[str(channels)].items()}
    nearest = min(entries, key=lambda w: (abs(w - W), w))
    return int(entries[nearest])
