"""Autotuner for the fused kernel's tile shape.

For each (channels, W) it times the fused kernel on a synthetic page with
every strip width that fits shared memory (512, 256, 128 output columns) and
several heights of the rows each CTA walks (the library's default split over
one CTA per SM, or a fixed number of rows per CTA, which sets the grid) and
keeps the fastest pair, then the fastest edge weight for it (the share of CTAs
given to the page's first and last strips, whose clipped windows take the
slower path).  The page is tall (4096 rows by default) so that, as
in a batch or a stream of pages, the W rows of warm-up at the top of each
strip segment are amortized.  Results are cached as JSON keyed by GPU name,
library version and a hash of the kernel sources, so tuning is done once per
machine and build; single-page calls take ``bnz_tile(tile_w, tile_h)`` from
the table (``tile_shape_for``) and batches their per-page ``tile_w``
(``tile_for``).
"""
from __future__ import annotations

import json
import os

from . import (BNZ_SAUVOLA, BnzError, alloc_pitched, bnz_binarize_dev, bnz_tile, load)

DEFAULT_WINDOWS = (15, 25, 31, 45, 61, 75, 101)
TILE_WIDTHS = (512, 256, 128)
TILE_HEIGHTS = (0, 128, 256, 512)   # rows per CTA; 0 = the library's split over one CTA per SM
EDGE_WEIGHTS = (16, 18, 20, 22, 24)  # an edge strip's row cost in sixteenths of an inner strip's


def build_key() -> str:
    """Library version and a hash of the kernel sources: a table tuned on another build is not reused."""
    import hashlib
    from . import bnz_version
    h = hashlib.sha256()
    csrc = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(name.encode() + f.read())
    return f"v{bnz_version()}-{h.hexdigest()[:12]}"


def cache_path(gpu_name: str | None = None) -> str:
    import torch
    name = gpu_name or torch.cuda.get_device_name()
    base = os.environ.get("BNZ_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "bnz")
    if base.endswith(".json"):
        return base
    tag = "".join(c if c.isalnum() else "_" for c in name)
    return os.path.join(base, f"tune-{tag}-{build_key()}.json")


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
         save: bool = True, heights=TILE_HEIGHTS) -> dict:
    """Return {"1": {"15": {"tile_w": 512, "tile_h": 0, "edge_weight": 20, "ms": ...}, ...}, "3": {...}} and
    cache it unless save=False."""
    import torch
    import synth
    from . import to_device_pitched
    load()
    table: dict = {"gpu": torch.cuda.get_device_name(), "shape": list(shape), "build": build_key()}
    for ch in channels:
        page = synth.page(shape[0], shape[1], seed, synth.STAINS if ch == 3 else synth.DOC, ch)
        src = to_device_pitched(page)
        out = alloc_pitched(shape[0], shape[1])
        best = {}
        for W in windows:
            timings = {}
            for tw in TILE_WIDTHS:
                for th in heights:
                    try:
                        timings[(tw, th)] = _time_one(src, out, W, bnz_tile(tw, th, 0, 0), reps)
                    except BnzError:
                        break  # this width does not fit shared memory
            (tw, th) = min(timings, key=timings.get)
            edge = {ew: _time_one(src, out, W, bnz_tile(tw, th, 0, ew), reps) for ew in EDGE_WEIGHTS}
            ew = min(edge, key=edge.get)
            best[str(W)] = {"tile_w": tw, "tile_h": th, "edge_weight": ew, "ms": round(edge[ew], 5)}
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


def _entry(table: dict | None, channels: int, W: int) -> dict | None:
    if not table or str(channels) not in table:
        return None
    entries = {int(k): v for k, v in table[str(channels)].items()}
    nearest = min(entries, key=lambda w: (abs(w - W), w))
    e = entries[nearest]
    return e if isinstance(e, dict) else {"tile_w": int(e), "tile_h": 0}


def tile_for(table: dict | None, channels: int, W: int) -> int:
    """Tuned strip width for the nearest tuned W (0 = let the library choose)."""
    e = _entry(table, channels, W)
    return int(e["tile_w"]) if e else 0


def tile_shape_for(table: dict | None, channels: int, W: int):
    """bnz_tile(tile_w, tile_h, 0, edge_weight) tuned for the nearest W, or None (library default)."""
    e = _entry(table, channels, W)
    return bnz_tile(int(e["tile_w"]), int(e["tile_h"]), 0, int(e.get("edge_weight", 0))) if e else None
