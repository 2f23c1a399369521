"""Tile-shape autotuner of the batched form.

The batched sweeps run over flattened extended lines (rows, or groups of yc adjacent columns, each with
its two halo nodes on either side, one after the other) in tiles of 192 node records, so no grid size
leaves a ragged tile; the x-tiles have one shape. What remains to choose is the y-tile width yc: 1, 2
or 4 columns of 192 / yc extended rows. Wider tiles load more contiguous bytes per row; narrower ones
form fewer halo records per interface. The choice never changes the arithmetic.

Grids are grouped in size classes (powers of two of nx); for each class every candidate is timed on
that class's grids with ``hw_batch_time_tiles`` (events around the batched sweep launches) and the
fastest is kept. Results are cached per device and class in a JSON file, so later batches reuse them
without timing.
"""
from __future__ import annotations

import json
import math
import os
from typing import Dict, Optional

YC_CANDIDATES = (1, 2, 4)
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_autotune_cache.json")


def size_class(n: int) -> int:
    return int(math.floor(math.log2(max(n, 2))))


def _device_key() -> str:
    try:
        import torch
        return torch.cuda.get_device_name(torch.cuda.current_device()).replace(" ", "_")
    except Exception:
        return "cuda"


def _load(path: str) -> Dict:
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def tune(batch, cache_path: Optional[str] = None, reps: int = 3, force: bool = False) -> Dict:
    """Choose and apply the y-tile width of every grid of ``batch`` (a BatchedSolver)."""
    import paper_2208_01260_gb300 as hw
    path = cache_path or DEFAULT_CACHE
    cache = _load(path)
    dev = cache.setdefault(_device_key() + ":flat", {"yc": {}})
    classes: Dict[int, list] = {}
    for i, g in enumerate(batch.grids):
        classes.setdefault(size_class(g.nx), []).append(i)
    timings: Dict[str, Dict[int, float]] = {}
    for c, ids in sorted(classes.items()):
        key = str(c)
        if force or key not in dev["yc"]:
            best = None
            for yc in YC_CANDIDATES:
                _, ms = hw.hw_batch_time_tiles(batch.h, ids, yc, reps)
                timings.setdefault(key, {})[yc] = ms
                if best is None or ms < best[0]:
                    best = (ms, yc)
            dev["yc"][key] = best[1]
    for i, g in enumerate(batch.grids):
        hw.hw_batch_set_tiles(batch.h, i, dev["yc"][str(size_class(g.nx))])
    try:
        with open(path, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
    except OSError:
        pass
    return {"choices": dev, "timings": timings}
