"""Tile-shape autotuner of the batched form.

The batched kernels take two tile shapes per grid: the row width tx of an x-tile (32, 64 or 128
threads, each row covering tx - 3 interfaces; 128/tx rows per tile) and the number of y-interfaces per
y-segment. Neither changes the
arithmetic. Grids are grouped in size classes (powers of two of nx for the x-tiles, of ny for the
y-segments); for each class every candidate is timed on that class's grids with
``hw_batch_time_tiles`` (events around the batched sweep launches) and the fastest is kept. Results
are cached per device and class in a JSON file, so later batches reuse them without timing.
"""
from __future__ import annotations

import json
import math
import os
from typing import Dict, Optional

TX_CANDIDATES = (32, 64, 128)
SEG_CANDIDATES = (16, 32, 64, 128, 256)
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
    """Choose and apply tile shapes for every grid of ``batch`` (a BatchedSolver)."""
    import paper_2208_01260_gb300 as hw
    path = cache_path or DEFAULT_CACHE
    cache = _load(path)
    dev = cache.setdefault(_device_key(), {"tx": {}, "seg": {}})
    grids = batch.grids
    xcls: Dict[int, list] = {}
    ycls: Dict[int, list] = {}
    for i, g in enumerate(grids):
        xcls.setdefault(size_class(g.nx), []).append(i)
        ycls.setdefault(size_class(g.ny), []).append(i)
    timings = {"tx": {}, "seg": {}}
    for c, ids in sorted(xcls.items()):
        key = str(c)
        if force or key not in dev["tx"]:
            best = None
            for tx in TX_CANDIDATES:
                ms, _ = hw.hw_batch_time_tiles(batch.h, ids, tx, 64, reps)
                timings["tx"].setdefault(key, {})[tx] = ms
                if best is None or ms < best[0]:
                    best = (ms, tx)
            dev["tx"][key] = best[1]
    for c, ids in sorted(ycls.items()):
        key = str(c)
        if force or key not in dev["seg"]:
            best = None
            for seg in SEG_CANDIDATES:
                _, ms = hw.hw_batch_time_tiles(batch.h, ids, 128, seg, reps)
                timings["seg"].setdefault(key, {})[seg] = ms
                if best is None or ms < best[0]:
                    best = (ms, seg)
            dev["seg"][key] = best[1]
    for i, g in enumerate(grids):
        hw.hw_batch_set_tiles(batch.h, i, dev["tx"][str(size_class(g.nx))], dev["seg"][str(size_class(g.ny))])
    try:
        with open(path, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
    except OSError:
        pass
    return {"choices": dev, "timings": timings}
