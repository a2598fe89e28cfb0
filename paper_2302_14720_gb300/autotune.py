"""Tile-shape autotuning for the tiled sweep.

The sweep's tile shape (tile width and height, rows per bond strip) changes
only its speed, never its results (every draw is keyed by site and counter,
and labels are canonical), so the fastest shape can be chosen by measurement
per lattice size. `tune` times every compiled shape on a lattice of each
requested side with the library's own per-phase CUDA-event timing, picks the
fastest, and installs the choice process-wide with sw_tune_shape (bucket =
ceil(log2 L)); `save` / `load` keep the table in a JSON file keyed by the
GPU's name so a later process can install it without measuring again.
"""
from __future__ import annotations

import json
import math
import os
from typing import Callable, Iterable

import numpy as np

from . import (SW_INIT_HOT, Lattice, sw_num_shapes, sw_shape_info, sw_timing, sw_timing_read, sw_tune_shape)


def bucket_of(L: int) -> int:
    """ceil(log2 L), the library's tuning bucket of side L."""
    return max(0, math.ceil(math.log2(L))) if L > 1 else 0


def time_shape(L: int, shape: int, beta: float = 0.44068679, sweeps: int = 5, warmup: int = 2,
               seed: int = 1) -> float:
    """Device milliseconds per sweep of side L with tile shape `shape`."""
    os.environ["SW_TILE_SHAPE"] = str(shape)
    try:
        lat = Lattice(L, beta, seed, SW_INIT_HOT)
    finally:
        os.environ.pop("SW_TILE_SHAPE", None)
    with lat:
        lat.sweep(warmup)
        sw_timing(lat.h, True)
        lat.sweep(sweeps)
        ms, n = sw_timing_read(lat.h)
        lat.observables(0, 1)  # checks the device error flag
    per = ms / np.maximum(n, 1)
    return float(per[:3].sum())


def choose(times: dict[int, float]) -> int:
    """The fastest shape; ties go to the lower index."""
    return min(sorted(times), key=lambda s: times[s])


def tune(sides: Iterable[int], shapes: Iterable[int] | None = None,
         timer: Callable[[int, int], float] = time_shape, install: bool = True) -> dict:
    """Measure every shape at every side; returns {bucket: {"shape", "L", "ms": {shape: ms}}}."""
    shapes = list(range(sw_num_shapes())) if shapes is None else list(shapes)
    table = {}
    for L in sides:
        times = {s: timer(L, s) for s in shapes}
        best = choose(times)
        b = bucket_of(L)
        table[b] = {"shape": best, "L": L, "ms": times, "info": sw_shape_info(best)}
        if install:
            sw_tune_shape(b, best)
    return table


def gpu_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name(0)
    except Exception:
        return "unknown"


def save(table: dict, path: str, device: str | None = None) -> None:
    data = {}
    if os.path.exists(path):
        with open(path) as fh:
            data = json.load(fh)
    data[device or gpu_name()] = {str(b): {"shape": v["shape"], "L": v["L"]} for b, v in table.items()}
    with open(path, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)


def load(path: str, device: str | None = None, install: bool = True) -> dict:
    """Install a saved table for this GPU (nothing if none was saved)."""
    if not os.path.exists(path):
        return {}
    with open(path) as fh:
        data = json.load(fh)
    entry = data.get(device or gpu_name(), {})
    table = {int(b): v for b, v in entry.items()}
    n = sw_num_shapes()
    if install:
        for b, v in table.items():
            if 0 <= v["shape"] < n:
                sw_tune_shape(b, v["shape"])
    return table
