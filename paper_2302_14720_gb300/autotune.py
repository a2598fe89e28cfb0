"""Autotuning of the tiled sweep and of the batched form.

The sweep's tile shape (tile width and height, rows per bond strip) changes
only its speed, never its results (every draw is keyed by site and counter,
and labels are canonical), so the fastest shape can be chosen by measurement
per lattice size. `tune` times every compiled shape on a lattice of each
requested side with the library's own per-phase CUDA-event timing, picks the
fastest, and installs the choice process-wide with sw_tune_shape (bucket =
ceil(log2 L)); `save` / `load` keep the table in a JSON file keyed by the
GPU's name so a later process can install it without measuring again.

For a batch, `tune_batch` searches the tile shape together with the batch's
schedule (per-phase launches or one fused persistent launch per chunk) and
the side up to which replicas run on the one-CTA path, by timing each
candidate on a scratch batch with the same replicas (again only speed
changes, never the chains); `apply_batch` sets the chosen schedule and
threshold on a live batch created with the chosen shape.
"""
from __future__ import annotations

import json
import math
import os
from typing import Callable, Iterable

import numpy as np

from . import (SW_INIT_HOT, SW_SCHEDULE_FUSED, SW_SCHEDULE_PHASES, SWError, Lattice, sw_batch_create,
               sw_batch_destroy, sw_batch_observables, sw_batch_set_schedule, sw_batch_set_small, sw_batch_sweep,
               sw_num_shapes, sw_shape_info, sw_timing, sw_timing_read, sw_tune_shape)


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
    # every kernel of the timed sweeps (a sweep's phase 3 may carry the next
    # sweep's phase 1), over the sweeps
    return float(ms.sum() / sweeps)


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


# ------------------------------------------------------------------ batches

def time_batch(L, beta, seed, shape: int, schedule: int, small_max_L: int, chunk: int = 10, chunks: int = 3,
               stream=None) -> float:
    """Device milliseconds per sweep of a scratch batch of these replicas
    under (shape, schedule, small_max_L): CUDA events around `chunks`
    replays of a `chunk`-sweep graph, after one warm-up chunk (capture)."""
    import torch
    st = stream or torch.cuda.Stream()
    b = sw_batch_create(L, beta, seed, shape=shape, stream=st.cuda_stream)
    try:
        sw_batch_set_schedule(b, schedule)
        sw_batch_set_small(b, small_max_L)
        sw_batch_sweep(b, chunk)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(chunks):
            sw_batch_sweep(b, chunk)
        e1.record(st)
        torch.cuda.synchronize()
        sw_batch_observables(b, 0, 0, 1)  # checks the device error flag
        return e0.elapsed_time(e1) / (chunk * chunks)
    finally:
        sw_batch_destroy(b)


def batch_candidates(shapes: Iterable[int], small=(0, 64, 181)) -> list[tuple[int, int, int]]:
    """(shape, schedule, small_max_L) triples; the fused schedule only for
    shapes whose phases 1 and 3 run the same block (64-row tiles of 2-row
    strips, 128-row tiles of 4-row strips)."""
    out = []
    for sh in shapes:
        info = sw_shape_info(sh)
        fused_ok = info["tile_h"] == 32 * info["strip_h"]
        for sched in ((SW_SCHEDULE_PHASES, SW_SCHEDULE_FUSED) if fused_ok else (SW_SCHEDULE_PHASES,)):
            for sm in small:
                out.append((sh, sched, sm))
    return out


def tune_batch(L, beta, seed, candidates: Iterable[tuple[int, int, int]] | None = None,
               timer: Callable[..., float] | None = None) -> dict:
    """The fastest (shape, schedule, small_max_L) for this set of replicas:
    {"shape", "schedule", "small_max_L", "ms_per_sweep", "ms": {candidate: ms}}."""
    timer = timer or (lambda sh, sc, sm: time_batch(L, beta, seed, sh, sc, sm))
    if candidates is None:
        candidates = batch_candidates([6, 4])
    times = {}
    for cand in candidates:
        try:
            times[cand] = timer(*cand)
        except SWError:
            continue  # a candidate the library refuses (e.g. a shape without the fused schedule)
    if not times:
        raise RuntimeError("no batch candidate could be timed")
    best = min(sorted(times), key=lambda c: times[c])
    return {"shape": best[0], "schedule": best[1], "small_max_L": best[2], "ms_per_sweep": times[best],
            "ms": {f"shape{c[0]}/schedule{c[1]}/small{c[2]}": t for c, t in times.items()}}


def apply_batch(b: int, choice: dict) -> None:
    """Set the tuned schedule and one-CTA threshold on a batch (created with
    choice["shape"])."""
    sw_batch_set_schedule(b, choice["schedule"])
    sw_batch_set_small(b, choice["small_max_L"])
