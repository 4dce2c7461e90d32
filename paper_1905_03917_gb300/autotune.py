"""Autotuner of the finite-volume tile shape.

For a grid-size bucket, every supported tile shape is timed on a real
problem of that bucket -- whole multi-time-step cycles, since the shape
also sets which cells a fluid's active tiles cover, how a small fluid's
tiles split and the tiles of the primitive recovery -- and the fastest is
kept in a JSON cache keyed by (kernel, bucket, device).  Tuning runs from a checkpoint and restores it,
so the tuned problem's state is unchanged.  Results never depend on the
tile shape (each face flux is computed by the same formula whichever tile
holds it).
"""
from __future__ import annotations

import json
import os
import time

SHAPES = [(32, 8), (32, 4), (16, 8), (16, 16), (64, 4)]
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def bucket(nx: int, ny: int) -> str:
    """Size bucket: cell count rounded up to a power of two, and the aspect."""
    n = nx * ny
    b = 1
    while b < n:
        b *= 2
    return f"cells<={b},{'wide' if nx >= 2 * ny else 'tall' if ny >= 2 * nx else 'square'}"


def device_key(device: int = 0) -> str:
    try:
        import torch
        p = torch.cuda.get_device_properties(device)
        return f"{p.name}/sm{p.major}{p.minor}/{p.multi_processor_count}"
    except Exception:
        return "unknown"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, data):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def measure(solver, shape, cycles=3):
    """Wall-clock milliseconds per multi-time-step cycle with the given tile
    shape (the stepping call returns once the GPU has finished)."""
    solver.set_tile_shape(*shape)
    solver.step_multi_dt(1)  # warm-up with this shape (graph rebuild)
    t0 = time.perf_counter()
    solver.step_multi_dt(cycles)
    return 1e3 * (time.perf_counter() - t0) / cycles


def tune(solver, cache=DEFAULT_CACHE, device=0, cycles=3, force=False):
    """Pick (and cache) the fastest tile shape for this solver's bucket,
    apply it to the solver and return (shape, record)."""
    key = f"k_fv_stage|{bucket(solver.nx, solver.ny)}|{device_key(device)}"
    data = _load(cache)
    if not force and key in data:
        shape = tuple(data[key]["shape"])
        solver.set_tile_shape(*shape)
        return shape, data[key]
    ckpt = solver.save()
    times = {}
    for shape in SHAPES:
        times[f"{shape[0]}x{shape[1]}"] = measure(solver, shape, cycles)
        solver.load_checkpoint(ckpt)
    best = min(SHAPES, key=lambda s: times[f"{s[0]}x{s[1]}"])
    rec = {"shape": list(best), "ms_per_cycle": times, "grid": [solver.nx, solver.ny]}
    data = _load(cache)
    data[key] = rec
    _store(cache, data)
    solver.set_tile_shape(*best)
    return best, rec


def tune_batch(batch, cache=DEFAULT_CACHE, device=0, cycles=3):
    """Tune one representative instance per bucket and apply its shape to
    every instance of the bucket; returns {bucket: shape}."""
    chosen = {}
    for s in batch.instances:
        b = bucket(s.nx, s.ny)
        if b not in chosen:
            chosen[b], _ = tune(s, cache=cache, device=device, cycles=cycles)
        else:
            s.set_tile_shape(*chosen[b])
    return chosen
