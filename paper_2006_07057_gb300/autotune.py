"""Autotuner for the batched solver's tile size.

For a given batch, each candidate tile size is planned and timed on a short
solve (CUDA events on the launching stream, after one warm-up); the fastest is
kept. Results are cached per (device, SM count, ldr, total-row bucket) in
_build/autotune.json next to the library, so a batch of the same shape class
reuses the choice.
"""
from __future__ import annotations

import json
import math
import os

import torch

from . import build as _build

CANDIDATES = (16 * 1024, 32 * 1024, 44 * 1024, 64 * 1024)
CACHE = os.path.join(_build.OUT, "autotune.json")
PROBE_ITERS = 6


def _key(solver) -> str:
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    rows = sum(p.x.n + p.y.n for p in solver.probs)
    bucket = int(math.log2(max(rows, 1)))
    return f"{props.name}|{props.multi_processor_count}|ldr={solver.ldr}|rows=2^{bucket}"


# The tuner works on one planned batch (an object with probs, records, ldr, mode
# and stream attributes).


def _load() -> dict:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(cache: dict) -> None:
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, CACHE)


def best_batch_tile(solver, candidates=CANDIDATES, use_cache: bool = True) -> int:
    """Tile bytes with the shortest measured batched solve for this batch."""
    from . import lsf_batch_plan, lsf_solve_batched

    key = _key(solver) + f"|{getattr(solver, 'mode', 'stored')}"
    cache = _load() if use_cache else {}
    if key in cache:
        return int(cache[key]["tile_bytes"])
    stream = solver.stream or torch.cuda.current_stream()
    info, _ = lsf_batch_plan(solver.records, solver.ldr, candidates[0], stream,
                             mode=getattr(solver, "mode", "stored"))
    if info.strategy == 1:
        return candidates[0]  # one cluster per problem: no tiles to size
    timings = {}
    for tb in candidates:
        info, plan = lsf_batch_plan(solver.records, solver.ldr, tb, stream,
                                    mode=getattr(solver, "mode", "stored"))
        lsf_solve_batched(info, plan, PROBE_ITERS, stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lsf_solve_batched(info, plan, PROBE_ITERS, stream)
        e1.record(stream)
        e1.synchronize()
        timings[tb] = e0.elapsed_time(e1)
    best = min(timings, key=timings.get)
    cache[key] = {"tile_bytes": best, "ms": timings}
    if use_cache:
        _save(cache)
    return best
