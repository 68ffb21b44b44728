"""Autotuner of the launch configuration of a context: the tile shape (the
i-group size: 1, 4 or 8 clusters of a column share one list and their
j-cluster loads), the persistent-grid size and the work units per list
segment.

Each candidate is timed with CUDA events over a few rebuild + force
evaluations on the caller's stream (a new group size rebuilds the lists
first); the fastest is applied and cached per (device, size bucket, number
of systems).  The candidates only change how work is split.  The block
count changes no result bit; the group size and the list split change where
the FP32 force sums of a cluster are cut before they join the fixed-point
totals, so results differ between candidates by FP32 rounding only (every
candidate is within the parity tolerances, and each is run-to-run
bit-identical).  The choice is deterministic for a given cache.
"""

from __future__ import annotations

import json
import math
import os

_CACHE: dict = {}

DEFAULT_CANDIDATES = ([dict(group_clusters=1, blocks_per_sm=b, list_split=s) for b in (2, 3, 4) for s in (1, 2, 4)]
                      + [dict(group_clusters=g, blocks_per_sm=b, list_split=s)
                         for g in (4, 8) for b in (2, 3) for s in (2, 4, 6)])


def _key(ctx) -> str:
    import torch
    dev = torch.cuda.get_device_name()
    bucket = int(math.log2(max(ctx.n_atoms, 1)))
    return f"{dev}|n2^{bucket}|sys{ctx.n_sys}"


def load_cache(path: str) -> None:
    if os.path.exists(path):
        _CACHE.update(json.load(open(path)))


def save_cache(path: str) -> None:
    with open(path, "w") as f:
        json.dump(_CACHE, f, indent=1, sort_keys=True)


def time_config(ctx, pos, q, typ, reps: int = 5) -> float:
    """Mean milliseconds of one rebuild + force evaluation."""
    import torch
    for _ in range(2):
        ctx.build(pos)
        ctx.forces(pos, q, typ)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        ctx.build(pos)
        ctx.forces(pos, q, typ)
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def autotune(ctx, pos, q, typ, candidates=None, reps: int = 5, use_cache: bool = True) -> dict:
    """Pick the fastest candidate for this context, apply it and return it
    with its timing table."""
    key = _key(ctx)
    if use_cache and key in _CACHE:
        best = _CACHE[key]["best"]
        ctx.set_tuning(**best)
        return _CACHE[key]
    table = []
    for cand in candidates or DEFAULT_CANDIDATES:
        try:
            ctx.set_tuning(**cand)
        except Exception:  # configuration not supported (shared memory)
            continue
        table.append((time_config(ctx, pos, q, typ, reps), cand))
    ctx.status()
    table.sort(key=lambda x: x[0])
    best = table[0][1]
    ctx.set_tuning(**best)
    rec = {"best": best, "ms": table[0][0], "table": [(round(t, 5), c) for t, c in table]}
    _CACHE[key] = rec
    return rec
