"""Autotuner of the primal-dual sweep schedule.

Every schedule (sweep kernel variant, block visiting order, resident CTAs per SM,
graph-captured loop) computes the same iterates bit for bit; they differ only in
speed, which depends on the map (block count, how neighbours are spread in block
index order) and the storage precision.  The tuner times candidate schedules on
the caller's own map with a few cold-start iterations each and keeps the fastest.

Call it before the solve it is meant to speed up: a trial starts from p = u = u^ = 0
and leaves its own iterate behind, which the next cold-start regularisation
discards.  Results are cached per (device, precision, block-count bucket), in memory
and optionally in a JSON file.
"""

from __future__ import annotations

import json
import math
import os

from . import native as N

# (sweep_kernel, order, ctas_per_sm, use_graph); ctas_per_sm 0 = the kernel's default
DEFAULT_CANDIDATES = (
    (2, 1, 0, 1), (2, 0, 0, 1), (2, 1, 2, 1), (2, 0, 2, 1), (2, 1, 3, 1),
    (3, 1, 0, 1), (3, 0, 0, 1), (1, 1, 0, 1), (0, 1, 0, 1), (2, 1, 0, 0),
    (4, 1, 0, 1), (4, 1, 2, 1), (4, 0, 2, 1), (4, 0, 0, 1), (4, 0, 3, 1),
    (5, 0, 0, 1), (5, 1, 0, 1), (5, 0, 2, 1),
    (6, 0, 0, 1), (6, 1, 0, 1), (6, 0, 1, 1), (6, 0, 3, 1),
    (7, 0, 2, 1), (7, 0, 0, 1), (7, 0, 3, 1), (8, 0, 2, 1), (8, 0, 0, 1), (8, 0, 3, 1),
    (9, 0, 0, 1), (9, 0, 1, 1), (9, 0, 3, 1),
)

_cache: dict = {}


def _bucket(n_blocks: int) -> int:
    return 0 if n_blocks <= 0 else int(round(math.log2(n_blocks) * 2))


def _key(ctx, precision: int, n_blocks: int) -> str:
    import torch
    dev = torch.cuda.get_device_name(torch.cuda.current_device()) if torch.cuda.is_available() else "cpu"
    return f"{dev}|p{precision}|b{_bucket(n_blocks)}"


def time_schedule(ctx, schedule, iters: int = 10, repeats: int = 2, stream=None) -> float:
    """Mean sweep time (ms per iteration) of one schedule on the context's current map."""
    N.denser_set_schedule(ctx, *schedule)
    N.denser_regularize(ctx, iters, 0.0, 0, stream)  # warm: records the graph, the block order
    best = math.inf
    for _ in range(repeats):
        st = N.denser_regularize(ctx, iters, 0.0, 0, stream)
        best = min(best, st.sweep_ms / max(st.iters, 1))
    return best


def autotune(ctx, precision: int = 0, iters: int = 10, candidates=DEFAULT_CANDIDATES, cache_file=None,
             stream=None, use_cache: bool = True) -> dict:
    """Picks and sets the fastest schedule for the context's map; returns
    {"schedule": ..., "ms_per_iter": ..., "table": [(schedule, ms), ...], "cached": bool}."""
    n_blocks = N.denser_num_blocks(ctx)
    key = _key(ctx, precision, n_blocks)
    if cache_file and os.path.exists(cache_file) and not _cache:
        try:
            with open(cache_file) as fh:
                _cache.update(json.load(fh))
        except (OSError, ValueError):
            pass
    if use_cache and key in _cache:
        hit = _cache[key]
        N.denser_set_schedule(ctx, *hit["schedule"])
        return dict(hit, cached=True)
    table = []
    for sch in candidates:
        try:
            table.append((tuple(sch), time_schedule(ctx, sch, iters, stream=stream)))
        except N.DenserError:
            continue
    if not table:
        raise RuntimeError("no schedule could be timed")
    best = min(table, key=lambda t: t[1])
    N.denser_set_schedule(ctx, *best[0])
    result = {"schedule": list(best[0]), "ms_per_iter": best[1], "table": [[list(s), t] for s, t in table]}
    _cache[key] = result
    if cache_file:
        try:
            with open(cache_file, "w") as fh:
                json.dump(_cache, fh, indent=1)
        except OSError:
            pass
    return dict(result, cached=False)
