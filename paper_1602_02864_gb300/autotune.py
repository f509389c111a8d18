"""Autotuned plans with a JSON cache.

spmm_autotune (in the library) times candidate warp-task plans for one call
shape and leaves the handle on the fastest.  This module remembers the
winner per (GPU, matrix shape and nonzeros, value type, k, X type,
orientation) in a JSON file, so a later process re-plans directly instead of
searching again.
"""
from __future__ import annotations

import json
import os
import tempfile

from . import spmm as _sp

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "spmm_autotune.json")

# A short candidate list for power-law graphs: task size, the short-row limit
# and the L2 policy of the X gathers are the knobs that mattered on R-MAT.
POWER_LAW_CANDIDATES = [dict(task_nnz=512, short_max=63, long_row=512, x_l2_policy=2),
                        dict(task_nnz=512, short_max=31, long_row=512, x_l2_policy=2),
                        dict(task_nnz=256, short_max=63, long_row=512, x_l2_policy=2),
                        dict(task_nnz=512, short_max=63, long_row=512, x_l2_policy=1)]


def _key(h, k, xtype, transpose) -> str:
    import torch
    info = _sp.spmm_get_info(h)
    return "|".join(str(x) for x in (torch.cuda.get_device_name(), info["n_rows"], info["n_cols"], info["nnz"],
                                     info["value_dtype"], k, xtype, int(bool(transpose))))


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(path, data):
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=os.path.dirname(path) or ".", suffix=".tmp")
    with os.fdopen(fd, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(matrix, k, xtype=_sp.SPMM_F32, transpose=False, cache_path: str | None = DEFAULT_CACHE, candidates=None,
         reps=3) -> dict:
    """Put `matrix` (a SparseMatrix) on the best plan for this call shape.
    Returns the chosen knobs (with "ms" and "cached")."""
    h = matrix.handle
    key = _key(h, k, xtype, transpose)
    cache = _load(cache_path) if cache_path else {}
    if key in cache:
        knobs = {n: v for n, v in cache[key].items() if n in ("task_nnz", "task_rows", "long_row", "short_max",
                                                                "x_l2_policy")}
        _sp.spmm_replan(h, _sp.spmm_opts(**knobs), int(transpose))
        return dict(cache[key], cached=True)
    best, times, cands = _sp.spmm_autotune(h, k, xtype, int(transpose), candidates, reps)
    choice = dict(cands[best], ms=float(times[best]))
    if cache_path:
        cache = _load(cache_path)
        cache[key] = choice
        _save(cache_path, cache)
    return dict(choice, cached=False)


def tune_batched(matrices, Xs, Ys, candidates=None, reps=5, transpose=False) -> dict:
    """Put every matrix of a spmm_apply_batched call on the one plan that
    makes the whole batched call fastest.  A plan timed on one small graph
    alone measures launch latency, not its share of a shared launch, so the
    batch is timed as a whole: each candidate is applied to every handle
    (spmm_replan), the batched call runs once to warm up and `reps` times
    under CUDA events, and the handles are left on the fastest.  Returns the
    chosen knobs with "ms" and the time of every candidate."""
    import torch
    cands = list(candidates) if candidates is not None else list(_sp.BUILTIN_GRID)
    handles = [m.handle for m in matrices]
    times = []
    for c in cands:
        o = _sp.spmm_opts(**c)
        for h in handles:
            _sp.spmm_replan(h, o, int(transpose))
        _sp.spmm_apply_batched(handles, Xs, Ys, transpose)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            _sp.spmm_apply_batched(handles, Xs, Ys, transpose)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / reps)
    best = min(range(len(cands)), key=lambda i: times[i])
    o = _sp.spmm_opts(**cands[best])
    for h in handles:
        _sp.spmm_replan(h, o, int(transpose))
    return dict(cands[best], ms=times[best], candidate_ms=times)
