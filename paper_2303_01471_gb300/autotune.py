"""Autotuner of the batched persistent launch (qhd_group_*).

The launch has three choices that change its speed but not its results'
accuracy bound: how many CTAs hold one instance (the split N = C * R of the
distributed axis: C CTAs of R rows, which also sets the cross-CTA DFT size and
the local row-transform batch), how many CTAs per SM the kernel is compiled for
(registers versus resident warps), and how many persistent clusters are
launched.  tune_group() times every candidate on the caller's own contexts with
CUDA events over a short evolution and keeps the fastest; the choice is cached
in a JSON file per (GPU, SM count, library build, mesh edges and batch sizes),
so a later run starts from it without timing.

Timing evolves the contexts: reset their states afterwards.
"""
from __future__ import annotations

import hashlib
import itertools
import json
import os
from typing import Dict, List, Optional

from . import build as _build
from . import qhd

CACHE_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tune")
CACHE_FILE = os.path.join(CACHE_DIR, "group.json")

# CTAs per instance allowed for each mesh edge (the engine holds at most 32 rows per CTA)
SUB_CHOICES = {64: (2, 4, 8), 128: (4, 8), 256: (8,)}
EDGE_SLOT = {64: 0, 128: 1, 256: 2}


def _library_id() -> str:
    h = hashlib.sha256()
    with open(_build.LIB, "rb") as fh:
        h.update(fh.read())
    return h.hexdigest()[:16]


def cache_key(sims) -> str:
    import torch
    p = torch.cuda.get_device_properties(sims[0].device)
    shapes = sorted((s.shape[0], s.batch) for s in sims)
    return f"{p.name}|{p.multi_processor_count}|{_library_id()}|{shapes}"


def candidates(sims) -> List[qhd.GroupConfig]:
    edges = sorted({s.shape[0] for s in sims})
    per_edge = [SUB_CHOICES[e] for e in edges]
    out = []
    for subs in itertools.product(*per_edge):
        sub = [0, 0, 0]
        for e, c in zip(edges, subs):
            sub[EDGE_SLOT[e]] = c
        for mb in (1, 2):
            out.append(qhd.GroupConfig.make(sub, mb, 0))
    return out


def time_config(sims, cfg: qhd.GroupConfig, T: float, dt: float, reps: int = 2) -> float:
    """Device time (ms) of one group evolution of T, best of `reps` after a warm-up."""
    import torch
    grp = qhd.Group(sims, cfg)
    try:
        best = float("inf")
        for r in range(reps + 1):
            for s in sims:
                s.reset_state()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(sims[0].stream)
            grp.evolve(T, dt)
            e1.record(sims[0].stream)
            e1.synchronize()
            if grp.status() != qhd.QHD_OK:
                raise qhd.QHDError(5, "group wait timed out while tuning")
            if r > 0:
                best = min(best, e0.elapsed_time(e1))
        return best
    finally:
        grp.close()


def tune_group(sims, T: float = 1.0, dt: float = 0.01, use_cache: bool = True,
               cache_file: Optional[str] = None) -> Dict:
    """Pick the fastest launch configuration for this group of contexts.
    Returns {"config": GroupConfig, "ms": timings per candidate, "cached": bool}."""
    cache_file = cache_file or CACHE_FILE
    key = cache_key(sims)
    cache = {}
    if use_cache and os.path.exists(cache_file):
        try:
            with open(cache_file) as fh:
                cache = json.load(fh)
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache:
        c = cache[key]["config"]
        return {"config": qhd.GroupConfig.make(c["sub"], c["min_blocks"], c["clusters"]),
                "ms": cache[key]["ms"], "cached": True}
    timings = []
    for cfg in candidates(sims):
        ms = time_config(sims, cfg, T, dt)
        timings.append((ms, cfg))
    timings.sort(key=lambda x: x[0])
    best = timings[0][1]
    entry = {"config": best.as_dict(), "ms": [[m, c.as_dict()] for m, c in timings],
             "probe": {"T": T, "dt": dt}}
    cache[key] = entry
    os.makedirs(os.path.dirname(cache_file), exist_ok=True)
    tmp = cache_file + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1)
    os.replace(tmp, cache_file)
    return {"config": best, "ms": entry["ms"], "cached": False}
