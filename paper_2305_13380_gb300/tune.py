"""Autotuning of the cell size (the cell margin over the largest support).

Larger cells stage more candidates per target; smaller ones leave less room
for smoothing lengths to grow before a rebuild is needed.  The tuner times a
few pool steps for each candidate margin and keeps the fastest; results are
cached in a JSON file keyed by GPU name and workload key."""
from __future__ import annotations

import json
import os

import torch

from . import pool, sph

CANDIDATES = (0.03, 0.05, 0.1, 0.2)
_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "tune_cache.json")


def _load():
    try:
        return json.load(open(_CACHE))
    except (OSError, ValueError):
        return {}


def best_margin(sims, key: str, steps: int = 3, candidates=CANDIDATES) -> float:
    name = torch.cuda.get_device_name()
    cache = _load()
    ck = f"{name}|{key}"
    if ck in cache:
        return float(cache[ck])
    best, best_ms = candidates[0], float("inf")
    for m in candidates:
        P = pool.Pool(sims, sph.sph_default_params(cell_margin=m))
        try:
            P.start()
        except sph.SPHError:
            continue  # this margin cannot hold the supports of some simulation
        P.step()
        P.stream.synchronize()
        if P.status():
            continue
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(P.stream)
        for _ in range(steps):
            P.step()
        e1.record(P.stream)
        P.stream.synchronize()
        ms = e0.elapsed_time(e1) / steps
        if P.status() == 0 and ms < best_ms:
            best, best_ms = m, ms
        del P
    cache[ck] = best
    os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
    with open(_CACHE, "w") as f:
        json.dump(cache, f, indent=1)
    return best
