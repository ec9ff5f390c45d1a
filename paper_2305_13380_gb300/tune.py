"""Autotuning of the cell geometry and work split of a pool: grid mode
(uniform cells or nested grids), cell margin over the largest support, the
leaf size n_leaf of the nested grids, and on the uniform grid the lanes per
target of the loops (threads per particle) and the force's pair evaluation
(gather, or each pair once with SPH_FLAG_SYMMETRIC).

Larger cells stage more candidates per target; smaller ones leave less room
for smoothing lengths to grow before a rebuild is needed; nested grids cost a
second sort but keep every target's neighbour cells near its own support.
The tuner times a few pool steps for each candidate and keeps the fastest;
results are cached in a JSON file keyed by GPU name and workload key.

Uniform cells are only tried when every simulation's starting smoothing
lengths span less than SPREAD_UNIFORM: on strongly clustered inputs a cell
sized by the widest particle holds thousands of the densest ones, and a single
step takes seconds."""
from __future__ import annotations

import json
import os

import numpy as np
import torch

from . import pool, sph

MARGINS = (0.03, 0.05, 0.1, 0.2)
LEAVES = (8, 16, 32)
LANES = (0, 2, 4)  # lanes per target on the uniform grid (0: automatic)
SPREAD_UNIFORM = 8.0
_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "tune_cache.json")


def _load():
    try:
        return json.load(open(_CACHE))
    except (OSError, ValueError):
        return {}


def candidates(sims) -> list[dict]:
    """Parameter overrides to try, nested grids first."""
    out = [dict(flags=sph.SPH_FLAG_TREE, cell_margin=m, n_leaf=k) for m in MARGINS for k in LEAVES]
    spread = max(float(np.max(s["h0"]) / np.min(s["h0"])) for s in sims)
    if spread < SPREAD_UNIFORM:
        out += [dict(flags=0, cell_margin=m, lanes_per_target=t) for m in MARGINS for t in LANES]
        # each force pair evaluated once (measured slower on this GPU; kept so
        # that the choice is measured per workload)
        out += [dict(flags=sph.SPH_FLAG_SYMMETRIC, cell_margin=0.05)]
    return out


def _time(sims, over: dict, steps: int, give_up_ms: float) -> float | None:
    P = pool.Pool(sims, sph.sph_default_params(**over))
    try:
        P.start()
    except sph.SPHError:
        return None  # these cells cannot hold the supports of some simulation
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(P.stream)
    P.step()
    e1.record(P.stream)
    P.stream.synchronize()
    first = e0.elapsed_time(e1)
    if P.status() or first > give_up_ms:
        return None
    e0.record(P.stream)
    for _ in range(steps):
        P.step()
    e1.record(P.stream)
    P.stream.synchronize()
    if P.status():
        return None
    return e0.elapsed_time(e1) / steps


def tune(sims, key: str, steps: int = 3) -> dict:
    """Times every candidate on a pool of `sims` (or takes the record of this
    GPU and `key` from the cache): {"best": overrides, "best_ms": ms,
    "default_ms": ms of the library's defaults on the same grid mode,
    "times": [[overrides, ms or None], ...]}."""
    name = torch.cuda.get_device_name()
    cache = _load()
    ck = f"{name}|{key}"
    rec = cache.get(ck)
    if isinstance(rec, dict) and "best" in rec:
        return rec
    best, best_ms, times = None, float("inf"), []
    for over in candidates(sims):
        ms = _time(sims, over, steps, give_up_ms=4.0 * best_ms)
        times.append([over, ms])
        if ms is not None and ms < best_ms:
            best, best_ms = over, ms
    if best is None:
        raise RuntimeError("no candidate cell geometry ran without a device status")
    # the defaults of the chosen grid mode (margin 0.05, n_leaf 16, automatic lanes)
    tree = bool(best.get("flags", 0) & sph.SPH_FLAG_TREE)
    dflt = [ms for o, ms in times if ms is not None and o.get("cell_margin") == 0.05 and
            (o.get("n_leaf") == 16 if tree else (o.get("flags", 0) == 0 and o.get("lanes_per_target", 0) == 0))
            and bool(o.get("flags", 0) & sph.SPH_FLAG_TREE) == tree]
    rec = {"best": best, "best_ms": best_ms, "default_ms": dflt[0] if dflt else None, "times": times}
    cache[ck] = rec
    os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
    with open(_CACHE, "w") as f:
        json.dump(cache, f, indent=1)
    return rec


def best_params(sims, key: str, steps: int = 3) -> dict:
    """The fastest parameter overrides (flags, cell_margin, n_leaf,
    lanes_per_target) for a pool of `sims`, from the cache when this GPU has
    seen `key`."""
    return dict(tune(sims, key, steps)["best"])


def partition(sims) -> list[list[int]]:
    """Indices of the simulations whose starting smoothing lengths span less
    than SPREAD_UNIFORM (candidates for the uniform grid), then of the rest
    (nested grids only); empty parts are dropped."""
    spread = [float(np.max(s["h0"]) / np.min(s["h0"])) for s in sims]
    parts = [[i for i, v in enumerate(spread) if v < SPREAD_UNIFORM],
             [i for i, v in enumerate(spread) if v >= SPREAD_UNIFORM]]
    return [p for p in parts if p]


def best_split(sims, key: str, steps: int = 3) -> list[tuple[list[int], dict]]:
    """The simulations split by partition(), each part with its own tuned
    parameter overrides (cached per part)."""
    out = []
    for k, idx in enumerate(partition(sims)):
        part = [sims[i] for i in idx]
        out.append((idx, best_params(part, key=f"{key}|part{k}-{len(idx)}", steps=steps)))
    return out

