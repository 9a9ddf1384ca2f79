"""Self-written autotuner for the batched MUCA sweep launch (a8).

The knobs are the ones muca_set_launch exposes: persistent work-queue grid vs one block per
tile, the number of resident blocks per SM of the persistent grid (chains are latency-bound,
so tiles sharing an SM sub-partition slow each other down), and sweeps per launch.  A
candidate is timed with CUDA events on a scratch context with the same composition of tiles
(same dim, L and chain counts, a different seed), so tuning never advances the caller's
chains, whose results do not depend on the choice anyway.  The winner is cached in a JSON
file keyed by the GPU name and the composition.
"""
from __future__ import annotations

import json
import os
from pathlib import Path

from . import eamc
from .build import BUILD

CACHE = BUILD / "autotune.json"
CANDIDATES = [
    {"persistent": False, "blocks_per_sm": 0, "sweeps_per_launch": 0},
    {"persistent": True, "blocks_per_sm": 1, "sweeps_per_launch": 0},
    {"persistent": True, "blocks_per_sm": 2, "sweeps_per_launch": 0},
    {"persistent": True, "blocks_per_sm": 0, "sweeps_per_launch": 0},
    {"persistent": True, "blocks_per_sm": 2, "sweeps_per_launch": 64},
]


def signature(groups) -> str:
    """groups: list of (dim, L, n_chains)."""
    return ";".join(f"{d}x{L}x{n}" for d, L, n in groups)


def _load():
    try:
        return json.loads(CACHE.read_text())
    except Exception:
        return {}


def _store(db):
    CACHE.parent.mkdir(parents=True, exist_ok=True)
    tmp = CACHE.with_suffix(f".{os.getpid()}.tmp")
    tmp.write_text(json.dumps(db, indent=1, sort_keys=True))
    os.replace(tmp, CACHE)


def tune(groups, sweeps: int = 40, repeats: int = 2, use_cache: bool = True, device: int = 0):
    """Returns the fastest launch configuration for this composition of tiles."""
    import torch
    key = f"{torch.cuda.get_device_name(device)}|{signature(groups)}|{sweeps}"
    db = _load() if use_cache else {}
    if key in db:
        return db[key]["best"]
    stream = torch.cuda.Stream(device=device)
    ctx = eamc.Context(seed=0x5EED, device=device, stream=stream.cuda_stream)
    rid = 0
    for dim, L, n in groups:
        ctx.init_disorder(dim, L, n, rid0=rid)
        rid += n
    results = []
    for cand in CANDIDATES:
        ctx.set_launch(cand["persistent"], cand["sweeps_per_launch"], cand["blocks_per_sm"])
        ctx.run_sweeps(max(2, sweeps // 8))  # warm-up
        best = None
        for _ in range(repeats):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.run_sweeps(sweeps)
            e1.record(stream)
            stream.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        results.append({**cand, "ms": best})
    ctx.close()
    winner = min(results, key=lambda r: r["ms"])
    best = {k: winner[k] for k in ("persistent", "blocks_per_sm", "sweeps_per_launch")}
    if use_cache:
        db[key] = {"best": best, "trials": results}
        _store(db)
    return best


def apply(ctx: "eamc.Context", groups, **kw):
    best = tune(groups, **kw)
    ctx.set_launch(best["persistent"], best["sweeps_per_launch"], best["blocks_per_sm"])
    return best
