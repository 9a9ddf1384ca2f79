"""Self-written autotuner for the batched MUCA sweep launch (a8).

Knobs:
  * chains per tile for each lattice size (muca_set_tile_width): 32, or the narrow width that
    brings the acceptance thresholds into shared memory (16 at L = 7, 8; in the colour order also
    8 at L = 9, 10 and 4 at L = 11, 12).  A narrow tile runs each of
    its chains faster but holds half as many, so it wins when the batch is smaller than what the
    GPU can hold and loses when tiles queue for SMs;
  * the persistent work-queue grid vs one block per tile, and the resident blocks per SM of the
    persistent grid (chains are latency-bound, so tiles sharing an SM sub-partition slow each
    other down);
  * sweeps per launch.
In the colour order (muca_set_sweep_order) the even-L chains run in their own kernel, one block
per tile: there only the tile width is tuned.  The order itself is the caller's choice (it changes
the trajectories), never the tuner's.
A candidate is timed with CUDA events on a scratch context with the same composition of chains
(same dim, L and chain counts, a different seed), so tuning never advances the caller's chains,
whose results do not depend on the choice anyway.  The winner is cached in a JSON file keyed by
the GPU name and the composition.  Tile widths fix the layout, so they are chosen before the
caller's chains are created: tune() first, then prepare(ctx, best) before ea_init_disorder and
launch(ctx, best) after it (apply() does the last two for a context that has no chains yet).
"""
from __future__ import annotations

import itertools
import json
import os
from pathlib import Path

from . import eamc
from .build import BUILD

CACHE = BUILD / "autotune.json"
LAUNCHES = [
    {"persistent": False, "blocks_per_sm": 0, "sweeps_per_launch": 0},
    {"persistent": True, "blocks_per_sm": 1, "sweeps_per_launch": 0},
    {"persistent": True, "blocks_per_sm": 2, "sweeps_per_launch": 0},
    {"persistent": True, "blocks_per_sm": 0, "sweeps_per_launch": 0},
    {"persistent": True, "blocks_per_sm": 2, "sweeps_per_launch": 64},
]


def signature(groups) -> str:
    """groups: list of (dim, L, n_chains)."""
    return ";".join(f"{d}x{L}x{n}" for d, L, n in groups)


# above this many width assignments the tuner searches in stages instead of trying them all
MAX_WIDTH_COMBOS = 12


def width_options(groups, order: int = 0):
    """Tile-width assignments: every L at 32, and each L that has narrow widths at each of them
    (all combinations; tune() searches in stages when there are more than MAX_WIDTH_COMBOS)."""
    narrow = sorted({(d, L) for d, L, _ in groups if eamc.narrow_widths(d, L, order)})
    choices = [[32] + eamc.narrow_widths(d, L, order) for d, L in narrow]
    out = []
    for pick in itertools.product(*choices):
        out.append({str(L): w for (d, L), w in zip(narrow, pick) if w != 32})
    return out


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


def tune(groups, sweeps: int = 40, repeats: int = 2, use_cache: bool = True, device: int = 0,
         order: int = 0):
    """Returns the fastest configuration for this composition of chains in sweep order `order`:
    {"widths": {L: width}, "persistent", "blocks_per_sm", "sweeps_per_launch"}."""
    import torch
    key = f"{torch.cuda.get_device_name(device)}|{signature(groups)}|{sweeps}|order{order}"
    launches = LAUNCHES if order == 0 else LAUNCHES[:1]
    db = _load() if use_cache else {}
    if key in db:
        return db[key]["best"]
    stream = torch.cuda.Stream(device=device)
    results = []

    def trial(widths):
        ctx = eamc.Context(seed=0x5EED, device=device, stream=stream.cuda_stream)
        ctx.set_sweep_order(order)
        for L, w in widths.items():
            ctx.set_tile_width(int(L), w)
        rid = 0
        for dim, L, n in groups:
            ctx.init_disorder(dim, L, n, rid0=rid)
            rid += n
        for cand in launches:
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
            results.append({"widths": widths, **cand, "ms": best})
        ctx.close()
        return min(r["ms"] for r in results if r["widths"] == widths)

    combos = width_options(groups, order)
    if len(combos) <= MAX_WIDTH_COMBOS:
        for widths in combos:
            trial(widths)
    else:
        # staged: every size's narrow widths alone (the others in full tiles), then the sizes'
        # winners together
        base = trial({})
        pick = {}
        for d, L in sorted({(d, L) for d, L, _ in groups if eamc.narrow_widths(d, L, order)}):
            best_ms = base
            for w in eamc.narrow_widths(d, L, order):
                ms = trial({str(L): w})
                if ms < best_ms:
                    best_ms, pick[str(L)] = ms, w
        if len(pick) > 1:
            trial(dict(pick))
    winner = min(results, key=lambda r: r["ms"])
    best = {k: winner[k] for k in ("widths", "persistent", "blocks_per_sm", "sweeps_per_launch")}
    if use_cache:
        db[key] = {"best": best, "trials": results}
        _store(db)
    return best


def prepare(ctx: "eamc.Context", best):
    """Tile widths of the chosen configuration (before the chains are created)."""
    for L, w in best.get("widths", {}).items():
        ctx.set_tile_width(int(L), int(w))


def launch(ctx: "eamc.Context", best):
    ctx.set_launch(best["persistent"], best["sweeps_per_launch"], best["blocks_per_sm"])


def apply(ctx: "eamc.Context", groups, **kw):
    """Tunes for `groups` and configures ctx, which must not hold chains yet."""
    best = tune(groups, **kw)
    prepare(ctx, best)
    launch(ctx, best)
    return best
