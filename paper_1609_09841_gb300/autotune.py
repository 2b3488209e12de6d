"""Autotuner of the kernels' schedules (tile shape x z-chunk).

``tune``: for a single plan and a pair of device states it times every
compiled tile shape (hermite_schedule_count) with each candidate z-chunk on
the device (CUDA events, after a warm-up launch), keeps the fastest, applies
it to the plan and caches it in a JSON file keyed by GPU name, order,
precision, state type and grid.

``tune_batch``: for a batched plan it picks a tile shape and a z-chunk per
order (the per-m schedules of the one persistent launch).

The tuning launches are real half steps of the caller's states (their
contents are overwritten).
"""
import json
import os

from . import capi

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "hermite_gb300", "autotune.json")
ZCHUNKS = (8, 16, 32, 64)


def _key(plan, device_name):
    return f"{device_name}|m={plan.m}|{plan.prec}|{plan.state}|{plan.variant}|{plan.grid}"


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def tune(plan, x, y, zchunks=ZCHUNKS, reps=2, cache=DEFAULT_CACHE, force=False):
    """Pick and apply the fastest (tile, zchunk) for `plan`; returns
    {"tile", "zchunk", "ms", "table"} (table: every timing, ms per step)."""
    import torch
    name = torch.cuda.get_device_name()
    key = _key(plan, name)
    db = _load(cache) if cache else {}
    if not force and key in db:
        best = db[key]
        capi.check(capi.lib.hermite_set_schedule(plan.handle, best["tile"], best["zchunk"]))
        return best
    table = {}
    for tile in range(capi.lib.hermite_schedule_count(plan.handle)):
        for zc in zchunks:
            capi.check(capi.lib.hermite_set_schedule(plan.handle, tile, zc))
            plan.step(x, y, 0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for r in range(reps):
                plan.step(x, y, r % 2) if r % 2 == 0 else plan.step(y, x, 1)
            e1.record()
            torch.cuda.synchronize()
            table[f"{tile}/{zc}"] = e0.elapsed_time(e1) / reps
    best_key = min(table, key=table.get)
    tile, zc = (int(v) for v in best_key.split("/"))
    capi.check(capi.lib.hermite_set_schedule(plan.handle, tile, zc))
    best = {"tile": tile, "zchunk": zc, "ms": table[best_key], "table": table}
    if cache:
        db[key] = best
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        tmp = cache + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(db, fh, indent=1)
        os.replace(tmp, cache)
    return best


BATCH_ZCHUNKS = (8, 16, 32, 48, 64, 96)
BATCH_TILES = (0, 1)
# whole z-chunk triples (orders 1, 2, 3) timed first; the search starts from the fastest
BATCH_STARTS = ((8, 8, 8), (16, 16, 16), (32, 16, 8), (32, 32, 16), (64, 32, 16), (96, 48, 32))


def _time_batch(bplan, a, b, reps):
    import torch
    bplan.step(a, b, 0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for r in range(reps):
        if r % 2 == 0:
            bplan.step(a, b, 0)
        else:
            bplan.step(b, a, 1)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_batch(bplan, a, b, zchunks=BATCH_ZCHUNKS, tiles=BATCH_TILES, starts=BATCH_STARTS, reps=3, sweeps=2,
               timer=None):
    """Pick and apply the fastest tile shape x z-chunk of every order present
    in a batched plan.  The orders share one persistent launch, so they are
    tuned by coordinate search: from the fastest of the whole z-chunk triples
    `starts` (first tile shapes), each order in turn (heaviest first) has every
    (tile, zchunk) pair timed with the other orders held at their current
    choice, and keeps the fastest; `sweeps` passes over the orders.  Timing:
    `reps` batched half steps after a warm-up one (CUDA events), or
    timer(bplan) if given.  Returns {"tile", "zchunk" (per order 1..3), "ms",
    "table" (every timing)}."""
    if timer is None:
        def timer(p):
            return _time_batch(p, a, b, reps)
    orders = sorted({s["m"] for s in bplan.sims}, reverse=True)
    tile = [0, 0, 0]
    bplan.set_tiles(tile)
    table = {}
    best_ms, zc = None, None
    for z3 in starts:
        bplan.set_schedule(z3)
        ms = timer(bplan)
        table[f"start {list(z3)}"] = ms
        if best_ms is None or ms < best_ms:
            best_ms, zc = ms, list(z3)
    for sweep in range(sweeps):
        for m in orders:
            choice = (tile[m - 1], zc[m - 1])
            for t in tiles:
                for z in zchunks:
                    if (t, z) == choice:
                        continue
                    tt, zz = list(tile), list(zc)
                    tt[m - 1], zz[m - 1] = t, z
                    bplan.set_tiles(tt)
                    bplan.set_schedule(zz)
                    ms = timer(bplan)
                    table[f"sweep {sweep} m={m} tile={t} zchunk={z}"] = ms
                    if ms < best_ms:
                        best_ms, choice = ms, (t, z)
            tile[m - 1], zc[m - 1] = choice
    bplan.set_tiles(tile)
    bplan.set_schedule(zc)
    return {"tile": tile, "zchunk": zc, "ms": best_ms, "table": table}
