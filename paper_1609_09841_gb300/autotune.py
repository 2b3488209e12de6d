"""Autotuner of the fused kernel's schedule (tile shape x z-chunk).

For a plan and a pair of device states it times every compiled tile shape
(hermite_schedule_count) with each candidate z-chunk on the device (CUDA
events, after a warm-up launch), keeps the fastest, applies it to the plan
and caches it in a JSON file keyed by GPU name, order, precision, state type
and grid.  The tuning launches are real half steps of the caller's states
(their contents are overwritten).
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


BATCH_ZCHUNKS = ((8, 8, 8), (16, 16, 16), (32, 16, 8), (32, 32, 16), (64, 32, 16), (96, 48, 32))


def tune_batch(bplan, a, b, options=BATCH_ZCHUNKS, reps=2):
    """Pick and apply the fastest per-order z-chunks of a batched plan by
    timing `reps` batched half steps for each option; returns
    {"zchunk", "ms", "table"}."""
    import torch
    table = {}
    for zc in options:
        bplan.set_schedule(zc)
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
        table[zc] = e0.elapsed_time(e1) / reps
    best = min(table, key=table.get)
    bplan.set_schedule(best)
    return {"zchunk": list(best), "ms": table[best], "table": {str(k): v for k, v in table.items()}}
