"""Launch-schedule autotuner of the batched collision kernels.

The speed of the batched electron-ion step depends on two choices that the
best value of shifts with the occupancy distribution of the cells:

  * the register budget of the scan kernel, compiled for a minimum of 2 to
    6 resident blocks per SM (more registers per thread against more warps
    to hide memory latency);
  * the persistent grid, as blocks per SM (0 = as many as fit).

``tune`` times every candidate on a scratch copy of the caller's particle
state (a collision step changes that state) with CUDA events, keeps the
fastest, applies it to the context and stores it in a JSON cache keyed by
device and workload shape, so that later runs on the same shape skip the
search.  All timed work runs in the library's kernels.
"""
from __future__ import annotations

import json
import os

CANDIDATES = ((4, 0), (5, 0), (6, 0), (3, 0), (2, 0), (4, 3), (5, 4))


def default_cache_path() -> str:
    return os.environ.get("PCC_TUNE_CACHE",
                          os.path.join(os.path.dirname(os.path.abspath(__file__)), ".tune_cache.json"))


def shape_key(torch, n_cells: int, live: dict) -> str:
    name = torch.cuda.get_device_name()
    parts = "|".join(f"{k}={live[k]}" for k in sorted(live))
    return f"{name}|cells={n_cells}|{parts}"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, cache):
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _scratch_copy(pcc, sp):
    c = lambda t: None if t is None else t.clone()
    return pcc.DeviceSpecies(c(sp.ux), c(sp.uy), c(sp.uz), c(sp.w), c(sp.pid), c(sp.cell_start), c(sp.cell_count),
                             c(sp.cell_added), c(sp.x))


def tune(ctx, pcc, torch, n_cells, material_of_cell, ion_mass, species: dict, dt, seed, step=0,
         precision=None, cache_path=None, reps=3, candidates=CANDIDATES, use_cache=True):
    """Choose (min_blocks_per_sm, blocks_per_sm) for the electron-ion launch
    and apply it with ``ctx.set_schedule``.  ``species`` maps em, ep, ph, ion
    to DeviceSpecies.  Returns {"schedule": (m, b), "ms": {...}, "cached": bool}."""
    precision = pcc.FP32_BATCHED if precision is None else precision
    live = {k: int(v.cell_count.sum().item()) for k, v in species.items()}
    key = shape_key(torch, n_cells, live)
    path = cache_path or default_cache_path()
    cache = _load(path) if use_cache else {}
    if key in cache:
        m, b = cache[key]["schedule"]
        ctx.set_schedule(m, b)
        return {"schedule": (m, b), "ms": cache[key].get("ms", {}), "cached": True}

    work = {k: _scratch_copy(pcc, v) for k, v in species.items()}
    stream = torch.cuda.current_stream()
    mask = pcc.BREMS | pcc.TRIDENT | pcc.GROUP_EM
    timings = {}
    for m, b in candidates:
        ctx.set_schedule(m, b)
        ms = []
        for r in range(reps + 1):
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            pcc.collide(ctx, n_cells, material_of_cell, ion_mass, work["em"], work["ep"], work["ph"], work["ion"],
                        dt, seed, step + r, mask=mask, precision=precision)
            t1.record(stream)
            for k in ("em", "ep", "ph"):
                work[k].cell_added.zero_()      # drop this trial's secondaries
            torch.cuda.synchronize()
            if r > 0:                            # the first run warms the variant
                ms.append(t0.elapsed_time(t1))
        ms.sort()
        timings[f"{m},{b}"] = ms[len(ms) // 2]
    best = min(timings, key=timings.get)
    m, b = (int(v) for v in best.split(","))
    ctx.set_schedule(m, b)
    ctx.read_status()                            # clear the trial counters
    del work
    if use_cache:
        cache[key] = {"schedule": [m, b], "ms": timings}
        try:
            _store(path, cache)
        except OSError:
            pass
    return {"schedule": (m, b), "ms": timings, "cached": False}
