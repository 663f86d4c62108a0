"""Launch-schedule autotuner of the batched collision kernels.

The speed of the batched step depends on choices whose best value shifts
with the occupancy distribution of the cells:

  * the register budget of the scan kernel, compiled for a minimum of 2 to
    6 resident blocks per SM (more registers per thread against more warps
    to hide memory latency);
  * the persistent grid, as blocks per SM (0 = as many as fit);
  * per species group, the size classes at which the scan gives a cell a
    whole warp or a group of 16, 8, 4 or 2 lanes (pcc_set_scan_classes): a
    narrow group wastes fewer lanes on a small cell, but a warp runs its
    groups to the largest trip count among them.

``tune`` times candidates on a scratch copy of the caller's particle state
(a collision step changes that state) with CUDA events: every register
budget and grid cap for the electron-ion group, then a coordinate descent
over the four class thresholds of the electron and photon groups (steps of
one and two half-octave classes, kept when 1 % faster).  It applies the
fastest setting to the context and stores it in a JSON cache keyed by device
and workload shape, so that later runs on the same shape skip the search.
All timed work runs in the library's kernels.
"""
from __future__ import annotations

import json
import os

CANDIDATES = ((4, 0), (5, 0), (6, 0), (3, 0), (2, 0), (4, 3), (5, 4))
N_CLASSES = 34                 # size classes of the scan, two per octave
CLASS_MOVES = (-2, -1, 1, 2)   # threshold steps tried by the descent
CLASS_GROUPS = (0, 2)          # electrons and photons (positrons are few)


def valid_classes(t) -> bool:
    """Thresholds {warp, g16, g8, g4} the library accepts."""
    return len(t) == 4 and 0 <= t[3] <= t[2] <= t[1] <= t[0] <= N_CLASSES


def descend(start, cost, moves=CLASS_MOVES, gain=0.01, sweeps=2):
    """Coordinate descent over integer thresholds: from `start`, try each
    coordinate moved by each step in `moves`, keep a move that lowers
    cost() by more than the fraction `gain`, repeat up to `sweeps` times.
    Returns (best thresholds, best cost, every cost measured)."""
    best = list(start)
    c_best = cost(best)
    seen = {tuple(best): c_best}
    for _ in range(sweeps):
        improved = False
        for i in range(len(best)):
            for d in moves:
                cand = list(best)
                cand[i] += d
                if not valid_classes(cand) or tuple(cand) in seen:
                    continue
                c = cost(cand)
                seen[tuple(cand)] = c
                if c < c_best * (1.0 - gain):
                    best, c_best, improved = cand, c, True
        if not improved:
            break
    return best, c_best, seen


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
         precision=None, cache_path=None, reps=3, candidates=CANDIDATES, use_cache=True, classes=True):
    """Choose (min_blocks_per_sm, blocks_per_sm) for the electron-ion launch
    and, with ``classes``, the scan-class thresholds of the electron and
    photon groups; apply them to ``ctx``.  ``species`` maps em, ep, ph, ion
    to DeviceSpecies.  Returns {"schedule": (m, b), "classes": {group:
    thresholds}, "ms": {...}, "cached": bool}."""
    precision = pcc.FP32_BATCHED if precision is None else precision
    live = {k: int(v.cell_count.sum().item()) for k, v in species.items()}
    key = shape_key(torch, n_cells, live)
    path = cache_path or default_cache_path()
    cache = _load(path) if use_cache else {}
    if key in cache:
        m, b = cache[key]["schedule"]
        ctx.set_schedule(m, b)
        cls = {int(g): list(t) for g, t in cache[key].get("classes", {}).items()}
        for g, t in cls.items():
            ctx.set_scan_classes(g, t)
        return {"schedule": (m, b), "classes": cls, "ms": cache[key].get("ms", {}), "cached": True}

    work = {k: _scratch_copy(pcc, v) for k, v in species.items()}
    stream = torch.cuda.current_stream()

    def timed(mask):
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
        return ms[len(ms) // 2]

    mask_em = pcc.BREMS | pcc.TRIDENT | pcc.GROUP_EM
    timings = {}
    for m, b in candidates:
        ctx.set_schedule(m, b)
        timings[f"{m},{b}"] = timed(mask_em)
    best = min(timings, key=timings.get)
    m, b = (int(v) for v in best.split(","))
    ctx.set_schedule(m, b)
    chosen = {}
    if classes:
        group_mask = {0: mask_em, 2: pcc.BH | pcc.GROUP_PH}
        for g in CLASS_GROUPS:
            def cost(t, g=g):
                ctx.set_scan_classes(g, t)
                return timed(group_mask[g])
            start = ctx.scan_classes(g)
            t_best, c_best, seen = descend(start, cost)
            ctx.set_scan_classes(g, t_best)
            chosen[g] = t_best
            timings[f"classes{g}:{start}"] = seen[tuple(start)]
            timings[f"classes{g}:{t_best}"] = c_best
    ctx.read_status()                            # clear the trial counters
    del work
    if use_cache:
        cache[key] = {"schedule": [m, b], "classes": {str(g): t for g, t in chosen.items()}, "ms": timings}
        try:
            _store(path, cache)
        except OSError:
            pass
    return {"schedule": (m, b), "classes": chosen, "ms": timings, "cached": False}
