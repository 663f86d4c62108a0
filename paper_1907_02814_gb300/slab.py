"""Positron yield of a Cu slab filled with Maxwell-Juttner fast electrons,
the foil study of Sec. IV (fig. confront_theo_simu_029) without fields.

The paper's slab is a 5-15 um Cu plasma (n_i = 8e22 cm^-3, Z* = 5) in a 1D3V
PIC code, where sheath fields confine the fast electrons and expand the
ions.  With no fields and perfect confinement the slab is uniform and the
isotropic electron population stays uniform, so where an electron or
positron sits does not change its collisions: the leptons and ions are held
in place, and only the photons are transported (straight lines at c,
removed when they leave the slab), because their path inside the slab sets
the Bethe-Heitler yield.  Every collision (Brems, Bethe-Heitler, Trident)
runs through pcc_collide on the batched FP32 path; the photon push here is a
field-free transport harness, not part of the collision method.

Yields are positrons per kJ of initial fast-electron kinetic energy after a
given time, split by the channel recorded in each secondary's identifier.
Collisional stopping (impact ionisation, elastic scattering) and the sheath
fields are not modelled, so the electrons keep radiating and the yields grow
with time instead of saturating as in the paper's runs.

    python -m paper_1907_02814_gb300.slab            # the 3 x 3 sweep
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import pcc
from . import workloads as W

C_LIGHT = 299792458.0
MEV_J = 1.602176634e-13
CH_TRIDENT = (2, 3)      # channel field of secondary ids: Trident by e- or e+ projectiles
CH_BH = 4                # Bethe-Heitler


def _live_flat(torch, sp):
    """Live particles of a DeviceSpecies as flat tensors (storage order)."""
    cnt = sp.cell_count.long()
    n = int(cnt.sum())
    first = torch.repeat_interleave(sp.cell_start[:-1].long(), cnt)
    run0 = torch.cumsum(cnt, 0) - cnt
    idx = first + (torch.arange(n, device=cnt.device) - torch.repeat_interleave(run0, cnt))
    cell = torch.repeat_interleave(torch.arange(cnt.numel(), device=cnt.device), cnt)
    return {"ux": sp.ux[idx], "uy": sp.uy[idx], "uz": sp.uz[idx], "w": sp.w[idx], "pid": sp.pid[idx],
            "x": sp.x[idx], "cell": cell, "n": n}


def _push_photons(torch, t, dt, dx, nx):
    """x += c n_x dt within the photon's column of nx cells; photons outside
    [0, nx dx) leave the slab."""
    k = torch.sqrt(t["ux"] * t["ux"] + t["uy"] * t["uy"] + t["uz"] * t["uz"])
    x = t["x"] + (t["ux"] / k) * float(C_LIGHT * dt)
    keep = (x >= 0.0) & (x < nx * dx)
    out = {f: t[f][keep] for f in ("ux", "uy", "uz", "w", "pid")}
    out["x"] = x[keep]
    col = t["cell"][keep] // nx
    ix = torch.clamp(torch.floor(out["x"] / dx).long(), 0, nx - 1)
    out["cell"] = (col * nx + ix).to(torch.int32)
    out["n"] = int(keep.sum())
    return out


def run_slab(ctx, torch, thickness_um, mean_kinetic_mev, time_ps=2.0, dt=1e-15, electrons=1 << 24, dx_um=0.25,
             e_per_cell=8192, photon_slack=1024, seed=6):
    """One slab run (``electrons`` fast electrons in columns of the slab with
    e_per_cell per cell); returns the positron yields per kJ by channel."""
    nx = int(round(thickness_um / dx_um))
    columns = max(1, electrons // (e_per_cell * nx))
    wl = W.cu_slab_mj(thickness_um, mean_kinetic_mev, e_per_cell=e_per_cell, dx_um=dx_um, columns=columns,
                      seed=seed, dt=dt)
    n_cells = wl.n_cells
    em0 = wl.species["em"]
    T = np.sqrt(1.0 + em0["ux"].astype(np.float64) ** 2 + em0["uy"] ** 2 + em0["uz"] ** 2) - 1.0
    energy_kj = float((em0["w"].astype(np.float64) * T).sum()) * W.MEC2_MEV * MEV_J / 1e3   # per unit slab volume x dx
    m = wl.materials[0]
    ctx.tables_build([pcc.material(m.Z, m.Zstar, m.n_i, m.T_e)], pcc.table_spec(cutoff_exp=2))
    dev = {}
    for name, d in wl.species.items():
        n = len(d["w"])
        slack = photon_slack if name == "ph" else 256
        sp = pcc.DeviceSpecies.empty(n_cells, n + (slack + 1) * n_cells, with_x=True)
        src = pcc.particles_to_device(d) if n else {
            "n": 0, "ux": None, "uy": None, "uz": None, "w": None, "pid": None, "cell": None,
            "x": torch.zeros(0, device="cuda")}
        pcc.bin(ctx, src, n_cells, sp, slack_abs=slack, slack_rel=0.0)
        dev[name] = sp
    mat = torch.zeros(n_cells, dtype=torch.int32, device="cuda")
    steps = int(round(time_ps * 1e-12 / dt))
    ctx.read_status()
    status = 0
    t0 = time.perf_counter()
    for s in range(steps):
        pcc.collide(ctx, n_cells, mat, wl.ion_mass, dev["em"], dev["ep"], dev["ph"], dev["ion"], dt, seed, s,
                    precision=pcc.FP32_BATCHED)
        for k in ("em", "ep", "ph"):
            pcc.append_secondaries(ctx, n_cells, dev[k])
        t = _push_photons(torch, _live_flat(torch, dev["ph"]), dt, wl.dx, nx)
        ph = pcc.DeviceSpecies.empty(n_cells, t["n"] + (photon_slack + 1) * n_cells, with_x=True)
        pcc.bin(ctx, t, n_cells, ph, slack_abs=photon_slack, slack_rel=0.0)
        dev["ph"] = ph
        if s % 200 == 199:
            status |= ctx.read_status()[0]
    status |= ctx.read_status()[0]
    torch.cuda.synchronize()
    elapsed = time.perf_counter() - t0
    ep = dev["ep"].live_host()
    ch = ((ep["pid"] >> np.uint64(41)) & np.uint64(7)).astype(np.int64)
    sec = (ep["pid"] >> np.uint64(63)) == 1
    w = ep["w"].astype(np.float64)
    bh, tri = sec & (ch == CH_BH), sec & np.isin(ch, CH_TRIDENT)
    return {"thickness_um": thickness_um, "mean_kinetic_mev": mean_kinetic_mev, "time_ps": time_ps, "dt_fs": dt * 1e15,
            "electrons": len(T), "cells": n_cells, "columns": columns, "steps": steps, "status": int(status),
            "bh_per_kj": float(w[bh].sum()) / energy_kj, "trident_per_kj": float(w[tri].sum()) / energy_kj,
            "bh_count": int(bh.sum()), "trident_count": int(tri.sum()), "seconds": elapsed}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--thickness", type=float, nargs="+", default=[5.0, 10.0, 15.0])
    ap.add_argument("--mean-mev", type=float, nargs="+", default=[1.0, 3.0, 10.0])
    ap.add_argument("--time-ps", type=float, default=2.0)
    ap.add_argument("--electrons", type=int, default=1 << 24)
    args = ap.parse_args()
    import torch
    from . import build
    build.build()
    ctx = pcc.Context(0)
    for l in args.thickness:
        for T in args.mean_mev:
            r = run_slab(ctx, torch, l, T, time_ps=args.time_ps, electrons=args.electrons)
            print(json.dumps(r), flush=True)
    ctx.close()


if __name__ == "__main__":
    main()
