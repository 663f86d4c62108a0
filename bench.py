#!/usr/bin/env python3
"""Benchmark of the pairwise collision step (Brems + Trident + Bethe-Heitler)
on the batched uneven-cell workload: 2^20 solid-Cu cells, log-normal electron
occupancy (median 64, sigma 1.5, capped at 8192; about 2.0e8 electrons),
3e7 ions, 0.25 N_e photons, dt = 1 fs, FP32 state.

One step = collide (electron-ion, positron-ion, photon-ion kernels) + commit
of the secondaries of the three species.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|fp64]
  python bench.py --impl reference     # the CPU oracle on a bounded sample
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = "batched_cu_1048576cells_lognormal_median64_sigma1.5_cap8192_dt1fs"
METRIC = "collision pairs/s"
UNIT = "pairs/s"
FALLBACK_HBM = 6800.0


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM, "fallback"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1907_02814_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".h")):
            h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel_tag):
    """Per-launch DRAM bytes from the committed ncu summary, if it was taken
    on the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", f"{kernel_tag}.txt")
    if not os.path.exists(p):
        return None
    vals = {}
    for line in open(p):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_hash") != source_hash():
        return None
    try:
        return float(vals["dram_bytes_per_launch_full_workload"])
    except (KeyError, ValueError):
        return None


# ------------------------------------------------------------------ setup --
def setup(ctx, pcc, W, torch, counts, slack):
    mat = counts["material"]
    ctx.tables_build([pcc.material(mat.Z, mat.Zstar, mat.n_i, mat.T_e)], pcc.table_spec())
    parts = W.batched_cu_device(counts, device="cuda")
    n_cells = len(counts["e"])
    dev = {}
    for name in ("em", "ion", "ph"):
        p = parts[name]
        sa, sr = slack[name]
        cap = int(p["n"] + sa * n_cells + int(np.ceil(sr * p["n"])) + n_cells)
        sp = pcc.DeviceSpecies.empty(n_cells, cap)
        pcc.bin(ctx, p, n_cells, sp, slack_abs=sa, slack_rel=sr)
        dev[name] = sp
        del parts[name]
    sa, sr = slack["ep"]
    dev["ep"] = pcc.DeviceSpecies.empty(n_cells, sa * n_cells)
    pcc.bin(ctx, {"n": 0, "ux": None, "uy": None, "uz": None, "w": None, "pid": None, "cell": None}, n_cells,
            dev["ep"], slack_abs=sa, slack_rel=sr)
    torch.cuda.synchronize()
    return dev


def live_counts(dev, torch):
    return {k: int(v.cell_count.sum().item()) for k, v in dev.items()}


def ei_pairs_and_bytes(dev, torch):
    """Pairs and algorithmic bytes of the electron-ion launch: 16 B per
    projectile and per target record of every cell with both, plus 20 B of
    per-cell metadata (starts, counts, material)."""
    ce = dev["em"].cell_count.long()
    ci = dev["ion"].cell_count.long()
    both = (ce > 0) & (ci > 0)
    pairs = int(torch.where(both, torch.maximum(ce, ci), torch.zeros_like(ce)).sum().item())
    recs = int((ce[both].sum() + ci[both].sum()).item())
    n_cells = ce.numel()
    return pairs, 16 * recs + 20 * n_cells


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_1907_02814_gb300 import build, pcc
    from paper_1907_02814_gb300 import workloads as W

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    pcc.load()
    ctx = pcc.Context(local)
    counts = W.batched_cu(seed=3 + rank)
    n_cells = len(counts["e"])
    slack = {"em": (4, 0.02), "ep": (6, 0.0), "ph": (8, 0.05), "ion": (0, 0.0)}
    dev = setup(ctx, pcc, W, torch, counts, slack)
    mat_of_cell = torch.zeros(n_cells, dtype=torch.int32, device="cuda")
    ledger = torch.zeros((n_cells, 4), dtype=torch.float32, device="cuda")
    prec = pcc.FP32_BATCHED if args.precision == "fp32" else pcc.FP64_PLAIN
    stream = torch.cuda.current_stream()
    dt, seed = counts["dt"], counts["seed"]
    ion_mass = counts["ion_mass"]
    launches_per_step = 6

    def step(s, ev=None):
        if ev is not None:
            ev[0].record(stream)
        pcc.collide(ctx, n_cells, mat_of_cell, ion_mass, dev["em"], dev["ep"], dev["ph"], dev["ion"], dt, seed, s,
                    mask=pcc.BREMS | pcc.TRIDENT | pcc.GROUP_EM, precision=prec, ledger=ledger)
        if ev is not None:
            ev[1].record(stream)
        pcc.collide(ctx, n_cells, mat_of_cell, ion_mass, dev["em"], dev["ep"], dev["ph"], dev["ion"], dt, seed, s,
                    mask=pcc.BREMS | pcc.TRIDENT | pcc.BH | pcc.GROUP_EP | pcc.GROUP_PH, precision=prec,
                    ledger=ledger)
        for k in ("em", "ep", "ph"):
            pcc.append_secondaries(ctx, n_cells, dev[k])

    for s in range(args.warmup):
        step(s)
    torch.cuda.synchronize()
    ctx.read_status()
    pairs_ei, bytes_ei = ei_pairs_and_bytes(dev, torch)
    before = live_counts(dev, torch)

    clocks = ClockSampler(local)
    clocks.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    start.record(stream)
    for s in range(args.steps):
        step(args.warmup + s, evs[s])
    end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = start.elapsed_time(end)
    ei_ms = [a.elapsed_time(b) for a, b in evs]
    status, stats = ctx.read_status()
    pairs = sum(stats["pairs"])
    events = sum(stats["created"])
    t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    tot = torch.tensor([pairs, events], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    ms_max = float(t.item())
    pairs_all, events_all = float(tot[0].item()), float(tot[1].item())

    # end-to-end through the C ABI with host buffers
    e2e = e2e_measure(args, ctx, pcc, torch, dev, n_cells, mat_of_cell, ion_mass, dt, seed, prec)

    peak, peak_kind = peaks()
    ei_avg = float(np.mean(ei_ms))
    achieved = bytes_ei / (ei_avg * 1e-3) / 1e9
    traffic = profiled_traffic("collide_ei_batched" if prec == pcc.FP32_BATCHED else "collide_ei_plain")
    result = {
        "metric": METRIC, "value": pairs_all / (ms_max * 1e-3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if prec == pcc.FP32_BATCHED else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells": n_cells, "electrons": before["em"], "ions": before["ion"],
                   "photons": before["ph"], "positrons": before["ep"], "precision": args.precision,
                   "l2": "inputs larger than L2 (about 6 GB of particle records per step)",
                   "parallelism": f"replicas{world}"},
        "events_per_s": events_all / (ms_max * 1e-3),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "collide electron-ion (Brems+Trident) batched" if prec == pcc.FP32_BATCHED
                     else "collide electron-ion plain FP64",
                     "bytes_per_launch": bytes_ei, "ms_per_launch": ei_avg, "peak_kind": peak_kind},
        "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
        "status": status,
    }
    if rank == 0 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(counts, budget_s=args.cpu_budget)
    if rank == 0:
        print(json.dumps(result))
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def e2e_measure(args, ctx, pcc, torch, dev, n_cells, mat_of_cell, ion_mass, dt, seed, prec):
    """Same step through the C ABI, with every step's particle state copied in
    from pinned host buffers and the step's counters and ledger read back."""
    names = ("em", "ep", "ph")
    fields = ("ux", "uy", "uz", "w", "pid")
    host = {k: {f: getattr(dev[k], f).cpu().pin_memory() for f in fields} for k in names}
    ledger = torch.zeros((n_cells, 4), dtype=torch.float32, device="cuda")
    led_h = torch.zeros((n_cells, 4), dtype=torch.float32).pin_memory()
    h2d = sum(t.numel() * t.element_size() for d in host.values() for t in d.values())
    d2h = led_h.numel() * 4 + 13 * 8
    stream = torch.cuda.current_stream()
    n = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(n):
        for k in names:
            for f in fields:
                getattr(dev[k], f).copy_(host[k][f], non_blocking=True)
        pcc.collide(ctx, n_cells, mat_of_cell, ion_mass, dev["em"], dev["ep"], dev["ph"], dev["ion"], dt, seed,
                    10_000 + s, precision=prec, ledger=ledger)
        for k in names:
            pcc.append_secondaries(ctx, n_cells, dev[k])
        led_h.copy_(ledger, non_blocking=True)
        _, st = ctx.read_status(stream)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    pairs = sum(st["pairs"])
    return {"value": pairs / (el / n), "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "steps": n}


# ---------------------------------------------------------- CPU oracle leg --
def oracle_sample(counts, budget_s, seed=11):
    """Run the FP64 oracle on a random 1/256 subset of the cells for about
    budget_s seconds of CPU time; returns pairs/s and the sample description."""
    from oracle import oracle as orc
    from paper_1907_02814_gb300 import workloads as W
    n_cells = len(counts["e"])
    rng = np.random.default_rng(seed)
    sub = np.sort(rng.choice(n_cells, n_cells // 256, replace=False))
    data = W.batched_cu_host(counts, cells=sub)
    remap = np.zeros(n_cells, np.int32)
    remap[sub] = np.arange(len(sub), dtype=np.int32)
    for d in data.values():
        if len(d["cell"]):
            d["cell"] = remap[d["cell"]]
    m = counts["material"]
    T = orc.OracleTables([orc.material(m.Z, m.Zstar, m.n_i, m.T_e)], orc.table_spec())
    sp = {k: orc.OracleSpecies(v, cap=len(v["w"]) + 200000) for k, v in data.items()}
    mats = np.zeros(len(sub), np.int32)
    pairs = 0.0
    steps = 0
    t0 = time.process_time()
    while True:
        _, st = orc.step(T, len(sub), mats, sp["em"], sp["ep"], sp["ph"], sp["ion"], counts["ion_mass"],
                         counts["dt"], counts["seed"], steps)
        pairs += sum(st["pairs"])
        steps += 1
        if time.process_time() - t0 >= budget_s:
            break
    el = time.process_time() - t0
    return pairs / el, f"{len(sub)} of {n_cells} cells (1/256, same occupancy law), {steps} oracle steps", steps


def cpu_baseline(counts, budget_s=10.0):
    v, sample, _ = oracle_sample(counts, budget_s)
    return {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_1907_02814_gb300 import workloads as W
    counts = W.batched_cu(seed=3)
    per_step = []
    for s in range(args.warmup + args.steps):
        v, sample, _ = oracle_sample(counts, budget_s=args.cpu_budget / max(1, args.steps + args.warmup), seed=11 + s)
        if s >= args.warmup:
            per_step.append(v)
    value = float(np.mean(per_step))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "precision": "fp64 oracle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
