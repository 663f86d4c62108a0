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

FULL_CELLS = 1 << 20


def workload_name(cells):
    return f"batched_cu_{cells}cells_lognormal_median64_sigma1.5_cap8192_dt1fs"


def workload_counts(W, cells, seed):
    """The batched Cu workload; fewer cells keep the same occupancy law and
    the same ions per electron (3e7 ions per 2^20 cells)."""
    return W.batched_cu(n_cells=cells, seed=seed, total_ions=int(round(30_000_000 * cells / FULL_CELLS)))
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
    """SM clock and throttle reasons sampled during the timed region: NVML
    (every 5 ms) when the driver library can be opened, else nvidia-smi
    (every 100 ms).  Reads only; changes no setting."""
    SW_POWER_CAP, HW_SLOWDOWN, SW_THERMAL, HW_THERMAL = 0x4, 0x8, 0x20, 0x40

    def __init__(self, cuda_index, period_s=0.005):
        self.cuda_index = cuda_index
        self.period = period_s
        self.rows = []          # (sm_mhz, reason bits)
        self.max_mhz = None
        self.source = None
        self._stop = threading.Event()
        self.thread = None
        self.proc = None

    def _nvml_handle(self):
        import ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        h = ctypes.c_void_p()
        import torch
        p = torch.cuda.get_device_properties(self.cuda_index)
        tries = []
        uuid = getattr(p, "uuid", None)
        if uuid is not None:
            tries.append(("nvmlDeviceGetHandleByUUID", f"GPU-{uuid}".encode()))
        if hasattr(p, "pci_bus_id"):
            bus = f"{p.pci_domain_id:08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0".encode()
            tries.append(("nvmlDeviceGetHandleByPciBusId_v2", bus))
        for fn, arg in tries:
            if getattr(lib, fn)(ctypes.c_char_p(arg), ctypes.byref(h)) == 0:
                return lib, h
        if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.cuda_index), ctypes.byref(h)) == 0:
            return lib, h
        raise OSError("no NVML handle for this device")

    def start(self):
        import ctypes
        try:
            lib, h = self._nvml_handle()
            reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                lib.nvmlDeviceGetCurrentClocksThrottleReasons
            mx = ctypes.c_uint(0)
            if lib.nvmlDeviceGetMaxClockInfo(h, ctypes.c_int(1), ctypes.byref(mx)) == 0:
                self.max_mhz = float(mx.value)
            self.source = "nvml"

            def loop():
                c, r = ctypes.c_uint(0), ctypes.c_ulonglong(0)
                while not self._stop.is_set():
                    if lib.nvmlDeviceGetClockInfo(h, ctypes.c_int(1), ctypes.byref(c)) == 0 and \
                            reasons_fn(h, ctypes.byref(r)) == 0:
                        self.rows.append((float(c.value), int(r.value)))
                    time.sleep(self.period)
            self.thread = threading.Thread(target=loop, daemon=True)
            self.thread.start()
            return
        except (OSError, AttributeError):
            pass
        self._start_smi()

    def _start_smi(self):
        q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.cuda_index), "-lms", "100"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            return
        self.source = "nvidia-smi"
        bits = (self.HW_SLOWDOWN, self.HW_THERMAL, self.SW_THERMAL, self.SW_POWER_CAP)

        def read():
            for line in self.proc.stdout:
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 6 and f[0].replace(".", "").isdigit():
                    self.max_mhz = float(f[1]) if f[1].replace(".", "").isdigit() else self.max_mhz
                    self.rows.append((float(f[0]), sum(b for b, v in zip(bits, f[2:6]) if v == "Active")))
        self.thread = threading.Thread(target=read, daemon=True)
        self.thread.start()

    def stop(self):
        self._stop.set()
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)
        names = {self.HW_SLOWDOWN: "hw_slowdown", self.HW_THERMAL: "hw_thermal_slowdown",
                 self.SW_THERMAL: "sw_thermal_slowdown", self.SW_POWER_CAP: "sw_power_cap"}
        reasons = sorted({n for _, r in self.rows for b, n in names.items() if r & b})
        sm = [c for c, _ in self.rows]
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": self.max_mhz, "reasons": reasons,
                "samples": len(self.rows), "source": self.source}


# Sources of the collision kernels: the ncu summaries in profiles/ carry
# their hash and are used only while it still matches.
COLLIDE_SOURCES = ("pcc_collide.cu", "pcc_device.cuh", "pcc_internal.h", "pcc_physics.cuh")


def source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1907_02814_gb300", "csrc")
    for f in COLLIDE_SOURCES:
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


# Cell-region slack (absolute, relative) per species: room for the
# secondaries that the warm-up and timed steps append.
SLACK = {"em": (8, 0.05), "ep": (16, 0.0), "ph": (32, 0.3), "ion": (0, 0.0)}


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


# Algorithmic bytes (minimum traffic of the method, FP32 state): a particle
# record is u (12 B) + W (4 B) + id (8 B) = 24 B; per cell, a start and a
# count (8 B) of every species read, the material id (4 B) and the
# 16-byte ledger; writes of 12 B per changed projectile and 32 B per
# secondary (record + id).
REC_B, CELL_SPECIES_B, CELL_FIXED_B, CHANGED_B, SECONDARY_B = 24, 8, 20, 12, 32


def ei_bytes(live, n_cells, changed, secondaries):
    """One electron-ion collide launch: every electron and ion record."""
    return (REC_B * (live["em"] + live["ion"]) + (2 * CELL_SPECIES_B + CELL_FIXED_B) * n_cells
            + CHANGED_B * changed + SECONDARY_B * secondaries)


def step_bytes(live, n_cells, changed, secondaries):
    """One full step: the records of every species, the cell metadata of all
    four species, and the writes."""
    return (REC_B * (live["em"] + live["ep"] + live["ph"] + live["ion"])
            + (4 * CELL_SPECIES_B + CELL_FIXED_B) * n_cells + CHANGED_B * changed + SECONDARY_B * secondaries)


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_1907_02814_gb300 import build, pcc
    from paper_1907_02814_gb300 import tune as tuner
    from paper_1907_02814_gb300 import workloads as W

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    pcc.load()
    ctx = pcc.Context(local)
    counts = workload_counts(W, args.cells, 3 + rank)
    n_cells = len(counts["e"])
    dev = setup(ctx, pcc, W, torch, counts, SLACK)
    mat_of_cell = torch.zeros(n_cells, dtype=torch.int32, device="cuda")
    ledger = torch.zeros((n_cells, 4), dtype=torch.float32, device="cuda")
    prec = pcc.FP32_BATCHED if args.precision == "fp32" else pcc.FP64_PLAIN
    stream = torch.cuda.current_stream()
    dt, seed = counts["dt"], counts["seed"]
    ion_mass = counts["ion_mass"]
    mask = pcc.BREMS | pcc.TRIDENT | pcc.BH

    schedule = None
    if prec == pcc.FP32_BATCHED and not args.no_tune:
        schedule = tuner.tune(ctx, pcc, torch, n_cells, mat_of_cell, ion_mass, dev, dt, seed, step=90_000)

    def eager_step(s):
        pcc.collide(ctx, n_cells, mat_of_cell, ion_mass, dev["em"], dev["ep"], dev["ph"], dev["ion"], dt, seed, s,
                    mask=mask, precision=prec, ledger=ledger)
        for k in ("em", "ep", "ph"):
            pcc.append_secondaries(ctx, n_cells, dev[k])

    for s in range(args.warmup):
        eager_step(s)
    torch.cuda.synchronize()
    # the K timed steps as one CUDA graph, with events around each part of each step
    ctx.steps_capture(n_cells, mat_of_cell, ion_mass, dev["em"], dev["ep"], dev["ph"], dev["ion"], dt, seed,
                      step0=args.warmup, n_steps=args.steps, mask=mask, precision=prec, ledger=ledger, timing=True)
    torch.cuda.synchronize()
    ctx.read_status()
    before = live_counts(dev, torch)

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.05)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = pcc.launch_count()
    start.record(stream)
    ctx.steps_launch()
    end.record(stream)
    launches = pcc.launch_count() - launches0
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = start.elapsed_time(end)
    parts = ctx.steps_timing()            # [K][EI, EP, PH, commit] ms
    status, stats = ctx.read_status()
    after = live_counts(dev, torch)
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
    plain = plain_measure(args, ctx, pcc, torch, dev, n_cells, mat_of_cell, ion_mass, dt, seed, ledger,
                          pairs_all / args.steps / world) if prec == pcc.FP32_BATCHED and args.plain_steps > 0 else None
    emission = emission_measure(ctx, pcc, torch, W) if not args.no_emission else None

    peak, peak_kind = peaks()
    K = args.steps
    avg_live = {k: 0.5 * (before[k] + after[k]) for k in before}
    cr = stats["created"]                 # Brems e-, Brems e+, Trident e-, Trident e+, BH
    ei_changed = (cr[0] + cr[2]) / K
    ei_secondaries = (cr[0] + 2 * cr[2]) / K
    all_changed = (cr[0] + cr[1] + cr[2] + cr[3]) / K
    all_secondaries = (cr[0] + cr[1] + 2 * (cr[2] + cr[3] + cr[4])) / K
    b_ei = ei_bytes(avg_live, n_cells, ei_changed, ei_secondaries)
    b_step = step_bytes(avg_live, n_cells, all_changed, all_secondaries)
    ei_ms = float(np.mean(parts[:, 0]))
    step_ms = ms_max / K
    achieved = b_ei / (ei_ms * 1e-3) / 1e9
    achieved_step = b_step / (step_ms * 1e-3) / 1e9
    tag = "collide_ei_batched" if prec == pcc.FP32_BATCHED else "collide_ei_plain"
    result = {
        "metric": METRIC, "value": pairs_all / (ms_max * 1e-3), "unit": UNIT, "n_gpus": world,
        "steps": K, "warmup": args.warmup, "ms_per_step": step_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if prec == pcc.FP32_BATCHED else "f64", "data": "synthetic",
        "config": {"workload": workload_name(n_cells), "cells": n_cells, "electrons": before["em"], "ions": before["ion"],
                   "photons": before["ph"], "positrons": before["ep"], "precision": args.precision,
                   "l2": "inputs larger than L2 (about 7 GB of particle records), no flush",
                   "timed": f"{K} steps in one CUDA graph", "schedule": schedule and list(schedule["schedule"]),
                   "schedule_ms": schedule and schedule["ms"],
                   "parallelism": f"replicas{world}"},
        "events_per_s": events_all / (ms_max * 1e-3),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": profiled_traffic(tag),
                     "kernel": "pcc_collide electron-ion group (Brems + Trident), "
                               + ("batched FP32" if prec == pcc.FP32_BATCHED else "plain FP64"),
                     "bytes_per_launch": b_ei, "ms_per_launch": ei_ms, "peak_kind": peak_kind},
        "roofline_step": {"bound": "hbm", "achieved": achieved_step, "peak": peak, "unit": "GB/s",
                          "frac": achieved_step / peak, "bytes_per_step": b_step,
                          "ms_parts": {"ei": ei_ms, "ep": float(np.mean(parts[:, 1])),
                                       "ph": float(np.mean(parts[:, 2])), "commit": float(np.mean(parts[:, 3]))}},
        "e2e": e2e,
        "plain_fp64": plain and dict(plain, speedup_of_batched=plain["ms_per_step"] / (ms_max / K)),
        "expected_emission": emission,
        "gpu_launches": int(launches),
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


def plain_measure(args, ctx, pcc, torch, dev, n_cells, mat_of_cell, ion_mass, dt, seed, ledger, pairs_per_step):
    """The plain per-cell FP64 path (one block per cell) on the same state:
    eager steps timed with CUDA events; same kernels as the FP64 parity tests."""
    stream = torch.cuda.current_stream()
    ms = []
    for s in range(args.plain_steps + 1):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pcc.collide(ctx, n_cells, mat_of_cell, ion_mass, dev["em"], dev["ep"], dev["ph"], dev["ion"], dt, seed,
                    20_000 + s, precision=pcc.FP64_PLAIN, ledger=ledger)
        for k in ("em", "ep", "ph"):
            pcc.append_secondaries(ctx, n_cells, dev[k])
        b.record(stream)
        torch.cuda.synchronize()
        if s > 0:                       # the first step warms the plain kernels
            ms.append(a.elapsed_time(b))
    status, st = ctx.read_status()
    m = float(np.mean(ms))
    return {"ms_per_step": m, "value": pairs_per_step / (m * 1e-3), "unit": UNIT, "steps": len(ms),
            "status": status}


def emission_measure(ctx, pcc, torch, W, reps=5):
    """Expected-emission operator at 4096 cells x 512 samples x 64 nodes:
    forward and adjoint kernel times (CUDA events, median of reps)."""
    d = W.emission_params()
    params = torch.as_tensor(np.stack([d[k] for k in ("n_i", "T_e", "Zstar", "s_TF", "s_D")], 1),
                             dtype=torch.float32, device="cuda")
    g = torch.as_tensor(d["gamma"], dtype=torch.float32, device="cuda")
    w = torch.as_tensor(d["w"], dtype=torch.float32, device="cuda")
    gout = torch.ones((g.shape[0], 3), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    res = {}
    for name, fn in (("fwd", lambda: pcc.expected_emission_fwd(ctx, d["Z"], params, g, w)),
                     ("bwd", lambda: pcc.expected_emission_bwd(ctx, d["Z"], params, g, w, gout))):
        fn()
        ms = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        res[f"ms_{name}"] = float(np.median(ms))
    samples = g.numel()
    res.update({"cells": g.shape[0], "samples": samples, "nodes": 64,
                "fwd_samples_per_s": samples / (res["ms_fwd"] * 1e-3),
                "bwd_samples_per_s": samples / (res["ms_bwd"] * 1e-3)})
    ctx.read_status()
    return res


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
    counts = workload_counts(W, args.cells, 3)
    per_step = []
    for s in range(args.warmup + args.steps):
        v, sample, _ = oracle_sample(counts, budget_s=args.cpu_budget / max(1, args.steps + args.warmup), seed=11 + s)
        if s >= args.warmup:
            per_step.append(v)
    value = float(np.mean(per_step))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": workload_name(args.cells), "precision": "fp64 oracle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--cells", type=int, default=FULL_CELLS, help="smaller cases keep the occupancy law")
    ap.add_argument("--plain-steps", type=int, default=2, help="timed steps of the plain FP64 path (0: skip)")
    ap.add_argument("--no-emission", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
