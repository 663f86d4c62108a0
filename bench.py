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
    emission = emission_measure(ctx, pcc, torch, W, local) if not args.no_emission else None
    config2 = config2_measure(ctx, pcc, torch, W) if not args.no_config2 else None

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
                   "scan_classes": {str(g): ctx.scan_classes(g) for g in (0, 1, 2)},
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
        "config2": config2,
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


# Sources of the expected-emission kernels: the ncu summary's instruction
# counts are used only while its hash still matches.
EMISSION_SOURCES = ("pcc_emission.cu", "pcc_physics.cuh", "pcc_internal.h", "pcc_device.cuh")
EMISSION_PROFILE = "expected_emission_4096x512_full.md"
SM_LANES = 128          # FP32 lanes (and thread-instructions issued per clock) per SM


def emission_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1907_02814_gb300", "csrc")
    for f in EMISSION_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def emission_instructions():
    """Warp instructions per launch of the forward and adjoint emission
    kernels from the committed ncu summary, if it was taken on the current
    sources (else None)."""
    p = os.path.join(ROOT, "profiles", EMISSION_PROFILE)
    if not os.path.exists(p):
        return None
    text = open(p).read()
    if f"source_hash: {emission_source_hash()}" not in text:
        return None
    out, which = {}, None
    for line in text.splitlines():
        if line.startswith("## ") and "emission_kernel<0>" in line:
            which = "fwd"
        elif line.startswith("## ") and "emission_kernel<1>" in line:
            which = "bwd"
        elif which and line.startswith("- warp instructions:"):
            out[which] = float(line.split(":")[1].split()[0])
    return out if len(out) == 2 else None


def emission_measure(ctx, pcc, torch, W, local=0, reps=5):
    """Expected-emission operator at 4096 cells x 512 samples x 64 nodes:
    forward and adjoint kernel times (CUDA events, median of reps), and the
    issue roofline: warp instructions per launch (ncu) x 32 over the time,
    against SMs x 128 thread-instructions per clock at the sampled SM clock."""
    d = W.emission_params()
    params = torch.as_tensor(np.stack([d[k] for k in ("n_i", "T_e", "Zstar", "s_TF", "s_D")], 1),
                             dtype=torch.float32, device="cuda")
    g = torch.as_tensor(d["gamma"], dtype=torch.float32, device="cuda")
    w = torch.as_tensor(d["w"], dtype=torch.float32, device="cuda")
    gout = torch.ones((g.shape[0], 3), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    res = {}
    clocks = ClockSampler(local)
    clocks.start()
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
    clk = clocks.stop()
    samples = g.numel()
    res.update({"cells": g.shape[0], "samples": samples, "nodes": 64,
                "fwd_samples_per_s": samples / (res["ms_fwd"] * 1e-3),
                "bwd_samples_per_s": samples / (res["ms_bwd"] * 1e-3), "clocks": clk})
    inst = emission_instructions()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = clk["sm_mhz"] or clk["sm_max_mhz"]
    if inst and mhz:
        peak = sms * SM_LANES * mhz * 1e6 / 1e12
        res["roofline"] = {}
        for name in ("fwd", "bwd"):
            ach = inst[name] * 32 / (res[f"ms_{name}"] * 1e-3) / 1e12
            res["roofline"][name] = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "T thread-instr/s",
                                     "frac": ach / peak, "thread_instr_per_node":
                                         inst[name] * 32 / (samples * 64)}
    ctx.read_status()
    return res


def config2_measure(ctx, pcc, torch, W, steps=100, plain_steps=3):
    """The Au foil configuration (16384 cells, Poisson(256) electrons per cell,
    E^-2 on 0.1-100 MeV, 64 Au ions per cell with integer Z* in [10, 40]: 31
    material tables, 256 x 256, built in FP64), Brems + Bethe-Heitler, dt =
    1 fs: `steps` steps of collide + commit as one CUDA graph on the batched
    FP32 path, and eager steps of the plain FP64 path from the same initial
    state.  Particles are not moved between steps (the push of the transport
    run is a harness, not part of the collision step)."""
    wl = W.au_foil()
    ctx.tables_build([pcc.material(m.Z, m.Zstar, m.n_i, m.T_e) for m in wl.materials], pcc.table_spec())
    mat = torch.as_tensor(wl.material_of_cell, device="cuda")
    n_cells = wl.n_cells
    mask = pcc.BREMS | pcc.BH
    slack = {"em": 16, "ep": 16, "ph": 128, "ion": 0}
    empty = {"n": 0, "ux": None, "uy": None, "uz": None, "w": None, "pid": None, "cell": None, "x": None}

    def state():
        dev = {}
        for k, d in wl.species.items():
            n = len(d["w"])
            sp = pcc.DeviceSpecies.empty(n_cells, n + (slack[k] + 1) * n_cells, with_x=d.get("x") is not None)
            pcc.bin(ctx, pcc.particles_to_device(d) if n else empty, n_cells, sp, slack_abs=slack[k], slack_rel=0.0)
            dev[k] = sp
        return dev

    stream = torch.cuda.current_stream()
    res = {"workload": "au_foil_16384cells_poisson256_Z79_Zstar10-40_brems_bh_dt1fs", "cells": n_cells,
           "materials": len(wl.materials)}
    dev = state()
    ctx.read_status()
    ctx.steps_capture(n_cells, mat, wl.ion_mass, dev["em"], dev["ep"], dev["ph"], dev["ion"], wl.dt, wl.seed,
                      step0=0, n_steps=steps, mask=mask, precision=pcc.FP32_BATCHED)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    ctx.steps_launch()
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    status, st = ctx.read_status()
    res["fp32_batched"] = {"steps": steps, "ms_per_step": ms / steps, "value": sum(st["pairs"]) / (ms * 1e-3),
                           "events": sum(st["created"]), "unit": UNIT, "status": status,
                           "timed": f"{steps} steps in one CUDA graph"}
    dev = state()
    times, pairs = [], 0
    for s in range(plain_steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pcc.collide(ctx, n_cells, mat, wl.ion_mass, dev["em"], dev["ep"], dev["ph"], dev["ion"], wl.dt, wl.seed, s,
                    mask=mask, precision=pcc.FP64_PLAIN)
        for k in ("em", "ep", "ph"):
            pcc.append_secondaries(ctx, n_cells, dev[k])
        b.record(stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    status, st = ctx.read_status()
    m = float(np.mean(times))
    res["fp64_plain"] = {"steps": plain_steps, "ms_per_step": m, "value": sum(st["pairs"]) / plain_steps / (m * 1e-3),
                         "unit": UNIT, "status": status, "timed": "eager steps, CUDA events"}
    res["speedup_of_batched"] = m / res["fp32_batched"]["ms_per_step"]
    return res


# Slack of the end-to-end layout: each step starts again from the host state,
# so a region needs room for one step's secondaries only (about 4e4 events
# per step over 2^20 cells: a few in a small cell, 2 % covers the largest).
E2E_SLACK = {"em": (4, 0.02), "ep": (4, 0.0), "ph": (4, 0.02)}


def h2d_rate(torch, nbytes=1 << 30, reps=3):
    """Pinned host-to-device copy rate of this machine, GB/s (best of reps)."""
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    best = 0.0
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d.copy_(h, non_blocking=True)
        torch.cuda.synchronize()
        best = max(best, nbytes / (time.perf_counter() - t0) / 1e9)
    del h, d
    return best


def live_records(torch, sp):
    """The live particles of a species in storage order, as pcc_bin input."""
    cnt = sp.cell_count.long()
    n_cells = cnt.numel()
    n = int(cnt.sum())
    cell = torch.repeat_interleave(torch.arange(n_cells, device=cnt.device, dtype=torch.int32), cnt)
    first = torch.repeat_interleave(sp.cell_start[:-1].long(), cnt)
    run0 = torch.cumsum(cnt, 0) - cnt
    idx = first + (torch.arange(n, device=cnt.device) - torch.repeat_interleave(run0, cnt))
    return {"ux": sp.ux[idx], "uy": sp.uy[idx], "uz": sp.uz[idx], "w": sp.w[idx], "pid": sp.pid[idx], "cell": cell,
            "x": None, "n": n}


def e2e_measure(args, ctx, pcc, torch, dev, n_cells, mat_of_cell, ion_mass, dt, seed, prec):
    """Same step through the C ABI, with every step's particle state copied
    in from pinned host buffers and the step's counters and ledger read back
    (one untimed warm-up step, then up to 5 timed steps).
    The state is held in a layout of its own whose regions keep only the slack
    one step needs, so the copies are the live records plus about 3 %: per
    species the momenta, weights and ids of every slot and the live count of
    every cell (the ions, which a step only reads, stay resident)."""
    names = ("em", "ep", "ph")
    fields = ("ux", "uy", "uz", "w", "pid", "cell_count")
    state = {}
    for k in names:
        live = live_records(torch, dev[k])
        sa, sr = E2E_SLACK[k]
        cap = int(live["n"] + sa * n_cells + int(np.ceil(sr * live["n"])) + n_cells)
        sp = pcc.DeviceSpecies.empty(n_cells, cap)
        empty = {"n": 0, "ux": None, "uy": None, "uz": None, "w": None, "pid": None, "cell": None}
        pcc.bin(ctx, live if live["n"] else empty, n_cells, sp, slack_abs=sa, slack_rel=sr)
        state[k] = sp
        del live
    host = {k: {f: getattr(state[k], f).cpu().pin_memory() for f in fields} for k in names}
    ledger = torch.zeros((n_cells, 4), dtype=torch.float32, device="cuda")
    led_h = torch.zeros((n_cells, 4), dtype=torch.float32).pin_memory()
    h2d = sum(t.numel() * t.element_size() for d in host.values() for t in d.values())
    d2h = led_h.numel() * 4 + 13 * 8
    live_bytes = 24 * sum(int(state[k].cell_count.sum()) for k in names)
    n = max(1, min(args.steps, 5))

    cur = torch.cuda.current_stream()
    copy_ms = []

    def one_step(s, timed=False):
        if timed:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(cur)
        for k in names:
            for f in fields:
                getattr(state[k], f).copy_(host[k][f], non_blocking=True)
        if timed:
            e1.record(cur)
            copy_ms.append((e0, e1))
        pcc.collide(ctx, n_cells, mat_of_cell, ion_mass, state["em"], state["ep"], state["ph"], dev["ion"], dt, seed,
                    10_000 + s, precision=prec, ledger=ledger)
        for k in names:
            pcc.append_secondaries(ctx, n_cells, state[k])
        led_h.copy_(ledger, non_blocking=True)
        return ctx.read_status(torch.cuda.current_stream())

    one_step(100)                          # warm-up on the new layout, untimed
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(n):
        status, st = one_step(s, timed=True)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    h2d_ms = float(np.mean([a.elapsed_time(b) for a, b in copy_ms]))
    pairs = sum(st["pairs"])
    del state, host
    return {"value": pairs / (el / n), "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "live_record_bytes_per_step": int(live_bytes), "steps": n, "status": status,
            "ms_per_step": 1e3 * el / n, "h2d_ms_per_step": h2d_ms, "h2d_gbs_measured": h2d_rate(torch)}


# ---------------------------------------------------------- CPU oracle leg --
def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OracleSample:
    """The FP64 oracle on a fixed random 1/256 subset of the cells (same
    occupancy law), stepped in place; threads = OpenMP threads over cells."""

    def __init__(self, counts, seed=11):
        from oracle import oracle as orc
        from paper_1907_02814_gb300 import workloads as W
        self.orc = orc
        self.counts = counts
        n_cells = len(counts["e"])
        rng = np.random.default_rng(seed)
        self.sub = np.sort(rng.choice(n_cells, n_cells // 256, replace=False))
        self.data = W.batched_cu_host(counts, cells=self.sub)
        remap = np.zeros(n_cells, np.int32)
        remap[self.sub] = np.arange(len(self.sub), dtype=np.int32)
        for d in self.data.values():
            if len(d["cell"]):
                d["cell"] = remap[d["cell"]]
        m = counts["material"]
        self.T = orc.OracleTables([orc.material(m.Z, m.Zstar, m.n_i, m.T_e)], orc.table_spec())
        self.mats = np.zeros(len(self.sub), np.int32)
        self.reset()
        self.describe = f"{len(self.sub)} of {n_cells} cells (1/256, same occupancy law, fixed subset)"

    def reset(self):
        self.sp = {k: self.orc.OracleSpecies(v, cap=len(v["w"]) + 200000) for k, v in self.data.items()}
        self.steps = 0

    def step(self, threads):
        """One oracle step; returns (pairs, wall seconds)."""
        self.orc.set_threads(threads)
        c = self.counts
        t0 = time.perf_counter()
        _, st = self.orc.step(self.T, len(self.sub), self.mats, self.sp["em"], self.sp["ep"], self.sp["ph"],
                              self.sp["ion"], c["ion_mass"], c["dt"], c["seed"], self.steps)
        el = time.perf_counter() - t0
        self.orc.set_threads(1)
        self.steps += 1
        return sum(st["pairs"]), el

    def rate(self, threads, budget_s):
        """pairs/s over whole steps from the initial state, for about budget_s
        seconds of wall time."""
        self.reset()
        pairs = el = 0.0
        while True:
            p, t = self.step(threads)
            pairs += p
            el += t
            if el >= budget_s:
                return pairs / el, self.steps


def cpu_baseline(counts, budget_s=10.0):
    """The oracle timed on this host's cores: single-threaded and with OpenMP
    threads over the cells on every core this process may use."""
    cores = host_cores()
    s = OracleSample(counts)
    v1, n1 = s.rate(1, 0.5 * budget_s)
    threads = s.orc.set_threads(cores)
    s.orc.set_threads(1)
    vm, nm = s.rate(threads, 0.5 * budget_s)
    return {"value": vm, "unit": UNIT, "cores": threads, "cores_available": cores, "value_1t": v1,
            "value_omp": vm, "threads_omp": threads, "kind": "oracle",
            "sample": f"{s.describe}; {n1} steps single-threaded, {nm} steps on {threads} threads"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_1907_02814_gb300 import workloads as W
    counts = workload_counts(W, args.cells, 3)
    s = OracleSample(counts)
    cores = host_cores()
    threads = s.orc.set_threads(cores)
    s.orc.set_threads(1)
    for _ in range(args.warmup):
        s.step(threads)
    pairs = el = 0.0
    for _ in range(args.steps):
        p, t = s.step(threads)
        pairs += p
        el += t
    value = pairs / el
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args.cells), "precision": "fp64 oracle",
                   "sample": s.describe + " stepped in place; one oracle step per bench step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "cores_available": cores, "kind": "oracle",
                         "sample": f"{s.describe}; {args.steps} timed steps after {args.warmup} on {threads} threads"},
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
    ap.add_argument("--no-config2", action="store_true", help="skip the Au foil (16384-cell) leg")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
