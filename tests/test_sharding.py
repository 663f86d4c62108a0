"""The step shards by cells: every random number is keyed by (seed, step,
cell, slot or pair), so ranks that each own a range of cells (keeping the
global cell indices) reproduce the single-process step bit for bit.  Run as
world_size-2 gloo process groups on the CPU with the oracle; the same keying
is what makes the CUDA path's replicas independent.  The conservation
ledger is the one collective: a 3-double FP64 all-reduce over the ranks."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _workload():
    sys.path.insert(0, ROOT)
    from paper_1907_02814_gb300 import workloads as W
    rng = np.random.default_rng(5)
    e = rng.integers(0, 60, 40)
    return W.solid_cu(n_cells=40, e_per_cell=e, i_per_cell=rng.integers(1, 30, 40), seed=5, dt=300e-15,
                      T_mev=20.0, photons_per_cell=rng.integers(0, 20, 40))


def _run(wl, cells, steps=2):
    from oracle import oracle as orc
    keep = {k: np.isin(v["cell"], cells) for k, v in wl.species.items()}
    sub = {k: {f: (a[keep[k]] if a is not None else None) for f, a in v.items()} for k, v in wl.species.items()}
    T = orc.OracleTables([orc.material(m.Z, m.Zstar, m.n_i, m.T_e) for m in wl.materials],
                         orc.table_spec(n_rows=64, n_cols=64))
    sp = {k: orc.OracleSpecies(v, cap=len(v["w"]) + 50000) for k, v in sub.items()}
    for s in range(steps):
        orc.step(T, wl.n_cells, wl.material_of_cell, sp["em"], sp["ep"], sp["ph"], sp["ion"], wl.ion_mass, wl.dt,
                 wl.seed, s)
    return {k: sp[k].canonical() for k in ("em", "ep", "ph")}


def _totals(species):
    """FP64 conservation ledger of a population: total energy (rest mass
    included, in m_e c^2 per m^3), charge (in e per m^3) and weight."""
    e = 0.0
    q = 0.0
    n = 0.0
    for k, charge in (("em", -1.0), ("ep", 1.0), ("ph", 0.0)):
        d = species[k]
        u2 = d["ux"].astype(np.float64) ** 2 + d["uy"].astype(np.float64) ** 2 + d["uz"].astype(np.float64) ** 2
        w = d["w"].astype(np.float64)
        energy = np.sqrt(u2) if k == "ph" else np.sqrt(1.0 + u2)
        e += float(np.sum(w * energy))
        q += charge * float(np.sum(w))
        n += float(np.sum(w))
    return [e, q, n]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = _workload()
    cells = np.array_split(np.arange(wl.n_cells), world)[rank]
    mine = _run(wl, cells)
    got = [None] * world
    dist.all_gather_object(got, mine)
    # the ledger's one collective: a 3-double FP64 sum over the ranks
    ledger = torch.tensor(_totals(mine), dtype=torch.float64)
    dist.all_reduce(ledger)
    if rank == 0:
        q.put((got, ledger.tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_single_process_step():
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got, ledger = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    sys.path.insert(0, ROOT)
    wl = _workload()
    whole = _run(wl, np.arange(wl.n_cells))
    for k in ("em", "ep", "ph"):
        merged = {f: np.concatenate([g[k][f] for g in got]) for f in ("pid", "cell", "ux", "uy", "uz", "w")}
        order = np.lexsort((merged["pid"], merged["cell"]))
        for f in ("pid", "cell", "ux", "uy", "uz", "w"):
            assert np.array_equal(merged[f][order], whole[k][f]), (k, f)
    assert np.count_nonzero(whole["ph"]["pid"] >> np.uint64(63)) > 0
    # the all-reduced ledger equals the single-process one up to summation order
    assert ledger == pytest.approx(_totals(whole), rel=1e-13, abs=1e-13 * abs(_totals(whole)[0]))


def test_reference_arm_under_two_ranks_prints_one_line():
    """bench.py --impl reference under torchrun with 2 ranks: rank 0 runs the
    oracle and prints one JSON line, rank 1 exits 0 without work."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", "29561", os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1", "--cpu-budget", "1",
           "--cells", "8192"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle"
