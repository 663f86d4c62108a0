"""Parity at the benchmark's full size: one step of the 1048576-cell batched
Cu workload (about 2.0e8 electrons), launched exactly as the benchmark
launches it, checked cell by cell against the FP64 oracle on sampled cells
(the largest cells, cells with fewer projectiles than ions, and random ones).
The plain FP64 path must match bit for bit; the batched FP32 path within
its decision-mismatch bound."""
import numpy as np
import pytest

import precision_study as PS

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1907_02814_gb300 import workloads as W  # noqa: E402

SLACK = {"em": (8, 0.05), "ep": (16, 0.0), "ph": (32, 0.3), "ion": (0, 0.0)}
FIELDS = ("ux", "uy", "uz", "w", "pid")


@pytest.fixture(scope="module")
def pcc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_02814_gb300 import build, pcc as p
    build.build()
    return p


@pytest.fixture(scope="module")
def setup(pcc):
    ctx = pcc.Context(0)
    counts = W.batched_cu(seed=3)
    m = counts["material"]
    ctx.tables_build([pcc.material(m.Z, m.Zstar, m.n_i, m.T_e)], pcc.table_spec())
    n_cells = len(counts["e"])
    states = []
    for _ in range(2):
        parts = W.batched_cu_device(counts, device="cuda")
        dev = {}
        for name in ("em", "ion", "ph"):
            p = parts.pop(name)
            sa, sr = SLACK[name]
            cap = int(p["n"] + sa * n_cells + int(np.ceil(sr * p["n"])) + n_cells)
            sp = pcc.DeviceSpecies.empty(n_cells, cap)
            pcc.bin(ctx, p, n_cells, sp, slack_abs=sa, slack_rel=sr)
            dev[name] = sp
        sa, sr = SLACK["ep"]
        dev["ep"] = pcc.DeviceSpecies.empty(n_cells, sa * n_cells)
        pcc.bin(ctx, {"n": 0, "ux": None, "uy": None, "uz": None, "w": None, "pid": None, "cell": None}, n_cells,
                dev["ep"], slack_abs=sa, slack_rel=sr)
        states.append(dev)
    torch.cuda.synchronize()
    ce, ci, cg = counts["e"], counts["i"], counts["g"]
    rng = np.random.default_rng(7)
    largest = np.argsort(ce)[-8:]
    caseb = np.nonzero((ce > 0) & (ce < ci))[0]
    caseb = rng.choice(caseb, min(8, len(caseb)), replace=False) if len(caseb) else np.zeros(0, np.int64)
    photon_b = np.nonzero((cg > 0) & (cg < ci))[0]
    photon_b = rng.choice(photon_b, min(8, len(photon_b)), replace=False) if len(photon_b) else np.zeros(0, np.int64)
    rand = rng.choice(n_cells, 40, replace=False)
    sample = np.unique(np.concatenate([largest, caseb, photon_b, rand])).astype(np.int64)
    yield ctx, counts, states, sample
    ctx.close()


def gather(sp, cells):
    """Live particles of the given cells (storage order), copied to the host."""
    start = sp.cell_start.cpu().numpy()
    cnt = sp.cell_count.cpu().numpy()
    idx = np.concatenate([np.arange(start[c], start[c] + cnt[c]) for c in cells]).astype(np.int64)
    it = torch.as_tensor(idx, device=sp.w.device)
    out = {f: getattr(sp, f)[it].cpu().numpy() for f in FIELDS}
    out["pid"] = out["pid"].view(np.uint64)
    out["cell"] = np.repeat(np.asarray(cells, np.int32), cnt[cells])
    out["x"] = None
    return out


def oracle_step(orc, counts, before, n_cells):
    m = counts["material"]
    T = orc.OracleTables([orc.material(m.Z, m.Zstar, m.n_i, m.T_e)], orc.table_spec())
    sp = {k: orc.OracleSpecies(v, cap=len(v["w"]) + 100000) for k, v in before.items()}
    _, st = orc.step(T, n_cells, np.zeros(n_cells, np.int32), sp["em"], sp["ep"], sp["ph"], sp["ion"],
                     counts["ion_mass"], counts["dt"], counts["seed"], 0)
    assert st["rc"] == 0
    return sp, st


def gpu_step(pcc, ctx, counts, dev, precision):
    n_cells = len(counts["e"])
    mat = torch.zeros(n_cells, dtype=torch.int32, device="cuda")
    ctx.read_status()
    pcc.collide(ctx, n_cells, mat, counts["ion_mass"], dev["em"], dev["ep"], dev["ph"], dev["ion"], counts["dt"],
                counts["seed"], 0, precision=precision)
    for k in ("em", "ep", "ph"):
        pcc.append_secondaries(ctx, n_cells, dev[k])
    return ctx.read_status()


def test_full_size_plain_fp64_bit_exact_on_sampled_cells(pcc, setup, orc):
    ctx, counts, states, sample = setup
    n_cells = len(counts["e"])
    dev = states[0]
    before = {k: gather(dev[k], sample) for k in ("em", "ep", "ph", "ion")}
    status, _ = gpu_step(pcc, ctx, counts, dev, pcc.FP64_PLAIN)
    assert status == 0
    sp, st = oracle_step(orc, counts, before, n_cells)
    assert st["status"] == 0
    events = 0
    for k in ("em", "ep", "ph"):
        g = gather(dev[k], sample)
        o = sp[k].canonical()
        order = np.lexsort((g["pid"], g["cell"]))
        assert np.array_equal(g["pid"][order], o["pid"]), k
        assert np.array_equal(g["cell"][order], o["cell"]), k
        for f in ("ux", "uy", "uz"):
            np.testing.assert_allclose(g[f][order], o[f], rtol=2e-6, atol=1e-6, err_msg=f"{k}.{f}")
        assert np.array_equal(g["w"][order], o["w"]), k
        events += int(np.count_nonzero(o["pid"] >> np.uint64(63)))
    assert events > 0


def test_full_size_batched_fp32_on_sampled_cells(pcc, setup, orc):
    ctx, counts, states, sample = setup
    n_cells = len(counts["e"])
    dev = states[1]
    before = {k: gather(dev[k], sample) for k in ("em", "ep", "ph", "ion")}
    status, stats = gpu_step(pcc, ctx, counts, dev, pcc.FP32_BATCHED)
    assert status == 0
    sp, st = oracle_step(orc, counts, before, n_cells)
    pairs = sum(st["pairs"])
    # distinct events (secondary identifier without its last bit)
    g = PS.event_keys_all([gather(dev[k], sample) for k in ("em", "ep", "ph")])
    o = PS.event_keys_all([sp[k].canonical() for k in ("em", "ep", "ph")])
    mism = len(np.setxor1d(g, o))
    assert mism <= max(2, 1e-5 * pairs), (mism, pairs)
    # all pairs of the whole grid were visited
    ce, ci, cg = counts["e"], counts["i"], counts["g"]
    both = (ce > 0) & (ci > 0)
    assert stats["pairs"][0] == int(np.maximum(ce, ci)[both].sum())
    bothg = (cg > 0) & (ci > 0)
    assert stats["pairs"][2] == int(np.maximum(cg, ci)[bothg].sum())


def secondary_pids(sp):
    """Identifiers of the live secondaries (marker bit 63 set) on the device."""
    cnt = sp.cell_count.long()
    start = sp.cell_start[:-1].long()
    run0 = torch.cumsum(cnt, 0) - cnt
    n = int(cnt.sum())
    idx = torch.repeat_interleave(start, cnt) + (torch.arange(n, device=cnt.device) - torch.repeat_interleave(run0, cnt))
    pid = sp.pid[idx]
    return pid[pid < 0]


def test_full_size_fp32_vs_fp64_decision_mismatch(pcc, setup):
    """After the two tests above, both states have taken the same first step,
    one on the plain FP64 path and one on the batched FP32 path: over all
    ~2.3e8 pairs the events (identified by their secondaries' ids) differ in
    a fraction below 1e-5 of the pairs."""
    ctx, counts, states, sample = setup
    ce, ci, cg = counts["e"], counts["i"], counts["g"]
    pairs = int(np.maximum(ce, ci)[(ce > 0) & (ci > 0)].sum()) + int(np.maximum(cg, ci)[(cg > 0) & (ci > 0)].sum())
    # distinct events: a secondary identifier without its last bit (the two
    # leptons of a Trident or Bethe-Heitler pair share it)
    a = torch.unique(torch.cat([secondary_pids(states[0][k]) for k in ("em", "ep", "ph")]) >> 1)
    b = torch.unique(torch.cat([secondary_pids(states[1][k]) for k in ("em", "ep", "ph")]) >> 1)
    diff = int((~torch.isin(a, b)).sum()) + int((~torch.isin(b, a)).sum())
    total = int(a.numel())
    print(f"\n[full size] FP32 vs FP64 GPU: {diff} differing events of {total}, {pairs} pairs "
          f"({diff / pairs:.2e} per pair)")
    assert total > 50_000
    assert diff <= 1e-5 * pairs
