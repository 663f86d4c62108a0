"""The batching pattern: the multi-step loop captured as one CUDA graph
gives the same state as the same steps launched one call at a time; the
library's launch counter matches the kernels it enqueues; the schedule
autotuner applies and caches a candidate."""
import numpy as np
import pytest

import precision_study as PS

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1907_02814_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def pcc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_02814_gb300 import build, pcc as p
    build.build()
    return p


@pytest.fixture(scope="module")
def ctx(pcc):
    c = pcc.Context(0)
    yield c
    c.close()


def workload(n_cells=64, seed=11, dt=300e-15):
    rng = np.random.default_rng(seed)
    e = rng.integers(0, 120, n_cells)
    e[:2] = [0, 700]
    i = rng.integers(1, 50, n_cells)
    return W.solid_cu(n_cells=n_cells, e_per_cell=e, i_per_cell=i, seed=seed, dt=dt, T_mev=20.0,
                      photons_per_cell=rng.integers(0, 40, n_cells))


def to_device(pcc, ctx, wl, slack_abs=2048):
    dev = {}
    for name, d in wl.species.items():
        n = len(d["w"])
        sp = pcc.DeviceSpecies.empty(wl.n_cells, n + slack_abs * wl.n_cells + n // 2 + wl.n_cells)
        pcc.bin(ctx, pcc.particles_to_device(d), wl.n_cells, sp, slack_abs=slack_abs, slack_rel=0.5)
        dev[name] = sp
    return dev


def tables(pcc, ctx, wl):
    ctx.tables_build([pcc.material(m.Z, m.Zstar, m.n_i, m.T_e) for m in wl.materials],
                     pcc.table_spec(n_rows=128, n_cols=128))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_graph_matches_eager_steps(pcc, ctx, precision):
    """Three steps as one graph launch vs three steps of separate calls:
    identical particles (ids, momenta, weights), counters and status."""
    prec = pcc.FP64_PLAIN if precision == "fp64" else pcc.FP32_BATCHED
    wl = workload()
    tables(pcc, ctx, wl)
    mat = torch.as_tensor(wl.material_of_cell, device="cuda")
    steps = 3

    a = to_device(pcc, ctx, wl)
    la = torch.zeros((wl.n_cells, 4), dtype=torch.float32, device="cuda")
    ctx.read_status()
    for s in range(steps):
        pcc.collide(ctx, wl.n_cells, mat, wl.ion_mass, a["em"], a["ep"], a["ph"], a["ion"], wl.dt, wl.seed, s,
                    precision=prec, ledger=la)
        for k in ("em", "ep", "ph"):
            pcc.append_secondaries(ctx, wl.n_cells, a[k])
    st_a, stats_a = ctx.read_status()

    b = to_device(pcc, ctx, wl)
    lb = torch.zeros((wl.n_cells, 4), dtype=torch.float32, device="cuda")
    ctx.steps_capture(wl.n_cells, mat, wl.ion_mass, b["em"], b["ep"], b["ph"], b["ion"], wl.dt, wl.seed, 0, steps,
                      precision=prec, ledger=lb, timing=True)
    ctx.read_status()
    ctx.steps_launch()
    ms = ctx.steps_timing()
    st_b, stats_b = ctx.read_status()

    assert sum(stats_a["created"]) > 20
    # no region overflowed: which secondaries an overflow drops depends on
    # the order of the atomics, so only then could two runs differ
    assert st_a == 0 and st_b == 0
    assert stats_a["pairs"] == stats_b["pairs"]
    assert stats_a["accepted"] == stats_b["accepted"] and stats_a["created"] == stats_b["created"]
    for k in ("em", "ep", "ph"):
        ga, gb = a[k].live_host(), b[k].live_host()
        for f in ("pid", "cell", "ux", "uy", "uz", "w"):
            assert np.array_equal(ga[f], gb[f]), (k, f)
    # ledger columns: (sum, compensation) of radiated energy and of created
    # weight; a cell's event contributions are gathered with float atomics,
    # so only the compensated values are compared
    la, lb = la.cpu().numpy().astype(np.float64), lb.cpu().numpy().astype(np.float64)
    for c0 in (0, 2):
        np.testing.assert_allclose(lb[:, c0] - lb[:, c0 + 1], la[:, c0] - la[:, c0 + 1], rtol=1e-5, atol=0)
    assert ms.shape == (steps, 4) and np.all(ms >= 0) and ms.sum() > 0


def test_launch_count(pcc, ctx):
    """The counter adds 3 class-sort kernels and 4 per group for a batched
    call, 1 per plain group, 1 per commit, and the kernel nodes of a graph
    per graph launch."""
    wl = workload(n_cells=16, seed=12)
    tables(pcc, ctx, wl)
    mat = torch.as_tensor(wl.material_of_cell, device="cuda")
    d = to_device(pcc, ctx, wl)
    c0 = pcc.launch_count()
    pcc.collide(ctx, wl.n_cells, mat, wl.ion_mass, d["em"], d["ep"], d["ph"], d["ion"], wl.dt, wl.seed, 0,
                precision=pcc.FP32_BATCHED)
    assert pcc.launch_count() - c0 == 3 + 3 * 4
    c0 = pcc.launch_count()
    pcc.collide(ctx, wl.n_cells, mat, wl.ion_mass, d["em"], d["ep"], d["ph"], d["ion"], wl.dt, wl.seed, 1,
                mask=pcc.BREMS | pcc.GROUP_EM, precision=pcc.FP64_PLAIN)
    pcc.append_secondaries(ctx, wl.n_cells, d["em"])
    assert pcc.launch_count() - c0 == 2
    c0 = pcc.launch_count()
    ctx.steps_capture(wl.n_cells, mat, wl.ion_mass, d["em"], d["ep"], d["ph"], d["ion"], wl.dt, wl.seed, 5, 2,
                      precision=pcc.FP32_BATCHED)
    assert pcc.launch_count() == c0
    ctx.steps_launch()
    ctx.steps_launch()
    torch.cuda.synchronize()
    assert pcc.launch_count() - c0 == 2 * 2 * (15 + 3)
    ctx.read_status()


def test_tune_applies_and_caches(pcc, ctx, tmp_path):
    from paper_1907_02814_gb300 import tune
    wl = workload(n_cells=256, seed=13)
    tables(pcc, ctx, wl)
    mat = torch.as_tensor(wl.material_of_cell, device="cuda")
    d = to_device(pcc, ctx, wl)
    before = d["em"].ux.clone()
    path = str(tmp_path / "tune.json")
    defaults = {g: ctx.scan_classes(g) for g in (0, 1, 2)}
    r = tune.tune(ctx, pcc, torch, wl.n_cells, mat, wl.ion_mass, d, wl.dt, wl.seed, cache_path=path, reps=1)
    assert tuple(r["schedule"]) in tune.CANDIDATES and not r["cached"]
    sched = [k for k in r["ms"] if not k.startswith("classes")]
    assert len(sched) == len(tune.CANDIDATES) and all(v > 0 for v in r["ms"].values())
    assert set(r["classes"]) == set(tune.CLASS_GROUPS)
    for g, t in r["classes"].items():
        assert tune.valid_classes(t) and ctx.scan_classes(g) == list(t)
    assert torch.equal(d["em"].ux, before)          # trials ran on a scratch copy
    for g, t in defaults.items():
        ctx.set_scan_classes(g, t)
    r2 = tune.tune(ctx, pcc, torch, wl.n_cells, mat, wl.ion_mass, d, wl.dt, wl.seed, cache_path=path)
    assert r2["cached"] and tuple(r2["schedule"]) == tuple(r["schedule"])
    assert {g: list(t) for g, t in r2["classes"].items()} == {g: list(t) for g, t in r["classes"].items()}
    assert all(ctx.scan_classes(g) == list(t) for g, t in r["classes"].items())
    ctx.set_schedule(4, 0)
    for g, t in defaults.items():
        ctx.set_scan_classes(g, t)


def test_scan_classes_keep_the_events(pcc, ctx):
    """The lane-group setting of the scan is a performance choice: whole
    warps for every cell, 2-lane groups for every cell, and the default give
    the same pairs and the same events (it changes only the order of a
    cell's FP32 weight sums, so at most a decision within float rounding of
    its threshold could differ); bad thresholds are rejected."""
    wl = workload(n_cells=128, seed=14)
    tables(pcc, ctx, wl)
    mat = torch.as_tensor(wl.material_of_cell, device="cuda")
    defaults = {g: ctx.scan_classes(g) for g in (0, 1, 2)}
    out = []
    try:
        for thr in (None, [0, 0, 0, 0], [34, 34, 34, 34], [9, 7, 5, 3]):
            if thr is not None:
                for g in (0, 1, 2):
                    ctx.set_scan_classes(g, thr)
            d = to_device(pcc, ctx, wl)
            ctx.read_status()
            for s in range(2):
                pcc.collide(ctx, wl.n_cells, mat, wl.ion_mass, d["em"], d["ep"], d["ph"], d["ion"], wl.dt, wl.seed,
                            s, precision=pcc.FP32_BATCHED)
                for k in ("em", "ep", "ph"):
                    pcc.append_secondaries(ctx, wl.n_cells, d[k])
            st, stats = ctx.read_status()
            out.append((st, stats, {k: d[k].live_host() for k in ("em", "ep", "ph")}))
    finally:
        for g, t in defaults.items():
            ctx.set_scan_classes(g, t)
    st0, stats0, p0 = out[0]
    assert st0 == 0 and sum(stats0["created"]) > 10
    keys0 = PS.event_keys_all([p0[k] for k in ("em", "ep", "ph")])
    for st, stats, p in out[1:]:
        assert st == st0 and stats["pairs"] == stats0["pairs"]
        keys = PS.event_keys_all([p[k] for k in ("em", "ep", "ph")])
        assert len(np.setxor1d(keys, keys0)) <= 2
        assert abs(sum(stats["candidates"]) - sum(stats0["candidates"])) <= 4
    for bad in ([10, 12, 4, 0], [35, 2, 1, 0], [4, 3, 2, -1]):
        with pytest.raises(pcc.PccError, match="thresholds"):
            ctx.set_scan_classes(0, bad)
    with pytest.raises(pcc.PccError):
        ctx.set_scan_classes(3, [4, 3, 2, 1])
    assert ctx.scan_classes(0) == defaults[0]
