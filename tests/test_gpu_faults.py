"""Fault injection through the C ABI, none of which faults, traps or hangs
the GPU: out-of-range inputs set sticky status bits that the host reads
after the step, while the rest of the step proceeds; a forced give-up of
the batched kernels' bounded wait sets PCC_ST_TIMEOUT without changing any
result.  And checkpoint/resume: with counter-based random streams a run
resumed at step k from a saved state equals the uninterrupted run."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1907_02814_gb300 import workloads as W  # noqa: E402

SPEC = dict(n_rows=64, n_cols=64)
EMPTY = {"n": 0, "ux": None, "uy": None, "uz": None, "w": None, "pid": None, "cell": None}


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


def prec_of(pcc, precision):
    return pcc.FP64_PLAIN if precision == "fp64" else pcc.FP32_BATCHED


def to_device(pcc, ctx, species, n_cells, slack=600):
    dev = {}
    for name, d in species.items():
        n = len(d["w"])
        sp = pcc.DeviceSpecies.empty(n_cells, n + slack * n_cells + n)
        pcc.bin(ctx, pcc.particles_to_device(d) if n else EMPTY, n_cells, sp, slack_abs=slack, slack_rel=1.0)
        dev[name] = sp
    return dev


def run(pcc, ctx, wl, precision, steps=1, step0=0, mat=None, species=None, mask=7):
    """Steps step0 .. step0 + steps - 1 on fresh device copies of the
    workload's particles (or of `species`); returns (dev, status, stats)."""
    ctx.tables_build([pcc.material(m.Z, m.Zstar, m.n_i, m.T_e) for m in wl.materials], pcc.table_spec(**SPEC))
    dev = to_device(pcc, ctx, species or wl.species, wl.n_cells)
    mat = torch.as_tensor(wl.material_of_cell if mat is None else mat, device="cuda")
    ctx.read_status()
    status, stats = 0, []
    for s in range(step0, step0 + steps):
        pcc.collide(ctx, wl.n_cells, mat, wl.ion_mass, dev["em"], dev["ep"], dev["ph"], dev["ion"], wl.dt, wl.seed, s,
                    mask=mask, precision=prec_of(pcc, precision))
        for k in ("em", "ep", "ph"):
            pcc.append_secondaries(ctx, wl.n_cells, dev[k])
        st, sts = ctx.read_status()
        status |= st
        stats.append(sts)
    return dev, status, stats


def oracle_status(orc, wl, species=None, mask=7, mat=None):
    T = orc.OracleTables([orc.material(m.Z, m.Zstar, m.n_i, m.T_e) for m in wl.materials], orc.table_spec(**SPEC))
    sp = {k: orc.OracleSpecies(v, cap=len(v["w"]) + 100000) for k, v in (species or wl.species).items()}
    _, st = orc.step(T, wl.n_cells, wl.material_of_cell if mat is None else mat, sp["em"], sp["ep"], sp["ph"],
                     sp["ion"], wl.ion_mass, wl.dt, wl.seed, 0, mask=mask)
    return st


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_energy_above_table_is_flagged(pcc, ctx, orc, precision):
    """Electrons at gamma = 5000, above the table's 2000: the last row serves
    and PCC_ST_TABLE_RANGE is set, as in the oracle."""
    wl = W.solid_cu(n_cells=8, e_per_cell=32, i_per_cell=8, seed=41, dt=50e-15, beam_gamma=5000.0)
    _, status, stats = run(pcc, ctx, wl, precision)
    assert status & pcc.ST_TABLE_RANGE
    assert int(oracle_status(orc, wl)["status"]) & 1
    assert stats[0]["pairs"][0] == 8 * 32


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_long_time_step_is_flagged(pcc, ctx, orc, precision):
    """A step so long that n sigma v dt exceeds 1: PCC_ST_PROB_LARGE, as in
    the oracle; every pair then collides."""
    wl = W.solid_cu(n_cells=8, e_per_cell=32, i_per_cell=8, seed=42, dt=1e-9, T_mev=5.0)
    _, status, stats = run(pcc, ctx, wl, precision, mask=1)
    assert status & pcc.ST_PROB_LARGE
    assert int(oracle_status(orc, wl, mask=1)["status"]) & 2
    assert stats[0]["accepted"][0] == 8 * 32


def test_every_pair_a_candidate_in_large_cells(pcc, ctx, orc):
    """Large cells (2048 electrons, scanned by whole warps) in a step so long
    that every pair collides: every pair is then a candidate, more than the
    scan's per-warp staging holds at once, and all of them reach the queue
    (the accepted pairs equal the oracle's: all but those whose electron lies
    below the Brems threshold)."""
    wl = W.solid_cu(n_cells=2, e_per_cell=2048, i_per_cell=16, seed=44, dt=1e-7, T_mev=5.0)
    _, status, stats = run(pcc, ctx, wl, "fp32", mask=1)
    assert status & pcc.ST_PROB_LARGE     # (the photon store overflows too: 2048 new photons per cell)
    assert stats[0]["pairs"][0] == 2 * 2048
    assert stats[0]["candidates"][0] == 2 * 2048
    ost = oracle_status(orc, wl, mask=1)
    assert int(ost["status"]) & 2
    assert stats[0]["accepted"][0] == int(ost["accepted"][0]) > 2 * 2048 - 16


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_nonfinite_momentum_is_flagged(pcc, ctx, precision):
    """A NaN momentum: PCC_ST_NONFINITE; the step finishes and every pair is
    still counted.  The batched path reads a momentum only for pairs that
    pass the quick reject, so the step is long enough here (bound >= 1) that
    every pair is evaluated."""
    wl = W.solid_cu(n_cells=8, e_per_cell=32, i_per_cell=8, seed=43, dt=1e-10, T_mev=30.0)
    em = dict(wl.species["em"])
    em["ux"] = em["ux"].copy()
    em["ux"][5] = np.nan
    species = dict(wl.species, em=em)
    _, status, stats = run(pcc, ctx, wl, precision, species=species, mask=1)
    assert status & pcc.ST_NONFINITE
    assert stats[0]["pairs"][0] == 8 * 32


def test_batched_flags_only_conditions_met_by_evaluated_pairs(pcc, ctx):
    """The documented difference between the paths: the batched FP32 path
    reads a projectile's momentum only for pairs that pass the quick reject,
    so a NaN momentum and an energy above the table in cells whose pairs are
    all rejected from their accept digits alone raise no status bit there,
    while the plain FP64 path, which evaluates every pair, flags both.  With
    dt = 1e-22 s the per-material bound gives an accept threshold of 0, so
    no pair is a candidate; no event happens on either path."""
    wl = W.solid_cu(n_cells=8, e_per_cell=32, i_per_cell=8, seed=48, dt=1e-22, T_mev=2.0)
    em = {k: (v.copy() if v is not None else None) for k, v in wl.species["em"].items()}
    em["ux"][3] = np.nan
    g = 5000.0                        # above the table's gamma_max = 2000
    em["ux"][17], em["uy"][17], em["uz"][17] = np.sqrt(g * g - 1.0), 0.0, 0.0
    species = dict(wl.species, em=em)
    _, st64, stats64 = run(pcc, ctx, wl, "fp64", species=species)
    _, st32, stats32 = run(pcc, ctx, wl, "fp32", species=species)
    assert st64 & pcc.ST_NONFINITE and st64 & pcc.ST_TABLE_RANGE
    assert stats32[0]["candidates"][0] == 0
    assert st32 == 0, pcc.status_bits(st32)
    assert stats64[0]["pairs"] == stats32[0]["pairs"] and stats64[0]["pairs"][0] == 8 * 32
    assert sum(stats64[0]["created"]) == sum(stats32[0]["created"]) == 0


@pytest.mark.parametrize("gamma,flagged", [(2e7, True), (1e6, False)])
def test_trident_bound_range_is_flagged(pcc, ctx, gamma, flagged):
    """The batched path's Trident quick-reject bound is proven for ion-frame
    Lorentz factors up to 1e7: an evaluated pair above it raises
    PCC_ST_BOUND_RANGE (batched path only; the plain path has no bound).  The
    step is long enough that every pair is a candidate."""
    wl = W.solid_cu(n_cells=4, e_per_cell=16, i_per_cell=4, seed=49, dt=1e-10, beam_gamma=gamma)
    _, st32, stats32 = run(pcc, ctx, wl, "fp32", mask=pcc.TRIDENT)
    _, st64, _ = run(pcc, ctx, wl, "fp64", mask=pcc.TRIDENT)
    assert stats32[0]["candidates"][0] == 4 * 16
    assert bool(st32 & pcc.ST_BOUND_RANGE) == flagged, pcc.status_bits(st32)
    assert st64 & pcc.ST_BOUND_RANGE == 0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_material_index_out_of_range_is_flagged(pcc, ctx, precision):
    """A cell whose material index is past the tables: PCC_ST_NONFINITE, and
    that cell is skipped (its pairs are not counted) while the others run."""
    wl = W.solid_cu(n_cells=8, e_per_cell=32, i_per_cell=8, seed=44, dt=50e-15)
    mat = np.zeros(8, np.int32)
    mat[3] = 7
    _, status, stats = run(pcc, ctx, wl, precision, mat=mat, mask=1)
    assert status & pcc.ST_NONFINITE
    assert stats[0]["pairs"][0] == 7 * 32


def test_step_index_out_of_range_is_flagged(pcc, ctx):
    """Step indices of 2^19 and above no longer fit the secondaries' id
    field: PCC_ST_ID_RANGE."""
    wl = W.solid_cu(n_cells=4, e_per_cell=16, i_per_cell=4, seed=45, dt=50e-15)
    for precision in ("fp64", "fp32"):
        _, status, _ = run(pcc, ctx, wl, precision, step0=1 << 19)
        assert status & pcc.ST_ID_RANGE, precision


def test_forced_wait_timeout_changes_nothing_but_the_status(pcc, ctx):
    """With the bounded waits set to give up at once, every staged launch
    reports PCC_ST_TIMEOUT and falls back to the global table rows, which
    hold the same values: the particles come out identical."""
    wl = W.solid_cu(n_cells=64, e_per_cell=128, i_per_cell=16, seed=46, dt=300e-15, T_mev=20.0,
                    photons_per_cell=32)
    ref, st_ref, stats_ref = run(pcc, ctx, wl, "fp32", steps=2)
    ctx.set_wait_limit(0)
    try:
        got, st_got, stats_got = run(pcc, ctx, wl, "fp32", steps=2)
    finally:
        ctx.set_wait_limit()
    assert st_ref & pcc.ST_TIMEOUT == 0
    assert st_got & pcc.ST_TIMEOUT
    assert (st_got & ~pcc.ST_TIMEOUT) == st_ref
    assert sum(sum(s["created"]) for s in stats_ref) > 20
    assert [s["created"] for s in stats_got] == [s["created"] for s in stats_ref]
    for k in ("em", "ep", "ph"):
        a, b = ref[k].live_host(), got[k].live_host()
        for f in ("pid", "cell", "ux", "uy", "uz", "w"):
            assert np.array_equal(a[f], b[f]), (k, f)
    # the context stays usable: a normal step afterwards reports no timeout
    _, st_after, _ = run(pcc, ctx, wl, "fp32", steps=1)
    assert st_after & pcc.ST_TIMEOUT == 0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_checkpoint_and_resume(pcc, ctx, precision):
    """Six steps in one go, against three steps, a checkpoint of every
    species to the host, a new binning from it, and steps 3-5: identical
    particles (ids, cells, momenta, weights) and counters."""
    wl = W.solid_cu(n_cells=48, e_per_cell=96, i_per_cell=24, seed=47, dt=300e-15, T_mev=20.0,
                    photons_per_cell=24)
    full, st_full, stats_full = run(pcc, ctx, wl, precision, steps=6)
    part, _, stats_a = run(pcc, ctx, wl, precision, steps=3)
    saved = {}
    for k in ("em", "ep", "ph", "ion"):
        h = part[k].live_host()
        saved[k] = {"ux": h["ux"], "uy": h["uy"], "uz": h["uz"], "w": h["w"], "pid": h["pid"], "cell": h["cell"],
                    "x": None}
    resumed, st_res, stats_b = run(pcc, ctx, wl, precision, steps=3, step0=3, species=saved)
    assert sum(sum(s["created"]) for s in stats_full) > 50
    assert [s["created"] for s in stats_a + stats_b] == [s["created"] for s in stats_full]
    assert [s["pairs"] for s in stats_a + stats_b] == [s["pairs"] for s in stats_full]
    for k in ("em", "ep", "ph"):
        a, b = full[k].live_host(), resumed[k].live_host()
        for f in ("pid", "cell", "ux", "uy", "uz", "w"):
            assert np.array_equal(a[f], b[f]), (precision, k, f)
