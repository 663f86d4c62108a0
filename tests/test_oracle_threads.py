"""The oracle's OpenMP leg (threads over the cells of a group, used to time
the CPU baseline on all host cores) gives the single-threaded result bit for
bit: every cell touches only its own particles, ledger entry and absorbed-
photon flags, secondaries take atomically claimed slots and the canonical
(cell, id) order does not depend on where they landed."""
import numpy as np
import pytest

from paper_1907_02814_gb300 import workloads as W


def run(orc, wl, threads, steps=3):
    got = orc.set_threads(threads)
    try:
        m = wl.materials
        T = orc.OracleTables([orc.material(x.Z, x.Zstar, x.n_i, x.T_e) for x in m],
                             orc.table_spec(n_rows=64, n_cols=64))
        sp = {k: orc.OracleSpecies(v, cap=len(v["w"]) + 50000) for k, v in wl.species.items()}
        ledger = np.zeros((wl.n_cells, 2))
        stats = []
        for s in range(steps):
            _, st = orc.step(T, wl.n_cells, wl.material_of_cell, sp["em"], sp["ep"], sp["ph"], sp["ion"],
                             wl.ion_mass, wl.dt, wl.seed, s, ledger=ledger)
            stats.append(st)
        return got, {k: sp[k].canonical() for k in ("em", "ep", "ph")}, ledger, stats
    finally:
        orc.set_threads(1)


def test_result_does_not_depend_on_thread_count(orc):
    rng = np.random.default_rng(12)
    n_cells = 96
    wl = W.solid_cu(n_cells=n_cells, e_per_cell=rng.integers(0, 120, n_cells), i_per_cell=rng.integers(1, 40, n_cells),
                    seed=12, dt=300e-15, T_mev=20.0, photons_per_cell=rng.integers(0, 50, n_cells))
    _, ref, led_ref, st_ref = run(orc, wl, 1)
    assert sum(sum(s["created"]) for s in st_ref) > 100
    for threads in (2, 5):
        got, out, led, st = run(orc, wl, threads)
        if got == 1:
            pytest.skip("oracle built without OpenMP")
        assert [s["created"] for s in st] == [s["created"] for s in st_ref]
        assert [s["pairs"] for s in st] == [s["pairs"] for s in st_ref]
        assert [s["status"] for s in st] == [s["status"] for s in st_ref]
        for k in ("em", "ep", "ph"):
            for f in ("pid", "cell", "ux", "uy", "uz", "w"):
                assert np.array_equal(out[k][f], ref[k][f]), (threads, k, f)
        assert np.array_equal(led, led_ref)
