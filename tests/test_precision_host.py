"""Host bookkeeping of the precision study (tests/precision_study.py) on
the oracle's own output: event keys decode to the cell and channel of the
event, one key per created event, and the host pair count equals the
oracle's counters."""
import numpy as np

import precision_study as PS
from paper_1907_02814_gb300 import workloads as W


def test_event_keys_and_pairs_from_an_oracle_step(orc):
    wl = W.solid_cu(n_cells=24, e_per_cell=np.arange(24) % 7 * 9, i_per_cell=5, seed=8, dt=4e-13,
                    photons_per_cell=np.arange(24) % 5 * 3)
    m = wl.materials[0]
    T = orc.OracleTables([orc.material(m.Z, m.Zstar, m.n_i, m.T_e)], orc.table_spec(n_rows=48, n_cols=48))
    sp = {k: orc.OracleSpecies(v, cap=len(v["w"]) + 20000) for k, v in wl.species.items()}
    n_cells = wl.n_cells
    for s in range(2):
        before = {k: sp[k].canonical() for k in ("em", "ep", "ph")}
        nion = PS.cell_counts(wl.species["ion"], n_cells)
        pc = sum(PS.pairs_per_cell(PS.cell_counts(before[k], n_cells), nion) for k in ("em", "ep", "ph"))
        _, st = orc.step(T, n_cells, wl.material_of_cell, sp["em"], sp["ep"], sp["ph"], sp["ion"], wl.ion_mass,
                         wl.dt, wl.seed, s)
        assert sum(st["pairs"]) == int(pc.sum())
        after = {k: sp[k].canonical() for k in ("em", "ep", "ph")}
        keys = PS.event_keys([after[k] for k in ("em", "ep", "ph")], s)
        assert len(keys) == int(sum(st["created"])) > 0
        assert np.array_equal(np.bincount(PS.key_channel(keys), minlength=5), np.asarray(st["created"], int))
        for k in ("em", "ep", "ph"):
            d = after[k]
            sec = PS.is_secondary(d["pid"]) & (PS.secondary_step(d["pid"]) == s)
            assert np.array_equal(PS.key_cell(d["pid"][sec] >> np.uint64(1)), d["cell"][sec].astype(np.int64))
        # no secondary of an earlier step is counted again
        assert len(PS.event_keys([after[k] for k in ("em", "ep", "ph")], s + 7)) == 0


def test_energy_and_weight_sums():
    d = {"ux": np.array([0.0, 3.0, 0.0], np.float32), "uy": np.array([0.0, 4.0, 0.0], np.float32),
         "uz": np.array([0.0, 0.0, 1.0], np.float32), "w": np.array([2.0, 1.0, 3.0], np.float32),
         "cell": np.array([0, 0, 2], np.int32)}
    np.testing.assert_allclose(PS.energy_per_cell(d, 3, photon=False), [2.0 + np.sqrt(26.0), 0.0, 3 * np.sqrt(2.0)])
    np.testing.assert_allclose(PS.energy_per_cell(d, 3, photon=True), [5.0, 0.0, 3.0])
    np.testing.assert_allclose(PS.weight_per_cell(d, 3), [3.0, 0.0, 3.0])
    assert list(PS.pairs_per_cell([0, 3, 5, 2], [4, 0, 2, 7])) == [0, 0, 5, 7]
    np.testing.assert_allclose(PS.rel([1.0, 0.0, 2.0], [2.0, 0.0, 2.0]), [0.5, 0.0, 0.0])
