"""The seeded synthetic inputs of the batched Cu workload follow their stated
recipe: log-normal electron occupancy (median 64, sigma 1.5, capped at
8192), ions in proportion with at least one per occupied cell, photons
0.25 N_e, electron kinetic energies exponential with mean 1 MeV, photon
energies with density k^-2 on [2, 200] m_e c^2, and draws that depend only
on (seed, cell), so a subset of cells gives the same particles."""
import numpy as np
import pytest
from scipy import stats

from paper_1907_02814_gb300 import workloads as W


@pytest.fixture(scope="module")
def counts():
    return W.batched_cu(n_cells=1 << 15, seed=3, total_ions=int(round(30_000_000 * (1 << 15) / (1 << 20))))


def test_occupancy_law(counts):
    e = counts["e"]
    assert e.max() <= 8192
    assert abs(np.median(e) - 64) <= 2
    occ = e[(e >= 1) & (e < 8192)]
    # log-normal with sigma 1.5: the interquartile range of ln N is 2 * 0.674 sigma
    q1, q3 = np.percentile(np.log(occ), [25, 75])
    assert (q3 - q1) == pytest.approx(2 * 0.6745 * 1.5, rel=0.05)
    i = counts["i"]
    assert np.all(i[e > 0] >= 1) and np.all(i[e == 0] == 0)
    assert abs(i.sum() - 30_000_000 * (1 << 15) / (1 << 20)) <= (e > 0).sum()
    g = counts["g"]
    assert g.sum() / e.sum() == pytest.approx(0.25, rel=0.01)
    assert np.all(g <= e)


def test_particle_laws(counts):
    cells = np.arange(0, 1 << 15, 64)
    d = W.batched_cu_host(counts, cells=cells)
    em, ph = d["em"], d["ph"]
    u2 = em["ux"].astype(np.float64) ** 2 + em["uy"].astype(np.float64) ** 2 + em["uz"].astype(np.float64) ** 2
    T_mev = (np.sqrt(1.0 + u2) - 1.0) * W.MEC2_MEV
    assert stats.kstest(T_mev, stats.expon(scale=1.0).cdf).pvalue > 1e-3
    k = np.sqrt(ph["ux"].astype(np.float64) ** 2 + ph["uy"].astype(np.float64) ** 2 + ph["uz"].astype(np.float64) ** 2)
    assert k.min() >= 2.0 * (1 - 1e-6) and k.max() <= 200.0 * (1 + 1e-6)
    cdf = lambda x: (1.0 / 2.0 - 1.0 / x) / (1.0 / 2.0 - 1.0 / 200.0)       # density k^-2 on [2, 200]
    assert stats.kstest(k, cdf).pvalue > 1e-3
    # isotropic directions: mean cosine 0 and <cos^2> = 1/3
    mu = em["uz"].astype(np.float64) / np.sqrt(u2)
    assert abs(mu.mean()) < 4 / np.sqrt(3 * len(mu)) and abs((mu ** 2).mean() - 1 / 3) < 0.01
    assert np.array_equal(np.unique(em["cell"]), cells[counts["e"][cells] > 0])


def test_subset_draws_match_the_full_draw(counts):
    sub = np.array([5, 77, 1000, 31000])
    a = W.batched_cu_host(counts, cells=sub)
    full_cells = np.arange(0, 31001)
    b = W.batched_cu_host(counts, cells=full_cells)
    for k in ("em", "ion", "ph"):
        m = np.isin(b[k]["cell"], sub)
        for f in ("ux", "uy", "uz", "w", "pid", "cell"):
            assert np.array_equal(a[k][f], b[k][f][m]), (k, f)
