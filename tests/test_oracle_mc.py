"""Pins of the oracle's tables, pairing and Monte Carlo step (Sec. III.A)
against quadrature, brute force and the paper's analytic thin-target yield
(Eq. N_br_theo1/2, Fig. valid_brem_tf), and the same thin-target check for
Bethe-Heitler and Trident pair creation."""
import math

import numpy as np
import pytest
from scipy import integrate, stats

from paper_1907_02814_gb300 import workloads as W

C_LIGHT = 299792458.0


def quad(f, a, b, **kw):
    kw.setdefault("epsabs", 0.0)
    kw.setdefault("epsrel", 1e-11)
    kw.setdefault("limit", 400)
    return integrate.quad(f, a, b, **kw)[0]


@pytest.fixture(scope="module")
def cu_tables(orc):
    spec = orc.table_spec(n_rows=64, n_cols=64)
    mats = [orc.material(29, 5, 8.5e28, 100.0), orc.material(79, 30, 5.9e28, 1e3)]
    return orc.OracleTables(mats, spec)


# -------------------------------------------------------------- tables ---
def test_brems_table_matches_quadrature(orc, cu_tables):
    """sigma_B(T) = int_{x_min}^1 dsigma/dk T dx and the CDF columns equal
    adaptive quadrature of the oracle's own dsigma/dk (pins the table
    quadrature, not the formula)."""
    T = cu_tables
    sp = T.spec
    for m in (0, 1):
        s = T.screening(m)
        for r in (0, 17, 40, 63):
            Tk = T.row_value(r)
            g = 1.0 + Tk
            f = lambda lx: orc.dsdk_brems(s, g, math.exp(lx) * Tk) * Tk * math.exp(lx)
            pts = [math.log(0.5)] + [math.log1p(-10.0 ** -j) for j in range(1, 9)]
            tot = quad(f, math.log(sp.x_min), 0.0, points=pts)
            assert T.brems_sigma[m, r] == pytest.approx(tot, rel=1e-8)
            for c in (10, 32, 60):
                xc = T.col_value(orc.TB_BREMS, c)
                part = quad(f, math.log(sp.x_min), math.log(xc))
                assert T.brems_cdf[m, r, c] == pytest.approx(part / tot, rel=1e-8, abs=1e-12)


def test_bh_table_matches_quadrature(orc, cu_tables):
    T = cu_tables
    s = T.screening(0)
    for r in (0, 30, 63):
        kk = 2.0 + T.row_value(r)
        pts = [1.0 + (kk - 2.0) * 10.0 ** -j for j in range(1, 9)]
        pts += [kk - 1.0 - (kk - 2.0) * 10.0 ** -j for j in range(1, 9)]
        tot = quad(lambda g: orc.dsdg_bh(s, kk, g), 1.0, kk - 1.0, points=sorted(pts))
        assert T.bh_sigma[0, r] == pytest.approx(tot, rel=1e-8)
        # symmetric plateau: CDF at y = 1/2 is 1/2
        F = T.bh_cdf[0, r]
        assert F[0] == 0.0 and F[-1] == 1.0 and np.all(np.diff(F) >= 0)


def test_trident_tables_normalised_and_monotone(cu_tables):
    """Trident pair-energy and split CDFs: normalised, monotone and (split)
    symmetric about gamma_p/2.  Their values are pinned in
    test_oracle_trident.py (exact antiderivative, adaptive quadrature)."""
    T = cu_tables
    for F in (T.tri_gp_cdf, T.tri_split_cdf):
        assert np.all(F[:, 0] == 0.0) and np.all(F[:, -1] == 1.0)
        assert np.all(np.diff(F, axis=1) >= 0)
    n = T.spec.n_cols
    mid = T.tri_split_cdf[:, :]
    assert np.allclose(mid + mid[:, ::-1], 1.0, atol=1e-9)


def test_sampler_reproduces_row_cdf(orc, cu_tables):
    """Inverse-CDF sampling at an exact row reproduces that row's CDF (KS)."""
    T = cu_tables
    rng = np.random.default_rng(4)
    r = 40
    Tk = T.row_value(r)
    xs = np.array([T.sample(orc.TB_BREMS, 0, Tk, 0.5, u) for u in rng.uniform(size=4000)])
    grid = np.array([T.col_value(orc.TB_BREMS, c) for c in range(T.spec.n_cols)])
    F = T.brems_cdf[0, r]
    cdf = lambda x: np.interp(np.log(x), np.log(grid), F)
    assert stats.kstest(xs, cdf).pvalue > 1e-3
    assert xs.min() >= T.spec.x_min and xs.max() <= 1.0


@pytest.mark.parametrize("table", ["TB_BREMS", "TB_BH", "TB_TRI_GP", "TB_TRI_SPLIT"])
def test_sampler_mixes_neighbour_rows(orc, cu_tables, table):
    """Between rows j and j+1, at fractional log position f, the stochastic
    row pick (the upper row when u_row < f) makes the samples follow
    (1-f) F_j + f F_{j+1}, each row's CDF interpolated linearly in the
    column's spacing variable (ln y for the log-spaced Brems and Trident
    pair-energy columns, y for BH and the split).  Checked by KS on every
    table kind."""
    T = cu_tables
    tb = getattr(orc, table)
    arr = {"TB_BREMS": T.brems_cdf[1], "TB_BH": T.bh_cdf[1], "TB_TRI_GP": T.tri_gp_cdf,
           "TB_TRI_SPLIT": T.tri_split_cdf}[table]
    mat = 1 if table in ("TB_BREMS", "TB_BH") else 0
    j, f = 47, 0.3
    r = T.row_value(j) * (T.row_value(j + 1) / T.row_value(j)) ** f
    rng = np.random.default_rng(12)
    u = rng.uniform(size=(5000, 2))
    xs = np.array([T.sample(tb, mat, r, a, b) for a, b in u])
    grid = np.array([T.col_value(tb, c) for c in range(T.spec.n_cols)])
    is_log = table in ("TB_BREMS", "TB_TRI_GP")
    tr = np.log if is_log else (lambda v: v)
    cdf = lambda x: (1 - f) * np.interp(tr(x), tr(grid), arr[j]) + f * np.interp(tr(x), tr(grid), arr[j + 1])
    assert stats.kstest(xs, cdf).pvalue > 1e-3
    assert xs.min() >= grid[0] and xs.max() <= grid[-1]
    # the pick itself: u_row just below f takes row j+1, just above takes row j,
    # and each inverts its row's CDF by linear interpolation
    for uc in np.linspace(0.03, 0.97, 11):
        for row, ur in ((j + 1, f - 1e-9), (j, f + 1e-9)):
            F = arr[row]
            lo = np.searchsorted(F, uc, side="right") - 1
            v = tr(grid[lo]) + (uc - F[lo]) / (F[lo + 1] - F[lo]) * (tr(grid[lo + 1]) - tr(grid[lo]))
            want = np.exp(v) if is_log else v
            assert T.sample(tb, mat, r, ur, uc) == pytest.approx(want, rel=1e-12, abs=1e-15), (row, uc)


def test_sigma_lookup_interpolation(orc, cu_tables):
    """Log-log interpolation is exact at rows, zero below the table and
    flags the range above it."""
    T = cu_tables
    for r in (0, 5, 63):
        v, st = T.sigma_lookup(orc.TB_BREMS, 0, T.row_value(r))
        assert v == pytest.approx(T.brems_sigma[0, r], rel=1e-12) and st == 0
    assert T.sigma_lookup(orc.TB_BREMS, 0, T.spec.T_min * 0.99)[0] == 0.0
    v, st = T.sigma_lookup(orc.TB_BREMS, 0, T.spec.T_max * 1.5)
    assert st & 1 and v == T.brems_sigma[0, -1]


# --------------------------------------------------------- permutation ---
@pytest.mark.parametrize("n", [1, 2, 3, 7, 31, 32, 33, 64, 100, 1000, 8192])
def test_permutation_is_bijection(orc, n):
    rk = orc.philox([0, 5, 9, 1], [1, 2])
    pos = [orc.perm_pos(s, n, rk) for s in range(n)]
    assert sorted(pos) == list(range(n))
    for s in range(0, n, max(1, n // 50)):
        assert orc.perm_elem(pos[s], n, rk) == s


@pytest.mark.parametrize("n", [2, 5, 13, 32, 33, 47, 100])
def test_permutation_uniform(orc, n):
    """Over many keys every element is equally likely at every position."""
    draws = 2000 if n <= 47 else 1000
    cnt = np.zeros((n, n))
    for t in range(draws):
        rk = orc.philox([t, 11, 3, 0], [99, 7])
        for s in range(n):
            cnt[s, orc.perm_pos(s, n, rk)] += 1
    chi2 = ((cnt - draws / n) ** 2 / (draws / n)).sum()
    dof = (n - 1) * (n - 1)
    assert stats.chi2.sf(chi2, dof) > 1e-4


# ----------------------------------------------------------- MC step -----
def _run(orc, wl, steps, mask, spec=None, cap_extra=20000):
    spec = spec or orc.table_spec(n_rows=128, n_cols=128)
    mats = [orc.material(m.Z, m.Zstar, m.n_i, m.T_e, m.s_TF, m.s_D) for m in wl.materials]
    T = orc.OracleTables(mats, spec)
    sp = {k: orc.OracleSpecies(v, cap=len(v["w"]) + cap_extra) for k, v in wl.species.items()}
    ledger = np.zeros((wl.n_cells, 2))
    tot = None
    for s in range(steps):
        _, st = orc.step(T, wl.n_cells, wl.material_of_cell, sp["em"], sp["ep"], sp["ph"], sp["ion"],
                         wl.ion_mass, wl.dt, wl.seed, s, mask, ledger)
        assert st["rc"] == 0
        tot = st if tot is None else {k: (np.add(tot[k], st[k]) if k != "status" else tot[k] | st[k])
                                      for k in st}
    return T, sp, ledger, tot


@pytest.mark.parametrize("u_ion", [1.0, -1.0])
def test_bh_rate_on_moving_ions_has_the_moller_flux(orc, u_ion):
    """Photons of k = 20 along +z on ions all moving along z with u = +-1
    (Eq. proba3 with the photon's k, k' and c in place of the electron's
    gamma, gamma' and v'): the collision rate is n_g n_i sigma(k') c (1 - beta_i . n),
    sigma at the Doppler-shifted ion-frame energy k' = k gamma_i (1 - beta_i . n)
    and the flux factor of a massless projectile on a moving target.
    Accepted events against that expectation, 4 sigma."""
    from paper_1907_02814_gb300 import workloads as W
    n_cells, N, k, w = 200, 256, 20.0, 2e26
    cell = np.repeat(np.arange(n_cells), N)
    z = np.zeros(len(cell))
    ph = W._species(z, z, np.full(len(cell), k), np.full(len(cell), w), cell)
    ion = W._species(z, z, np.full(len(cell), u_ion), np.full(len(cell), w), cell, pid0=10 ** 7)
    g_i = math.sqrt(1.0 + u_ion * u_ion)
    flux = 1.0 - u_ion / g_i                        # 1 - beta_i . n, n = +z
    kp = k * g_i * flux
    T = orc.OracleTables([orc.material(29, 0, 8.5e28, 0.0)], orc.table_spec(n_rows=128, n_cols=64))
    sigma, st_ = T.sigma_lookup(orc.TB_BH, 0, kp - 2.0)
    assert st_ == 0 and sigma > 0
    dt = 0.02 / (N * w * sigma * C_LIGHT * flux)      # x = 0.02 per pair
    x = N * w * sigma * C_LIGHT * flux * dt
    sp = {"em": orc.OracleSpecies(W.empty_species(), cap=100000), "ep": orc.OracleSpecies(W.empty_species(), cap=100000),
          "ph": orc.OracleSpecies(ph), "ion": orc.OracleSpecies(ion)}
    _, st = orc.step(T, n_cells, np.zeros(n_cells, np.int32), sp["em"], sp["ep"], sp["ph"], sp["ion"], 1e5, dt, 3, 0,
                     mask=orc.PROC_BH)
    pairs = n_cells * N
    assert st["pairs"][2] == pairs
    expect = pairs * -math.expm1(-x)
    got = st["accepted"][4]
    assert abs(got - expect) < 4.0 * math.sqrt(expect), (got, expect)
    assert st["created"][4] == got                   # equal weights: every accepted event is created


@pytest.mark.parametrize("ui", [(0.0, 0.0, 0.6), (0.0, 0.0, -0.6), (0.8, 0.0, 0.0)])
def test_brems_rate_on_moving_ions_has_the_moller_flux(orc, ui):
    """Electrons of gamma = 20 along +z on ions all moving with momentum ui
    (Eq. proba3 and the ion-frame transform of Sec. III.A): the collision rate is n_e n_i sigma(gamma')
    v_M with Moller's invariant flux v_M = sqrt(|v_e - v_i|^2 - |v_e x v_i|^2/c^2)
    written in lab velocities, and sigma at the ion-frame Lorentz factor
    gamma' = gamma_e gamma_i (1 - beta_e . beta_i).  4 sigma."""
    from paper_1907_02814_gb300 import workloads as W
    n_cells, N, w, ge = 200, 256, 2e26, 20.0
    cell = np.repeat(np.arange(n_cells), N)
    z = np.zeros(len(cell))
    ue = math.sqrt(ge * ge - 1.0)
    em = W._species(z, z, np.full(len(cell), ue), np.full(len(cell), w), cell)
    ion = W._species(np.full(len(cell), ui[0]), np.full(len(cell), ui[1]), np.full(len(cell), ui[2]),
                     np.full(len(cell), w), cell, pid0=10 ** 7)
    # float32 storage of the inputs, as the step reads them
    u_e = np.array([0.0, 0.0, float(np.float32(ue))])
    u_i = np.array([float(np.float32(v)) for v in ui])
    g_e, g_i = math.sqrt(1 + u_e @ u_e), math.sqrt(1 + u_i @ u_i)
    b_e, b_i = u_e / g_e, u_i / g_i
    v_m = math.sqrt((b_e - b_i) @ (b_e - b_i) - np.cross(b_e, b_i) @ np.cross(b_e, b_i))   # units of c
    g_p = g_e * g_i * (1.0 - b_e @ b_i)
    T = orc.OracleTables([orc.material(29, 0, 8.5e28, 0.0)], orc.table_spec(n_rows=128, n_cols=64))
    sigma, st_ = T.sigma_lookup(orc.TB_BREMS, 0, g_p - 1.0)
    assert st_ == 0 and sigma > 0
    dt = 0.02 / (N * w * sigma * C_LIGHT * v_m)
    x = N * w * sigma * C_LIGHT * v_m * dt
    sp = {"em": orc.OracleSpecies(em), "ep": orc.OracleSpecies(W.empty_species()),
          "ph": orc.OracleSpecies(W.empty_species(), cap=100000), "ion": orc.OracleSpecies(ion)}
    _, st = orc.step(T, n_cells, np.zeros(n_cells, np.int32), sp["em"], sp["ep"], sp["ph"], sp["ion"], 1e5, dt, 4, 0,
                     mask=orc.PROC_BREMS)
    pairs = n_cells * N
    assert st["pairs"][0] == pairs
    # pairs within one cell share a projectile only once each (N_e = N_i), so
    # every pair sees the unrecoiled electron
    expect = pairs * -math.expm1(-x)
    got = st["accepted"][0]
    assert abs(got - expect) < 4.0 * math.sqrt(expect), (got, expect)


def _one_pair_per_cell(W, n_cells, proj_u, w=1e27, seed=21):
    cell = np.arange(n_cells)
    z = np.zeros(n_cells)
    proj = W._species(proj_u[:, 0], proj_u[:, 1], proj_u[:, 2], np.full(n_cells, w), cell)
    ion = W._species(z, z, z, np.full(n_cells, w), cell, pid0=10 ** 7)
    return proj, ion


def _unit(u):
    u = np.asarray(u, np.float64)
    return u / np.linalg.norm(u, axis=1, keepdims=True)


def test_secondary_kinematics_with_ions_at_rest(orc):
    """Sec. III.A, ions at rest, one electron and one photon per cell and a
    step long enough that every pair collides: a Brems photon leaves along
    the electron, which keeps its direction and loses the photon's energy; a
    Trident pair leaves along the electron, which pays the pair's energy;
    a BH pair leaves along the photon and shares its energy."""
    from paper_1907_02814_gb300 import workloads as W
    rng = np.random.default_rng(31)
    n = 300
    nx, ny, nz = W._isotropic(rng, n)
    dirs = np.stack([nx, ny, nz], 1)
    T = orc.OracleTables([orc.material(29, 0, 8.5e28, 0.0)], orc.table_spec(n_rows=96, n_cols=64))
    tol = 2e-6                                    # float32 storage
    for mask, g in ((orc.PROC_BREMS, 50.0), (orc.PROC_TRIDENT, 50.0)):
        em, ion = _one_pair_per_cell(W, n, dirs * math.sqrt(g * g - 1))
        sp = {"em": orc.OracleSpecies(em, cap=2 * n), "ep": orc.OracleSpecies(W.empty_species(), cap=1000),
              "ph": orc.OracleSpecies(W.empty_species(), cap=1000), "ion": orc.OracleSpecies(ion)}
        _, st = orc.step(T, n, np.zeros(n, np.int32), sp["em"], sp["ep"], sp["ph"], sp["ion"], 1e5, 1e-3, 5, 0,
                         mask=mask)
        assert st["rc"] == 0 and st["status"] == 2   # x > 1: every pair collides
        e = sp["em"].as_dict()
        prim = e["pid"] < (1 << 63)
        ue = np.stack([e["ux"], e["uy"], e["uz"]], 1)[prim].astype(np.float64)
        order = np.argsort(e["cell"][prim])
        ue = ue[order]
        assert np.allclose(_unit(ue), dirs, atol=tol)
        ge = np.sqrt(1 + (ue ** 2).sum(1))
        if mask == orc.PROC_BREMS:
            assert st["created"][0] == n
            p = sp["ph"].as_dict()
            up = np.stack([p["ux"], p["uy"], p["uz"]], 1).astype(np.float64)[np.argsort(p["cell"])]
            assert np.allclose(_unit(up), dirs, atol=tol)
            assert np.allclose(ge + np.linalg.norm(up, axis=1), g, rtol=tol)
        else:
            assert st["created"][2] == n
            sec = {k: sp[k].as_dict() for k in ("em", "ep")}
            tot = ge.copy()
            for k in ("em", "ep"):
                d = sec[k]
                m = d["pid"] >= (1 << 63)
                u = np.stack([d["ux"], d["uy"], d["uz"]], 1).astype(np.float64)[m][np.argsort(d["cell"][m])]
                assert len(u) == n
                assert np.allclose(_unit(u), dirs, atol=tol)
                tot += np.sqrt(1 + (u ** 2).sum(1))
            assert np.allclose(tot, g, rtol=tol)
    # Bethe-Heitler: photons of k = 30
    k = 30.0
    ph, ion = _one_pair_per_cell(W, n, dirs * k)
    sp = {"em": orc.OracleSpecies(W.empty_species(), cap=1000), "ep": orc.OracleSpecies(W.empty_species(), cap=1000),
          "ph": orc.OracleSpecies(ph), "ion": orc.OracleSpecies(ion)}
    _, st = orc.step(T, n, np.zeros(n, np.int32), sp["em"], sp["ep"], sp["ph"], sp["ion"], 1e5, 1e-3, 5, 0,
                     mask=orc.PROC_BH)
    assert st["rc"] == 0 and st["status"] == 2
    assert st["created"][4] == n and sp["ph"].n == 0
    tot = np.zeros(n)
    for key in ("em", "ep"):
        d = sp[key].as_dict()
        u = np.stack([d["ux"], d["uy"], d["uz"]], 1).astype(np.float64)[np.argsort(d["cell"])]
        assert np.allclose(_unit(u), dirs, atol=tol)
        tot += np.sqrt(1 + (u ** 2).sum(1))
    assert np.allclose(tot, k, rtol=tol)


@pytest.mark.slow
def test_thin_target_yield_independent_of_weight_ratio(orc):
    """Fig. valid_brem_tf: a 40 MeV beam in neutral Cu (n_e = 1e21 cm^-3,
    n_i = 8e22 cm^-3) radiates N_gamma = n_e n_i v sigma_B t photons
    (Eq. N_br_theo1) whatever the weight ratio W_i/W_e in {2, 1, 1/2}, and
    the spectrum follows dsigma_B/dk (Eq. N_br_theo2)."""
    g = 1.0 + 40.0 / 0.51099895
    v = C_LIGHT * math.sqrt(1 - 1 / g ** 2)
    steps, dt, n_cells = 6, 150e-15, 48
    yields, spectra = {}, {}
    for ratio in (2.0, 1.0, 0.5):
        wl = W.thin_target_beam(ratio, n_cells=n_cells, e_per_cell=64, seed=11, dt=dt)
        T, sp, ledger, st = _run(orc, wl, steps, orc.PROC_BREMS)
        ph = sp["ph"].as_dict()
        yields[ratio] = (ledger[:, 1].sum(), len(ph["w"]))
        spectra[ratio] = np.sqrt(ph["ux"].astype(float) ** 2 + ph["uy"] ** 2 + ph["uz"] ** 2)
    s = T.screening(0)
    Tk = g - 1
    f = lambda lx: orc.dsdk_brems(s, g, math.exp(lx) * Tk) * Tk * math.exp(lx)
    sigma = quad(f, math.log(1e-7), 0.0)
    n_e, n_i = 1e27, 8e28
    expected = n_e * n_i * v * sigma * steps * dt * n_cells       # sum of photon weights over cells
    for ratio, (wsum, count) in yields.items():
        rel_err = 1 / math.sqrt(count)
        assert abs(wsum / expected - 1) < 4 * rel_err + 0.01, (ratio, wsum / expected, count)
    # spectrum (all ratios pooled) vs dsigma/dk: chi-square in log-k bins
    ks = np.concatenate(list(spectra.values()))
    edges = np.exp(np.linspace(math.log(1e-4 * Tk), math.log(Tk), 9))
    obs = np.histogram(ks, edges)[0]
    probs = np.array([quad(f, math.log(a / Tk), math.log(b / Tk)) for a, b in zip(edges[:-1], edges[1:])]) / sigma
    exp_counts = probs / probs.sum() * obs.sum()
    chi2 = ((obs - exp_counts) ** 2 / exp_counts).sum()
    assert stats.chi2.sf(chi2, len(obs) - 1) > 0.01


@pytest.mark.slow
def test_thin_target_bh_yield_independent_of_weight_ratio(orc):
    """The Bethe-Heitler counterpart of Fig. valid_brem_tf: a 100 MeV photon
    beam in neutral Cu (n_gamma = 1e21 cm^-3, n_i = 8e22 cm^-3) converts
    n_gamma (1 - (1 - q)^S) photons into pairs in S steps, q = n_i c
    sigma_BH dt (a converted photon is absorbed), whatever W_i/W_gamma in
    {2, 1, 1/2}; the positron energies follow dsigma_BH/dgamma_+ (Eq. dsdkbh)."""
    k = 100.0 / 0.51099895
    steps, dt, n_cells = 8, 4e-13, 256
    yields, spectra = {}, {}
    for ratio in (2.0, 1.0, 0.5):
        wl = W.thin_target_photon_beam(ratio, n_cells=n_cells, g_per_cell=64, seed=13, dt=dt)
        T, sp, ledger, st = _run(orc, wl, steps, orc.PROC_BH)
        ep, em = sp["ep"].as_dict(), sp["em"].as_dict()
        assert len(ep["w"]) == len(em["w"])
        yields[ratio] = (ep["w"].astype(float).sum(), len(ep["w"]))
        spectra[ratio] = np.sqrt(1.0 + ep["ux"].astype(float) ** 2 + ep["uy"] ** 2 + ep["uz"] ** 2)
    s = T.screening(0)
    sigma = quad(lambda gp: orc.dsdg_bh(s, k, gp), 1.0, k - 1.0)
    q = 8e28 * C_LIGHT * sigma * dt
    expected = 1e27 * (1.0 - (1.0 - q) ** steps) * n_cells        # sum of positron weights over cells
    for ratio, (wsum, count) in yields.items():
        print(f"\n[thin target BH] W_i/W_g = {ratio}: yield / theory = {wsum / expected:.4f} ({count} pairs)")
        assert count > 300
        assert abs(wsum / expected - 1) < 4 / math.sqrt(count) + 0.01, (ratio, wsum / expected, count)
    gp = np.concatenate(list(spectra.values()))
    edges = np.linspace(1.0, k - 1.0, 9)
    obs = np.histogram(gp, edges)[0]
    probs = np.array([quad(lambda g: orc.dsdg_bh(s, k, g), a, b) for a, b in zip(edges[:-1], edges[1:])]) / sigma
    exp_counts = probs / probs.sum() * obs.sum()
    chi2 = ((obs - exp_counts) ** 2 / exp_counts).sum()
    assert stats.chi2.sf(chi2, len(obs) - 1) > 0.01


@pytest.mark.slow
def test_thin_target_trident_yield_independent_of_weight_ratio(orc):
    """Coulomb Trident in the same thin target: a 500 MeV electron beam
    creates n_e n_i v sigma_T t pairs per unit volume (Gryaznykh fit of
    Sec. II.D), whatever W_i/W_e in {2, 1, 1/2}.  One step: the pairs created
    in a step become projectiles only after it, so a single step counts no
    cascade of secondary Tridents (which several steps would add at second
    order), and a recoiled electron's later pairs change sigma_T only at
    second order in its ~4 % conversion probability."""
    g = 1.0 + 500.0 / 0.51099895
    v = C_LIGHT * math.sqrt(1.0 - 1.0 / g ** 2)
    steps, dt, n_cells = 1, 3.2e-11, 256
    sigma = orc.sigma_trident(29, g)
    expected = 1e27 * 8e28 * v * sigma * steps * dt * n_cells
    for ratio in (2.0, 1.0, 0.5):
        wl = W.thin_target_beam(ratio, n_cells=n_cells, e_per_cell=64, seed=14, dt=dt, gamma=g)
        T, sp, ledger, st = _run(orc, wl, steps, orc.PROC_TRIDENT)
        ep = sp["ep"].as_dict()
        wsum, count = ep["w"].astype(float).sum(), len(ep["w"])
        print(f"\n[thin target Trident] W_i/W_e = {ratio}: yield / theory = {wsum / expected:.4f} ({count} pairs)")
        assert count > 300
        assert abs(wsum / expected - 1) < 4 / math.sqrt(count) + 0.015, (ratio, wsum / expected, count)


@pytest.mark.slow
def test_radiative_stopping_power_mc(orc):
    """The MC energy radiated per electron per unit length equals
    n_i int k dsigma/dk dk (Sec. III.B), within the MC error."""
    g = 1.0 + 40.0 / 0.51099895
    wl = W.thin_target_beam(1.0, n_cells=48, e_per_cell=64, seed=12, dt=150e-15)
    T, sp, ledger, st = _run(orc, wl, 6, orc.PROC_BREMS)
    ph = sp["ph"].as_dict()
    k = np.sqrt(ph["ux"].astype(float) ** 2 + ph["uy"] ** 2 + ph["uz"] ** 2)
    s = T.screening(0)
    Tk = g - 1
    f1 = lambda lx: orc.dsdk_brems(s, g, math.exp(lx) * Tk) * Tk * math.exp(lx)
    fk = lambda lx: f1(lx) * math.exp(lx) * Tk
    mean_k = quad(fk, math.log(1e-7), 0.0) / quad(f1, math.log(1e-7), 0.0)
    assert k.mean() == pytest.approx(mean_k, rel=4 * k.std() / k.mean() / math.sqrt(len(k)))
    # the ledger records the same radiated energy as the photons carry
    assert ledger[:, 0].sum() == pytest.approx((k * ph["w"]).sum(), rel=1e-6)


@pytest.mark.parametrize("mask,dt,boost", [(7, 50e-15, 8.0), (2, 3e-11, 60.0), (4, 1e-11, 1.0)])
def test_step_conserves_energy_and_charge(orc, mask, dt, boost):
    """With ions at rest every process conserves sum W*E (leptons with rest
    mass, photons k) and sum W*q; float32 storage bounds the drift.  The
    Trident-only and BH-only cases use long steps so that they fire."""
    wl = W.solid_cu(n_cells=24, e_per_cell=48, i_per_cell=16, seed=5, dt=dt, photons_per_cell=24)
    for c in ("ux", "uy", "uz"):
        wl.species["ion"][c][:] = 0
        wl.species["em"][c] *= boost

    def totals(sp):
        E = Q = 0.0
        for name, q in (("em", -1), ("ep", 1), ("ph", 0)):
            d = sp[name].as_dict()
            u2 = d["ux"].astype(float) ** 2 + d["uy"].astype(float) ** 2 + d["uz"].astype(float) ** 2
            e = np.sqrt(u2) if name == "ph" else np.sqrt(1 + u2)
            E += (d["w"] * e).sum()
            Q += q * d["w"].astype(float).sum()
        return E, Q

    spec = orc.table_spec(n_rows=96, n_cols=96)
    T = orc.OracleTables([orc.material(29, 5, 8.5e28, 100.0)], spec)
    sp = {k: orc.OracleSpecies(v, cap=len(v["w"]) + 50000) for k, v in wl.species.items()}
    E0, Q0 = totals(sp)
    created = np.zeros(5)
    for s in range(3):
        _, st = orc.step(T, wl.n_cells, wl.material_of_cell, sp["em"], sp["ep"], sp["ph"], sp["ion"],
                         wl.ion_mass, wl.dt, wl.seed, s, mask)
        created += st["created"]
    E1, Q1 = totals(sp)
    if mask == 7:
        assert created[0] > 20
    if mask == 4:
        assert created[4] > 20 and sp["ep"].n > 20
    if mask == 2:
        assert created[2] > 20 and sp["ep"].n > 20
    assert E1 == pytest.approx(E0, rel=1e-6)
    assert Q1 == pytest.approx(Q0, rel=1e-12)


def test_step_deterministic_and_cell_sharded(orc):
    """Random numbers are keyed by (seed, step, cell, slot), so the result does
    not depend on storage order or on which cells a call covers: running the
    two halves of the cells separately gives bit-identical particles."""
    wl = W.solid_cu(n_cells=16, e_per_cell=40, i_per_cell=24, seed=7, dt=400e-15, photons_per_cell=20)
    spec = orc.table_spec(n_rows=64, n_cols=64)
    T = orc.OracleTables([orc.material(29, 5, 8.5e28, 100.0)], spec)

    def run(species, cells):
        sub = {}
        for k, d in species.items():
            keep = np.isin(d["cell"], cells)
            sub[k] = {f: (v[keep] if v is not None else None) for f, v in d.items()}
        sp = {k: orc.OracleSpecies(v, cap=len(v["w"]) + 5000) for k, v in sub.items()}
        orc.step(T, wl.n_cells, wl.material_of_cell, sp["em"], sp["ep"], sp["ph"], sp["ion"],
                 wl.ion_mass, wl.dt, wl.seed, 3)
        return {k: sp[k].canonical() for k in ("em", "ep", "ph")}

    full = run(wl.species, np.arange(16))
    a = run(wl.species, np.arange(8))
    b = run(wl.species, np.arange(8, 16))
    # shuffled storage order
    rng = np.random.default_rng(1)
    shuffled = {}
    for k, d in wl.species.items():
        p = rng.permutation(len(d["w"]))
        shuffled[k] = {f: (v[p] if v is not None else None) for f, v in d.items()}
    sh = run(shuffled, np.arange(16))
    for k in ("em", "ep", "ph"):
        for f in ("ux", "uy", "uz", "w", "pid", "cell"):
            joined = np.concatenate([a[k][f], b[k][f]])
            assert np.array_equal(full[k][f], joined)
            assert np.array_equal(full[k][f], sh[k][f])
    assert len(full["ph"]["w"]) > 16 * 20      # Brems photons were created


def test_case_b_pairs_each_target_once(orc):
    """N_t > N_p: every ion takes part in exactly one macro-collision and each
    electron in ceil/floor(N_t/N_p) of them (Sec. III.A, N_ei = max)."""
    rk = orc.philox([0, 3, 1, 2], [5, 6])
    Np, Nt = 7, 45
    targets = [orc.perm_elem(j, Nt, rk) for j in range(Nt)]
    assert sorted(targets) == list(range(Nt))
    per_e = np.bincount([j % Np for j in range(Nt)], minlength=Np)
    assert per_e.max() - per_e.min() <= 1


# ---------------------------------------------------- accept decision ---
def test_accept_decision_is_exact(orc):
    """The accept decision compares U = (2^48 a + e + 1/2) 2^-64 with the
    collision probability p exactly, e = 2^16 w0 + (w1 >> 16) from the
    extension draw: checked in rational arithmetic for probabilities from
    1e-15 to 1 - 1e-9, with the 16-bit digit a on, just below and just above
    floor(2^16 p) (the tie reads e)."""
    from fractions import Fraction
    rng = np.random.default_rng(5)
    seed, cell, step = 0x1234ABCD5678, 77, 9
    ps = [1e-15, 3.3e-11, 2.0 ** -32, 2.0 ** -16, 7.7e-10, 1.234e-7, 5.9e-8, 1.5e-5, 0.01, 0.5, 1.0 - 1e-9] \
        + list(rng.uniform(0, 1e-3, 20))
    n = 0
    for p in ps:
        fl = int(Fraction(p) * 2 ** 16)
        for a in {max(fl - 1, 0), fl, min(fl + 1, 2 ** 16 - 1), int(rng.integers(0, 2 ** 16))}:
            for _ in range(2):
                c0, tg = int(rng.integers(0, 1 << 17)), 1 | (6 << 4) | (2 << 8)
                w = orc.philox([c0, cell, step, tg], [seed & 0xFFFFFFFF, seed >> 32])
                e = (w[0] << 16) | (w[1] >> 16)
                exact = Fraction(2 ** 48 * a + e) + Fraction(1, 2) < Fraction(p) * 2 ** 64
                assert orc.accept(a, p, c0, cell, step, tg, seed) == exact, (p, a)
                n += 1
    assert n > 150
    assert not orc.accept(0, 0.0, 0, 0, 0, 0, 0) and orc.accept(2 ** 16 - 1, 1.0, 0, 0, 0, 0, 0)
    with pytest.raises(ValueError):
        orc.accept(1 << 16, 0.5, 0, 0, 0, 0, 0)


def test_tiny_probabilities_are_honoured(orc):
    """A per-pair probability far below the 23-bit resolution of the event
    uniforms is still taken at its value: over all 2^16 first digits the
    decision accepts floor(2^16 p) of them outright and leaves exactly one to
    the rest e, so P(accept) = p to 2^-64."""
    for p in (3e-11, 2.5e-9, 4e-8, 1e-3):
        fl = math.floor(p * 2 ** 16)
        assert orc.accept(fl - 1, p, 0, 0, 0, 0, 0) if fl > 0 else True
        assert not orc.accept(fl + 1, p, 0, 0, 0, 0, 0)
        # the tie: over many extension draws the fraction accepted is frac(2^16 p)
        acc = sum(orc.accept(fl, p, c0, 1, 2, 3, 99) for c0 in range(4000))
        frac = p * 2 ** 16 - fl
        assert abs(acc / 4000 - frac) < 4 * math.sqrt(frac * (1 - frac) / 4000) + 1e-3
