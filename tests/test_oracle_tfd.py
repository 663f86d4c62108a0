"""Pins of the oracle's TFD-quadrature screening mode: the screening
functions I1, I2 of Eqs. (defphi1), (defphi2) with the form factor
(Eq. defF) of the full Thomas-Fermi-Debye potential (Eq. V_TFD), by
quadrature, and the tables built with them.

- Z* = 0 and Z* = Z leave one Yukawa term, where Eqs. (deriv_I1),
  (deriv_I2) give I1, I2 in closed form (evaluated here at 50 digits);
- delta -> 0 gives the closed form of Eq. (ITFD), cross term included;
- between them, a 30-digit tanh-sinh quadrature of the definitions, with
  the form factor written out here from Eq. (V_TFD);
- at Z* = 0 the reduced potential is the Thomas-Fermi one, and the two
  modes' tables coincide (the paper says so for neutral atoms); elsewhere
  the reduced formula stays close to the full potential (Sec. II.B.2-3,
  Sec. II.C, figs. cs_br_re_io, cs_br_ur_io, cs_bh_pp)."""
import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

DELTAS = [1e-12, 1e-8, 1e-5, 1e-3, 3e-2, 0.3, 0.7]


def closed_I12(d, L):
    """Eqs. (deriv_I1), (deriv_I2) for one Yukawa term of length L, 50 digits."""
    mp.mp.dps = 50
    d, L = mp.mpf(d), mp.mpf(L)
    L2, d2 = L * L, d * d
    I1 = L * d * (mp.atan(d * L) - mp.atan(L)) - L2 / 2 * (1 - d) ** 2 / (1 + L2) \
        + mp.log((1 + L2) / (1 + L2 * d2)) / 2
    two_I2 = 4 * L2 * L * d2 * d * (mp.atan(L * d) - mp.atan(L)) \
        + (1 + 3 * L2 * d2) * mp.log((1 + L2) / (1 + L2 * d2)) \
        + 6 * L2 * L2 * d2 / (1 + L2) * mp.log(d) \
        + L2 * (d - 1) * (d + 1 - 4 * L2 * d2) / (1 + L2)
    return float(I1), float(two_I2 / 2)


def defined_I12(d, s):
    """Eqs. (defphi1), (defphi2) with 1 - F(u) = sum_i (q_i/q) (L_i u)^2/(1 + (L_i u)^2)
    (the Fourier transform of each Yukawa term of Eq. V_TFD), 30 digits."""
    mp.mp.dps = 30
    d = mp.mpf(d)
    LTF, LD, eTF, eD = (mp.mpf(v) for v in (s.LTF, s.LD, s.etaTF, s.etaD))

    def one_minus_F(u):
        a, b = (LTF * u) ** 2, (LD * u) ** 2
        return eTF * a / (1 + a) + eD * b / (1 + b)

    f1 = lambda u: (u - d) ** 2 / u ** 3 * one_minus_F(u) ** 2
    f2 = lambda u: (u ** 3 - 6 * d * d * u * mp.log(u / d) + 3 * d * d * u - 4 * d ** 3) / u ** 4 * one_minus_F(u) ** 2
    pts = [d] + sorted(p for p in (1 / LD, 1 / LTF, 10 / LTF, 10 / LD) if d < p < 1) + [mp.mpf(1)]
    return float(mp.quad(f1, pts)), float(mp.quad(f2, pts))


def closed_I_tfd(s):
    """Eq. (ITFD)."""
    mp.mp.dps = 40
    A, B = mp.mpf(s.LTF) ** 2, mp.mpf(s.LD) ** 2
    eTF, eD = mp.mpf(s.etaTF), mp.mpf(s.etaD)
    h = lambda X: ((1 + X) * mp.log(1 + X) - X) / (1 + X)
    return float(eTF ** 2 / 2 * h(A) + eD ** 2 / 2 * h(B) + eTF * eD * (B * mp.log(1 + A) - A * mp.log(1 + B)) / (B - A))


def cu(orc, Zs, T):
    return orc.material(29, Zs, 8.5e28, T)


@pytest.mark.parametrize("Zs,T,which", [(0.0, 0.0, "LTF"), (29.0, 1e3, "LD"), (29.0, 30.0, "LD")])
def test_single_yukawa_limits_match_closed_forms(orc, Zs, T, which):
    s = orc.screening_tfd(cu(orc, Zs, max(T, 1e-3)))
    L = getattr(s, which)
    for d in DELTAS:
        q1, q2 = orc.I12_tfd_quad(s, d)
        c1, c2 = closed_I12(d, L)
        np.testing.assert_allclose(q1, c1, rtol=1e-10, err_msg=f"I1 delta={d}")
        np.testing.assert_allclose(q2, c2, rtol=1e-10, err_msg=f"I2 delta={d}")


@pytest.mark.parametrize("Zs,T", [(3.0, 30.0), (10.0, 1e3), (20.0, 1e4)])
def test_small_delta_limit_is_I_tfd(orc, Zs, T):
    s = orc.screening_tfd(cu(orc, Zs, T))
    ref = closed_I_tfd(s)
    q1, q2 = orc.I12_tfd_quad(s, 1e-15)
    # I(delta) - I(0) = O(delta L) for both
    np.testing.assert_allclose(q1, ref, rtol=1e-10)
    np.testing.assert_allclose(q2, ref, rtol=1e-10)


@pytest.mark.parametrize("Zs,T", [(5.0, 100.0), (14.0, 5e3)])
def test_mixed_potential_matches_high_precision_quadrature(orc, Zs, T):
    s = orc.screening_tfd(cu(orc, Zs, T))
    for d in (1e-9, 1e-5, 1e-3, 5e-2, 0.5):
        q1, q2 = orc.I12_tfd_quad(s, d)
        r1, r2 = defined_I12(d, s)
        np.testing.assert_allclose(q1, r1, rtol=1e-10, err_msg=f"I1 delta={d}")
        np.testing.assert_allclose(q2, r2, rtol=1e-10, err_msg=f"I2 delta={d}")


def test_outside_range_is_zero(orc):
    s = orc.screening_tfd(cu(orc, 5.0, 100.0))
    assert orc.I12_tfd_quad(s, 1.0) == (0.0, 0.0)
    assert orc.I12_tfd_quad(s, 2.0) == (0.0, 0.0)


def tables(orc, Zs, T, screening, n=64):
    return orc.OracleTables([cu(orc, Zs, max(T, 1e-3))], orc.table_spec(n_rows=n, n_cols=n, screening=screening))


def test_neutral_atoms_tables_coincide(orc):
    """Z* = 0: L_R = L_TF, so both modes give the same tables (to the closed
    forms' rounding near delta ~ 1, where Eq. deriv_I2 cancels)."""
    R, Q = tables(orc, 0.0, 0.0, orc.SCREEN_REDUCED), tables(orc, 0.0, 0.0, orc.SCREEN_TFD_QUAD)
    np.testing.assert_allclose(Q.brems_sigma, R.brems_sigma, rtol=1e-9)
    np.testing.assert_allclose(Q.bh_sigma, R.bh_sigma, rtol=1e-9)
    np.testing.assert_allclose(Q.brems_cdf, R.brems_cdf, rtol=1e-8, atol=1e-12)
    np.testing.assert_allclose(Q.bh_cdf, R.bh_cdf, rtol=1e-8, atol=1e-12)


@pytest.mark.parametrize("Zs,T", [(5.0, 100.0), (14.0, 5e3), (20.0, 1e4)])
def test_reduced_formula_stays_close_to_full_potential(orc, Zs, T):
    """The reduced potential matches the delta -> 0 limit exactly and departs
    from the full one at finite delta by well under the paper's plotted
    differences: below 1 % on the Brems total cross sections (gamma > 2;
    the non-relativistic rows use the full potential in both modes) and 3 %
    on the BH ones, for Cu from 100 eV to 10 keV."""
    R, Q = tables(orc, Zs, T, orc.SCREEN_REDUCED), tables(orc, Zs, T, orc.SCREEN_TFD_QUAD)
    g = np.array([1.0 + R.row_value(r) for r in range(64)])
    nr = g <= 2.0
    np.testing.assert_array_equal(Q.brems_sigma[0, nr], R.brems_sigma[0, nr])
    db = np.abs(R.brems_sigma[0, ~nr] / Q.brems_sigma[0, ~nr] - 1.0)
    dh = np.abs(R.bh_sigma[0] / Q.bh_sigma[0] - 1.0)
    print(f"\n[TFD] Z*={Zs} T={T} eV: reduced vs full potential, Brems max {db.max():.2e}, BH max {dh.max():.2e}")
    assert db.max() < 1e-2 and dh.max() < 3e-2
    assert db.max() > 1e-5   # the modes do differ


def test_regime_boundary_jumps(orc):
    """The piecewise Brems model (non-relativistic up to 2, relativistic up
    to 100, ultra-relativistic above) jumps at gamma1 = 2 (Eq. cs_br_nr
    with the Elwert factor below, Eq. csre above) and at gamma1 = 100
    (Eq. csur adds f_C).  The k-integrated cross sections on both sides,
    for both screening modes: about +190 % at gamma1 = 2 (the extreme-
    relativistic form of Eq. csre taken at its lower end) and about -1 % at
    gamma1 = 100 (the size of f_C(29) against I1 + 1)."""
    from scipy import integrate

    def sigma(s, g):
        T = g - 1.0
        f = lambda lx: orc.dsdk_brems(s, g, np.exp(lx) * T) * np.exp(lx) * T
        pts = [np.log(1e-7), np.log(0.5), np.log(0.99), 0.0]
        return sum(integrate.quad(f, a, b, limit=400, epsrel=1e-10)[0] for a, b in zip(pts[:-1], pts[1:]))

    m = cu(orc, 5.0, 100.0)
    for s in (orc.screening(m), orc.screening_tfd(m)):
        j2 = sigma(s, 2.0 + 1e-9) / sigma(s, 2.0) - 1.0
        j100 = sigma(s, 100.0 + 1e-7) / sigma(s, 100.0) - 1.0
        print(f"\n[regimes] tfd_quad={s.tfd_quad}: jump at gamma1=2 {j2:+.3f}, at gamma1=100 {j100:+.4f}")
        assert 1.5 < j2 < 2.5
        assert -0.02 < j100 < -0.005
