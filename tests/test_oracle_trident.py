"""Pins of the oracle's Trident shapes (Sec. II.D) against results that do
not come from the oracle itself.

- Pair-energy spectrum, relativistic side: integrated over the pair energy
  at large gamma_1, the high-energy Bhabha form gives the Landau-Lifshitz
  leading-logarithm total (28 / 27 pi) (Z alpha r_e)^2 ln^3 gamma_1 (the
  integral of ln g ln(gamma_1/g) / g over ln g is ln^3 gamma_1 / 6).  The
  oracle's spectrum must approach it with a deficit falling as 1/ln^2.
- Pair-energy spectrum, threshold side: the product-over-sum interpolation
  reduces to the low-energy Bhabha form, E_p^3 times a bracket whose
  corrections C, C_r, C_z vanish as 1/gamma_1 -> 0.
- The Gryaznykh fit of the total against the same leading-log total: the
  paper notes the fit may be about 4 times the exact cross section.
- The pair-energy CDF tables against adaptive quadrature.
- Split CDF: the shape is a quadratic times a logarithm, so its CDF has an
  exact antiderivative in elementary functions, written out here in a form
  the oracle does not use; the oracle's tables (Gauss-Legendre panels) must
  agree with it at every column.
"""
import math

import numpy as np
import pytest

ALPHA = 7.2973525693e-3
R_E = 2.8179403262e-15


def _integral_over_pair_energy(orc, Z, g1):
    from scipy.integrate import quad
    f = lambda t: orc.dsdgp_trident(Z, g1, math.exp(t)) * math.exp(t)
    cuts = [math.log(2.0 + 1e-12), math.log(3.0), math.log(10.0), math.log(100.0), math.log(g1 - 1.0)]
    return sum(quad(f, a, b, epsrel=1e-11, limit=400)[0] for a, b in zip(cuts, cuts[1:]))


def test_pair_spectrum_integrates_to_landau_lifshitz(orc):
    Z = 29
    ll_coef = 28.0 / (27.0 * math.pi) * (Z * ALPHA * R_E) ** 2
    scaled = []
    for g1 in (1e4, 1e6, 1e9, 1e12):
        L = math.log(g1)
        ratio = _integral_over_pair_energy(orc, Z, g1) / (ll_coef * L ** 3)
        # below the leading log by the threshold region (about 6.5 / L^2)
        assert 1.0 - 8.0 / L ** 2 < ratio < 1.0, (g1, ratio)
        scaled.append((ratio - 1.0) * L * L)
    # the deficit times L^2 settles: it is a subleading term, not a wrong prefactor
    assert max(scaled) - min(scaled) < 1.0
    # Z^2 scaling
    assert _integral_over_pair_energy(orc, 58, 1e6) == pytest.approx(4 * _integral_over_pair_energy(orc, 29, 1e6),
                                                                      rel=1e-9)


def test_pair_spectrum_threshold_is_low_energy_bhabha(orc):
    Z = 29
    pre = (Z * ALPHA * R_E) ** 2
    for g1, tol in ((1e2, 1e-3), (1e4, 1e-6), (1e8, 1e-9)):
        # C + C_r + C_z = O(x^2 ln(1/x^2)), x = 1/gamma_1
        lead = pre / 32.0 * (2.0 * math.log(g1) - 161.0 / 60.0)
        for eps in (1e-4, 1e-6):
            assert orc.dsdgp_trident(Z, g1, 2.0 + eps) / eps ** 3 == pytest.approx(lead, rel=tol), (g1, eps)
    # cubic rise: doubling E_p near threshold multiplies the spectrum by 8
    assert orc.dsdgp_trident(Z, 1e3, 2.0 + 2e-5) / orc.dsdgp_trident(Z, 1e3, 2.0 + 1e-5) == pytest.approx(8.0, rel=1e-4)


def test_fit_against_leading_log(orc):
    """The fit of the total over the leading-log total rises with gamma_1
    towards a constant between 3 and 5, the paper's 'about 4 times' (a wrong
    power of ten, power of Z or of the log would miss that band)."""
    Z = 29
    ratios = []
    for g1 in (1e6, 1e12, 1e40, 1e300):
        ll = 28.0 / (27.0 * math.pi) * (Z * ALPHA * R_E) ** 2 * math.log(g1) ** 3
        ratios.append(orc.sigma_trident(Z, g1) / ll)
    assert all(a < b for a, b in zip(ratios, ratios[1:]))
    assert 3.0 < ratios[-1] < 5.0
    assert orc.sigma_trident(2 * Z, 1e12) == pytest.approx(4.0 * orc.sigma_trident(Z, 1e12), rel=1e-14)


def _split_cdf_exact(y, p):
    """CDF in y of the clamped split shape at pair energy p = gamma_p, with
    gamma_+ = 1 + y (p - 2).  The shape (a^2 + (p-a)^2 + 2/3 a (p-a)) equals
    P(a) = 4/3 a^2 - 4/3 p a + p^2, symmetric under a -> p - a, and the log
    is positive between the roots a_-+ of a^2 - p a + p (none for p <= 4,
    where the split is uniform)."""
    if p <= 4.0:
        return y
    c = (p * p, -4.0 / 3.0 * p, 4.0 / 3.0)

    def h(x):        # antiderivative of P(x) ln x
        return sum(cn * (x ** (n + 1) * math.log(x) / (n + 1) - x ** (n + 1) / (n + 1) ** 2) for n, cn in enumerate(c))

    def g(a):        # antiderivative of P(a) [ln a + ln(p - a) - ln p]
        return h(a) - h(p - a) - math.log(p) * sum(cn * a ** (n + 1) / (n + 1) for n, cn in enumerate(c))

    d = math.sqrt(p * p - 4.0 * p)
    am, ap = 0.5 * (p - d), 0.5 * (p + d)
    a = min(max(1.0 + y * (p - 2.0), am), ap)
    return (g(a) - g(am)) / (g(ap) - g(am))


# The clamped shape's slope jumps where the log crosses zero; a Gauss panel
# that holds the jump converges as its width squared, hence the tolerance
# per column count (worst rows: 6.3e-6 at 64 columns, 4.2e-7 at 256).
@pytest.mark.parametrize("n_cols,tol", [(64, 2e-5), (256, 2e-6)])
def test_split_cdf_matches_exact_antiderivative(orc, n_cols, tol):
    T = orc.OracleTables([orc.material(29, 5, 8.5e28, 100.0)], orc.table_spec(n_rows=64, n_cols=n_cols))
    ys = [T.col_value(orc.TB_TRI_SPLIT, c) for c in range(n_cols)]
    checked_nonuniform = 0
    for r in range(64):
        p = 2.0 + T.row_value(r)
        exact = np.array([_split_cdf_exact(y, p) for y in ys])
        assert np.abs(T.tri_split_cdf[r] - exact).max() < tol, (r, p)
        checked_nonuniform += p > 4.0
    assert checked_nonuniform > 20


def test_pair_energy_cdf_matches_adaptive_quadrature(orc):
    """The pair-energy table rows (graded Gauss-Legendre panels in ln y)
    against adaptive quadrature of the same spectrum."""
    from scipy.integrate import quad
    T = orc.OracleTables([orc.material(29, 5, 8.5e28, 100.0)], orc.table_spec(n_rows=32, n_cols=48))
    ys = np.array([T.col_value(orc.TB_TRI_GP, c) for c in range(48)])
    for r in (4, 12, 20, 31):
        rowv = T.row_value(r)
        g1 = 3.0 + rowv
        f = lambda t: orc.dsdgp_trident(1, g1, 2.0 + math.exp(t) * rowv) * math.exp(t)
        parts = [quad(f, math.log(a), math.log(b), epsrel=1e-12, limit=200)[0] for a, b in zip(ys, ys[1:])]
        cum = np.concatenate([[0.0], np.cumsum(parts)])
        assert np.allclose(T.tri_gp_cdf[r], cum / cum[-1], rtol=0, atol=1e-7), r
