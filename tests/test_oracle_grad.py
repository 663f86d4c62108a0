"""Pins of the oracle's analytic gradient of the expected-emission operator
(the chain rule written out by hand, orc_expected_emission_grad_analytic),
each against something that does not come from the hand derivation:
  - d I1/dL and d I2/dL of the reduced screening functions against
    30-digit quadrature of the L-derivative of their integral definitions
    (Eqs. defphi1, defphi2 with the single-Yukawa form factor of Eq. defF);
  - the Jacobian of (L_TF, L_D, eta_D, L_R) against central differences of
    the oracle's own screening preparation (Eqs. LTF, LDH, ITFD, reduit);
  - the contracted gradient against the Richardson-extrapolated central
    differences of the FP64 operator, on both branches of max(lambda_D, r_i),
    at Z* = Z, and on non-relativistic, relativistic and ultra-relativistic
    samples;
  - at Z* = 0 the Z* component against one-sided differences from Z* > 0
    (the reading: lambda_D -> infinity there, and the derivative is the
    limit from the right)."""
import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")

NAMES = ("n_i", "T_e", "Zstar", "s_TF", "s_D")


def contracted(orc, mat, g, w, gout):
    return float(np.dot(gout, orc.expected_emission(mat, g, w)))


def with_param(orc, mat, k, v):
    p = {n: getattr(mat, n) for n in NAMES}
    p[NAMES[k]] = v
    return orc.material(mat.Z, p["Zstar"], p["n_i"], p["T_e"], p["s_TF"], p["s_D"])


@pytest.mark.parametrize("delta,L", [(1e-5, 54.0), (1e-3, 54.0), (0.05, 54.0), (0.07, 54.0), (0.4, 54.0),
                                     (1e-3, 5.0), (0.02, 5.0), (1e-4, 300.0), (0.01, 300.0), (0.3, 300.0),
                                     (0.9, 1000.0), (0.5, 2000.0)])
def test_dI12_dL_against_the_integral_definitions(orc, delta, L):
    """I1 = int_delta^1 (u - delta)^2/u^3 (1 - F)^2 du and I2 = int_delta^1
    [u^3 - 6 delta^2 u ln(u/delta) + 3 delta^2 u - 4 delta^3]/u^4 (1 - F)^2 du
    with 1 - F = (L u)^2/(1 + (L u)^2); their L-derivatives replace (1 - F)^2
    by 2 (1 - F) 2 L u^2/(1 + L^2 u^2)^2."""
    mp = mpmath.mp
    mp.dps = 30
    d, LL = mp.mpf(delta), mp.mpf(L)

    def dF2(u):
        omf = (LL * u) ** 2 / (1 + (LL * u) ** 2)
        return 2 * omf * 2 * LL * u ** 2 / (1 + (LL * u) ** 2) ** 2

    k1 = lambda u: (u - d) ** 2 / u ** 3 * dF2(u)
    k2 = lambda u: (u ** 3 - 6 * d ** 2 * u * mp.log(u / d) + 3 * d ** 2 * u - 4 * d ** 3) / u ** 4 * dF2(u)
    pts = sorted({d, max(d, 1 / LL), 1})
    pts = [p for p in pts if d <= p <= 1]
    r1 = float(mp.quad(k1, pts))
    r2 = float(mp.quad(k2, pts))
    a1, a2 = orc.dI12_dL(delta, L)
    assert abs(a1 - r1) <= 1e-11 * abs(r1), (a1, r1)
    assert abs(a2 - r2) <= 1e-11 * abs(r2), (a2, r2)


MATERIALS = [
    (29, 5.0, 8.5e28, 100.0, "r_i branch, solid Cu"),
    (29, 5.0, 1e25, 5e3, "Debye branch"),
    (29, 29.0, 3e27, 2e3, "Z* = Z"),
    (13, 13.0, 6e28, 1e4, "Al fully ionized, Debye branch"),
    (73, 20.0, 1e26, 1e3, "Ta"),
    (29, 14.0, 2e27, 300.0, "mid ionization"),
]


@pytest.mark.parametrize("Z,Zs,n_i,T_e,label", MATERIALS)
def test_screening_jacobian_against_differences(orc, Z, Zs, n_i, T_e, label):
    mat = orc.material(Z, Zs, n_i, T_e, 1.1, 0.9)
    s = orc.screening(mat)
    assert abs(s.lambdaD / s.ri - 1.0) > 0.05
    J = orc.screening_jacobian(mat)

    def S(m):
        q = orc.screening(m)
        return np.array([q.LTF, q.LD, q.etaD, q.LR])

    for k in range(5):
        v = getattr(mat, NAMES[k])
        h = 1e-5 * v
        fd = (S(with_param(orc, mat, k, v + h)) - S(with_param(orc, mat, k, v - h))) / (2 * h)
        scale = np.abs(S(mat)) / v
        np.testing.assert_allclose(J[:, k], fd, rtol=1e-7, atol=1e-9 * scale.max(), err_msg=f"{label} {NAMES[k]}")


def sample_set(rng, kind, n=16):
    lo, hi = {"nr": (0.01, 0.5), "rel": (1.2, 48.0), "ur": (60.0, 400.0), "mix": (0.05, 200.0)}[kind]
    T = 10.0 ** rng.uniform(np.log10(lo), np.log10(hi), n) / 0.51099895
    return 1.0 + T, rng.uniform(0.5, 2.0, n)


@pytest.mark.parametrize("kind", ["nr", "rel", "ur", "mix"])
@pytest.mark.parametrize("Z,Zs,n_i,T_e,label", MATERIALS)
def test_analytic_gradient_against_richardson_differences(orc, Z, Zs, n_i, T_e, label, kind):
    """|theta_k (analytic_k - fd_k)| <= 1e-7 (|f| + |theta_k fd_k|)."""
    rng = np.random.default_rng([Z, int(Zs), ("nr", "rel", "ur", "mix").index(kind)])
    g, w = sample_set(rng, kind)
    mat = orc.material(Z, Zs, n_i, T_e, 1.05, 0.95)
    gout = rng.uniform(0.5, 1.5, 3)
    a = orc.expected_emission_grad_analytic(mat, g, w, gout)
    fd = orc.expected_emission_grad(mat, g, w, gout)
    f = contracted(orc, mat, g, w, gout)
    th = np.array([getattr(mat, n) for n in NAMES])
    err = np.abs(th * (a - fd))
    assert np.all(err <= 1e-7 * (abs(f) + np.abs(th * fd))), (label, kind, a, fd)
    assert np.any(np.abs(th * a) > 1e-4 * abs(f))   # something depends on the screening


@pytest.mark.parametrize("Z,n_i,T_e", [(29, 8.5e28, 100.0), (73, 5.55e28, 1e3), (13, 1e26, 1e4)])
def test_zstar_zero_is_the_limit_from_the_right(orc, Z, n_i, T_e):
    """At Z* = 0 the forward does not depend on L_D, and the Z* derivative is
    the limit of one-sided differences (f(h) - f(0))/h as h -> 0+; the other
    components equal central differences."""
    rng = np.random.default_rng(Z)
    g, w = sample_set(rng, "mix", 24)
    mat = orc.material(Z, 0.0, n_i, T_e)
    gout = rng.uniform(0.5, 1.5, 3)
    a = orc.expected_emission_grad_analytic(mat, g, w, gout)
    f0 = contracted(orc, mat, g, w, gout)
    D = []
    for h in (1e-4, 1e-5, 1e-6, 1e-7):
        D.append((contracted(orc, with_param(orc, mat, 2, h), g, w, gout) - f0) / h)
    D = np.array(D)
    # the differences converge to the analytic value as h ln h
    errs = np.abs(D - a[2])
    assert errs[-1] < errs[0] and errs[-1] <= 2e-5 * abs(a[2]), (D, a[2])
    for k in (0, 1, 3, 4):
        v = getattr(mat, NAMES[k])
        h = 1e-4 * v
        fd = (contracted(orc, with_param(orc, mat, k, v + h), g, w, gout)
              - contracted(orc, with_param(orc, mat, k, v - h), g, w, gout)) / (2 * h)
        assert abs(v * (a[k] - fd)) <= 1e-6 * abs(f0), (NAMES[k], a[k], fd)
    assert a[1] == 0.0 and a[4] == 0.0      # nothing depends on T_e or s_D without a Debye term
