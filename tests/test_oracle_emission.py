"""Pins of the oracle's expected-emission operator (the rate form of the
thin-target yield, Eq. N_br_theo1/2, and the radiative stopping power of
Sec. III.B) and of its FP64 gradient with respect to the plasma parameters
theta = (n_i, T_e, Z*, s_TF, s_D)."""
import numpy as np
import pytest

C_LIGHT = 299792458.0


def one_sample(orc, mat, gamma, n_quad=64):
    return orc.expected_emission(mat, np.array([gamma]), np.array([1.0]), n_quad=n_quad)


def speed(gamma):
    return C_LIGHT * np.sqrt(1.0 - 1.0 / gamma ** 2)


@pytest.mark.parametrize("row", [40, 90, 140, 200, 250])
def test_rate_equals_table_cross_section(orc, row):
    """out[0] of a single electron of unit weight is n_i v sigma_B(gamma): the
    operator's one-panel 64-point rule against the table build's composite
    graded rule (an independent quadrature of the same integral)."""
    mat = orc.material(29, 5.0, 8.5e28, 100.0)
    spec = orc.table_spec()
    T = orc.OracleTables([mat], spec)
    gamma = 1.0 + T.row_value(row)
    out = one_sample(orc, mat, gamma)
    sigma = T.brems_sigma[0, row]
    # one 64-point panel resolves the tip feature (width ~1/gamma in x) to
    # ~1e-5 at gamma = 1500 and far better below
    np.testing.assert_allclose(out[0] / (mat.n_i * speed(gamma)), sigma, rtol=1e-5)


@pytest.mark.parametrize("gamma", [1.6, 7.0, 60.0, 350.0])
def test_power_equals_quadrature_of_k_dsigma(orc, gamma):
    """out[2] / (n_i v) = int k dsigma/dk dk over k/(gamma-1) in [1e-7, 1], by
    adaptive quadrature in k with the tip as a breakpoint."""
    from scipy import integrate
    mat = orc.material(29, 10.0, 8.5e28, 1e3)
    s = orc.screening(mat)
    T = gamma - 1.0
    f = lambda lx: np.exp(lx) * T * orc.dsdk_brems(s, gamma, np.exp(lx) * T) * np.exp(lx) * T
    pts = [np.log(1e-7), np.log(0.5), np.log(0.9), np.log(0.99), 0.0]
    ref = sum(integrate.quad(f, a, b, epsabs=0, epsrel=1e-11, limit=400)[0] for a, b in zip(pts[:-1], pts[1:]))
    out = one_sample(orc, mat, gamma)
    np.testing.assert_allclose(out[2] / (mat.n_i * speed(gamma)), ref, rtol=5e-6)


def samples(rng, n=24):
    T = 10.0 ** rng.uniform(np.log10(0.5), np.log10(200.0), n) / 0.51099895
    return 1.0 + T, rng.uniform(0.5, 2.0, n)


def contracted(orc, mat, g, w, gout):
    return float(np.dot(gout, orc.expected_emission(mat, g, w)))


def test_gradient_debye_branch_homogeneity(orc):
    """Where lambda_D > r_i, L_D is proportional to s_D T_e^(1/2) n_i^(-1/2), so
    T_e df/dT_e = s_D df/ds_D / 2 and n_i df/dn_i = f - s_D df/ds_D / 2."""
    rng = np.random.default_rng(1)
    g, w = samples(rng)
    mat = orc.material(29, 5.0, 1e25, 5e3)
    s = orc.screening(mat)
    assert s.lambdaD > 1.05 * s.ri
    gout = np.array([1.0, 0.3, 0.02])
    d = orc.expected_emission_grad(mat, g, w, gout)
    f = contracted(orc, mat, g, w, gout)
    np.testing.assert_allclose(mat.T_e * d[1], 0.5 * mat.s_D * d[4], rtol=1e-6)
    np.testing.assert_allclose(mat.n_i * d[0], f - 0.5 * mat.s_D * d[4], rtol=1e-6)
    assert abs(d[4]) > 1e-6 * abs(f)


def test_gradient_ion_sphere_branch(orc):
    """Where r_i > lambda_D, T_e drops out (df/dT_e = 0) and L_D is
    proportional to s_D n_i^(-1/3): n_i df/dn_i = f - s_D df/ds_D / 3."""
    rng = np.random.default_rng(2)
    g, w = samples(rng)
    mat = orc.material(29, 5.0, 8.5e28, 100.0)
    s = orc.screening(mat)
    assert s.ri > 1.05 * s.lambdaD
    gout = np.array([0.7, 1.0, 0.05])
    d = orc.expected_emission_grad(mat, g, w, gout)
    f = contracted(orc, mat, g, w, gout)
    assert abs(d[1]) <= 1e-9 * abs(f) / mat.T_e
    np.testing.assert_allclose(mat.n_i * d[0], f - mat.s_D * d[4] / 3.0, rtol=1e-6)


def test_gradient_special_cases(orc):
    """Fully ionized (Z* = Z): the Thomas-Fermi part carries no charge, so
    df/ds_TF = 0.  The pair rate depends on theta only through its n_i
    factor: d/dtheta = (R_pair / n_i, 0, 0, 0, 0)."""
    rng = np.random.default_rng(3)
    g, w = samples(rng)
    full = orc.material(29, 29.0, 3e27, 2e3)
    d = orc.expected_emission_grad(full, g, w, np.array([1.0, 0.0, 1e-3]))
    f = contracted(orc, full, g, w, np.array([1.0, 0.0, 1e-3]))
    assert abs(d[3]) <= 1e-9 * abs(f)
    mat = orc.material(29, 12.0, 2e27, 300.0)
    out = orc.expected_emission(mat, g, w)
    d = orc.expected_emission_grad(mat, g, w, np.array([0.0, 1.0, 0.0]))
    np.testing.assert_allclose(d[0], out[1] / mat.n_i, rtol=1e-9)
    assert np.all(np.abs(d[1:]) <= 1e-12 * abs(out[1]) * np.array([1 / mat.T_e, 1 / mat.Zstar, 1.0, 1.0]))


def test_gradient_matches_coarser_difference(orc):
    """The Richardson-extrapolated derivative agrees with a plain central
    difference at a smaller step to the latter's truncation error."""
    rng = np.random.default_rng(4)
    g, w = samples(rng, 8)
    mat = orc.material(29, 7.0, 5e26, 800.0)
    gout = np.array([1.0, 0.5, 0.01])
    d = orc.expected_emission_grad(mat, g, w, gout)
    names = ["n_i", "T_e", "Zstar", "s_TF", "s_D"]
    for k, name in enumerate(names):
        v = getattr(mat, name)
        h = 1e-5 * v
        lo, hi = orc.material(29, mat.Zstar, mat.n_i, mat.T_e, mat.s_TF, mat.s_D), \
            orc.material(29, mat.Zstar, mat.n_i, mat.T_e, mat.s_TF, mat.s_D)
        setattr(lo, name, v - h)
        setattr(hi, name, v + h)
        fd = (contracted(orc, hi, g, w, gout) - contracted(orc, lo, g, w, gout)) / (2 * h)
        np.testing.assert_allclose(d[k], fd, rtol=1e-6, atol=1e-9 * abs(d).max(), err_msg=name)
