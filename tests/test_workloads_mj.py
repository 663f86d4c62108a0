"""The Maxwell-Juttner fast-electron source of Sec. IV (Eq. mj), an input
generator: its normalisation (the Bessel-function identity behind Eq. mj),
the mean-energy limits the paper states, and the rejection sampler against
the distribution function (Kolmogorov-Smirnov) and the analytic mean."""
import numpy as np
import pytest
from scipy import integrate, special, stats

from paper_1907_02814_gb300 import workloads as W


def density_T(T, theta):
    """Eq. (mj) in the kinetic variable: gamma^2 beta exp(-gamma/theta) / (theta K2(1/theta))."""
    g = 1.0 + T
    return g * np.sqrt(T * (T + 2.0)) * np.exp(-g / theta) / (theta * special.kn(2, 1.0 / theta))


@pytest.mark.parametrize("theta", [0.05, 0.5, 2.0, 8.0])
def test_normalised(theta):
    assert integrate.quad(density_T, 0.0, np.inf, args=(theta,), limit=200)[0] == pytest.approx(1.0, rel=1e-8)
    mean = integrate.quad(lambda T: T * density_T(T, theta), 0.0, np.inf, limit=200)[0]
    assert W.maxwell_juttner_mean_kinetic(theta) == pytest.approx(mean, rel=1e-8)


def test_mean_energy_limits():
    """<T> ~ 3 theta / 2 for theta << 1 and ~ 3 theta for theta >> 1."""
    assert W.maxwell_juttner_mean_kinetic(1e-3) / 1e-3 == pytest.approx(1.5, rel=2e-3)
    assert W.maxwell_juttner_mean_kinetic(300.0) / 300.0 == pytest.approx(3.0, rel=2e-3)


@pytest.mark.parametrize("mean_mev", [1.0, 3.0, 10.0])
def test_sampler(mean_mev):
    theta = W.maxwell_juttner_theta(mean_mev)
    assert W.maxwell_juttner_mean_kinetic(theta) * W.MEC2_MEV == pytest.approx(mean_mev, rel=1e-12)
    T = W.maxwell_juttner_kinetic(np.random.default_rng(7), theta, 200_000)
    assert abs(T.mean() - W.maxwell_juttner_mean_kinetic(theta)) < 4 * T.std() / np.sqrt(len(T))
    grid = np.linspace(0.0, 40.0 * theta + 20.0, 4001)
    pdf = density_T(grid, theta)
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (pdf[1:] + pdf[:-1]) * np.diff(grid))])
    ks = stats.kstest(T, lambda t: np.interp(t, grid, cdf))
    assert ks.pvalue > 1e-3
