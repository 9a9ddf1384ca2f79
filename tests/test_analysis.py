"""Pins of the round-trip analysis (Secs. IV, V) against independent routes."""
import math

import numpy as np
import pytest
from scipy import integrate, stats

from paper_2011_08560_gb300 import analysis as an

PARAMS = [(200.0, 80.0, 0.3), (1e3, 500.0, 0.75), (50.0, 10.0, 1.4)]


@pytest.mark.parametrize("mu,beta,xi", PARAMS)
def test_cdf_pdf_quantile(mu, beta, xi):
    # scipy's genextreme is the same family with shape c = -xi
    ref = stats.genextreme(c=-xi, loc=mu, scale=beta)
    t = np.linspace(mu - beta / xi + 1e-6, mu + 20 * beta, 50)
    assert np.allclose(an.frechet_cdf(t, mu, beta, xi), ref.cdf(t), rtol=1e-10, atol=1e-14)
    assert np.allclose(an.frechet_pdf(t, mu, beta, xi), ref.pdf(t), rtol=1e-9, atol=1e-14)
    p = np.array([0.01, 0.3, 0.5, 0.9, 0.9999])
    assert np.allclose(an.frechet_cdf(an.quantile(p, mu, beta, xi), mu, beta, xi), p, rtol=1e-12)


@pytest.mark.parametrize("mu,beta,xi", PARAMS[:2])
def test_distribution_mean_is_the_integral(mu, beta, xi):
    num, _ = integrate.quad(lambda t: t * an.frechet_pdf(t, mu, beta, xi), mu - beta / xi, np.inf, limit=500)
    assert an.distribution_mean(mu, beta, xi) == pytest.approx(num, rel=1e-7)
    assert an.distribution_mean(mu, beta, 1.2) == math.inf


@pytest.mark.parametrize("mu,beta,xi", PARAMS)
@pytest.mark.parametrize("eps", [1e-4, 1e-2])
def test_quantile_mean_closed_form(mu, beta, xi, eps):
    # Eq. "quantile_mean" by numeric integration over p: int_0^{1-eps} Q(p) dp
    num, _ = integrate.quad(lambda p: an.quantile(p, mu, beta, xi), 0.0, 1.0 - eps, limit=1000, points=[0.5])
    assert an.quantile_mean(mu, beta, xi, eps) == pytest.approx(num, rel=1e-7)


def test_quantile_mean_tends_to_the_mean():
    assert an.quantile_mean(200.0, 80.0, 0.3, 1e-12) == pytest.approx(an.distribution_mean(200.0, 80.0, 0.3),
                                                                      rel=1e-6)


def test_fit_recovers_parameters_and_agrees_with_scipy():
    rng = np.random.default_rng(7)
    mu, beta, xi = 300.0, 120.0, 0.45
    x = stats.genextreme(c=-xi, loc=mu, scale=beta).rvs(size=4000, random_state=rng)
    m, b, s = an.frechet_fit(x)
    assert abs(s - xi) < 0.05 and abs(m - mu) / mu < 0.03 and abs(b - beta) / beta < 0.05
    c, loc, scale = stats.genextreme.fit(x)
    assert abs(-c - s) < 0.01 and abs(loc - m) / m < 0.005 and abs(scale - b) / b < 0.01


def test_running_mean_and_jackknife():
    x = np.array([1.0, 3.0, 5.0, 7.0])
    assert np.allclose(an.running_mean(x), [1.0, 2.0, 3.0, 4.0])
    r, err = an.jackknife(2 * x, x, np.mean)
    assert r == pytest.approx(2.0) and err == pytest.approx(0.0, abs=1e-12)
    rng = np.random.default_rng(1)
    a, b = rng.exponential(3.0, 500), rng.exponential(1.5, 500)
    r, err = an.jackknife(a, b, np.mean)
    assert abs(r - 2.0) < 4 * err + 0.2 and err > 0


def test_block_jackknife_reduces_to_leave_one_out():
    rng = np.random.default_rng(4)
    a, b = rng.exponential(3.0, 40), rng.exponential(1.5, 40)
    assert an.block_jackknife(a, b, np.mean, n_blocks=40) == pytest.approx(an.jackknife(a, b, np.mean), rel=1e-12)
    # the delete-one-block error of a mean ratio is close to the delta-method standard error
    a, b = rng.exponential(3.0, 4000), rng.exponential(1.5, 4000)
    r, err = an.block_jackknife(a, b, np.mean, n_blocks=20)
    delta = r * math.sqrt(np.var(a) / a.size / np.mean(a) ** 2 + np.var(b) / b.size / np.mean(b) ** 2)
    assert 0.5 * delta < err < 2.0 * delta


def test_relative_performance_recovers_known_ratios():
    """Paired samples from two Frechet laws: r_pop near the ratio of the distribution means,
    r_eps near the ratio of the quantile means of the true parameters (Table I quantities);
    realizations without a finite time in either method are left out."""
    rng = np.random.default_rng(11)
    pa, pb = (600.0, 250.0, 0.3), (200.0, 80.0, 0.25)
    a = stats.genextreme(c=-pa[2], loc=pa[0], scale=pa[1]).rvs(size=3000, random_state=rng)
    b = stats.genextreme(c=-pb[2], loc=pb[0], scale=pb[1]).rvs(size=3000, random_state=rng)
    a[:7] = np.inf
    out = an.relative_performance(a, b, eps=1e-4)
    assert out["pairs"] == 2993
    r_pop, e_pop = out["r_pop"]
    r_eps, e_eps = out["r_eps"]
    want_pop = an.distribution_mean(*pa) / an.distribution_mean(*pb)
    want_eps = an.quantile_mean(*pa, 1e-4) / an.quantile_mean(*pb, 1e-4)
    assert abs(r_pop - want_pop) < 4 * e_pop + 0.02 and e_pop > 0
    assert abs(r_eps - want_eps) < 4 * e_eps + 0.02 and e_eps > 0
