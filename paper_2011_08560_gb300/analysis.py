"""Round-trip-time analysis of Secs. IV and V (host side; the next step after the hot path).

Per method and lattice size the round-trip times tau_i of the realizations are fitted with
a Frechet (generalized extreme value, shape xi > 0) distribution, Eq. "cdf":
    F(tau) = exp[-(1 + xi (tau - mu)/beta)^(-1/xi)],   tau >= mu - beta/xi,
and compared through
    the distribution mean, Eq. "frechet_mean": mu + beta/xi [Gamma(1 - xi) - 1] (xi < 1, else inf),
    the running / population mean, Eq. "running_mean",
    the quantile function Q(p) = mu + beta/xi [(-ln p)^(-xi) - 1],
    the quantile mean, Eq. "quantile_mean": the integral of tau f(tau) up to Q(1 - eps)
        (as printed, not normalised by 1 - eps); with p = exp(-w) it equals
        (mu - beta/xi)(1 - eps) + (beta/xi) Gamma(1 - xi, -ln(1 - eps)),
    the relative performance r = mean(method) / mean(power law) with jackknife errors.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import optimize, special


def frechet_cdf(tau, mu, beta, xi):
    tau = np.asarray(tau, dtype=float)
    s = 1.0 + xi * (tau - mu) / beta
    with np.errstate(divide="ignore", invalid="ignore"):
        out = np.exp(-np.power(np.where(s > 0, s, np.nan), -1.0 / xi))
    return np.where(s > 0, out, 0.0)


def frechet_pdf(tau, mu, beta, xi):
    tau = np.asarray(tau, dtype=float)
    s = 1.0 + xi * (tau - mu) / beta
    with np.errstate(divide="ignore", invalid="ignore"):
        sp = np.where(s > 0, s, np.nan)
        out = (1.0 / beta) * np.power(sp, -1.0 / xi - 1.0) * np.exp(-np.power(sp, -1.0 / xi))
    return np.where(s > 0, out, 0.0)


def quantile(p, mu, beta, xi):
    p = np.asarray(p, dtype=float)
    return mu + beta / xi * (np.power(-np.log(p), -xi) - 1.0)


def distribution_mean(mu, beta, xi):
    return mu + beta / xi * (math.gamma(1.0 - xi) - 1.0) if xi < 1.0 else math.inf


def upper_gamma(s: float, x: float) -> float:
    """Gamma(s, x) = int_x^inf w^(s-1) e^-w dw for x > 0 and any real s."""
    if s > 0:
        return float(special.gammaincc(s, x) * special.gamma(s))
    if s == 0:
        return float(special.exp1(x))
    # Gamma(s, x) = (Gamma(s + 1, x) - x^s e^-x) / s, recursing up to s > 0
    return (upper_gamma(s + 1.0, x) - x ** s * math.exp(-x)) / s


def quantile_mean(mu, beta, xi, eps):
    w = -math.log1p(-eps)
    return (mu - beta / xi) * (1.0 - eps) + beta / xi * upper_gamma(1.0 - xi, w)


def running_mean(taus):
    taus = np.asarray(taus, dtype=float)
    return np.cumsum(taus) / np.arange(1, taus.size + 1)


def frechet_fit(taus):
    """Maximum-likelihood (mu, beta, xi) of Eq. "cdf" for xi > 0."""
    t = np.sort(np.asarray(taus, dtype=float))
    med, iqr = np.median(t), np.subtract(*np.percentile(t, [75, 25]))
    x0 = np.array([med, max(iqr, 1e-9 * abs(med) + 1e-12), 0.3])

    def nll(p):
        mu, lb, lx = p
        beta, xi = math.exp(lb), math.exp(lx)
        s = 1.0 + xi * (t - mu) / beta
        if np.any(s <= 0):
            return 1e300
        return float(np.sum(np.log(beta) + (1.0 / xi + 1.0) * np.log(s) + np.power(s, -1.0 / xi)))

    best = None
    for xi0 in (0.1, 0.3, 0.8, 1.5):
        start = np.array([x0[0], math.log(x0[1]), math.log(xi0)])
        r = optimize.minimize(nll, start, method="Nelder-Mead",
                              options={"xatol": 1e-10, "fatol": 1e-10, "maxiter": 40000, "maxfev": 40000})
        if best is None or r.fun < best.fun:
            best = r
    mu, lb, lx = best.x
    return float(mu), float(math.exp(lb)), float(math.exp(lx))


def jackknife(values_a, values_b, stat):
    """Ratio stat(a)/stat(b) over paired samples with a leave-one-out jackknife error."""
    a, b = np.asarray(values_a, dtype=float), np.asarray(values_b, dtype=float)
    n = a.size
    full = stat(a) / stat(b)
    loo = np.array([stat(np.delete(a, i)) / stat(np.delete(b, i)) for i in range(n)])
    err = math.sqrt((n - 1) / n * np.sum((loo - loo.mean()) ** 2))
    return float(full), float(err)


def block_jackknife(values_a, values_b, stat, n_blocks: int = 16):
    """Ratio stat(a)/stat(b) over paired samples with a delete-one-block jackknife error: the
    realizations are split into n_blocks contiguous blocks and each replicate leaves one out
    (with n_blocks = n this is the leave-one-out jackknife)."""
    a, b = np.asarray(values_a, dtype=float), np.asarray(values_b, dtype=float)
    n = a.size
    k = max(2, min(n_blocks, n))
    edges = np.linspace(0, n, k + 1).astype(int)
    full = stat(a) / stat(b)
    reps = []
    for i in range(k):
        keep = np.r_[0:edges[i], edges[i + 1]:n]
        reps.append(stat(a[keep]) / stat(b[keep]))
    reps = np.array(reps)
    err = math.sqrt((k - 1) / k * np.sum((reps - reps.mean()) ** 2))
    return float(full), float(err)


def relative_performance(taus_method, taus_pl, eps=1e-4, n_blocks: int = 16):
    """Table I quantities of a method relative to the power-law ensemble, over the realizations
    (paired samples) where both have a finite round-trip time: r_pop, the ratio of population
    means (Eq. "running_mean" at n = N), and r_eps, the ratio of quantile means (Eq.
    "quantile_mean") of the Frechet fits, each as (value, jackknife error)."""
    a, b = np.asarray(taus_method, dtype=float), np.asarray(taus_pl, dtype=float)
    ok = np.isfinite(a) & np.isfinite(b)
    a, b = a[ok], b[ok]
    pop = lambda x: float(np.mean(x))
    qm = lambda x: quantile_mean(*frechet_fit(x), eps)
    return {"r_pop": block_jackknife(a, b, pop, n_blocks), "r_eps": block_jackknife(a, b, qm, n_blocks),
            "pairs": int(a.size)}
