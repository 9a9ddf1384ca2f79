"""Pins of the oracle's accumulated (Berg) weight recursion.

The recursion combines the ln Omega differences that successive iterations estimate, each
weighted by its inverse Poisson variance.  The pins check it against the plain recursion
where the two must agree (first step), against the exact density of states of a small
lattice (convergence), against the fixed point W = P_SH / Omega, and against the statistics
of an inverse-variance mean (the variance of the combined estimate is 1 / sum of the inverse
variances, smaller than that of any other weighting).
"""
import numpy as np
import pytest

from tests.test_oracle_pins import _exact_lnomega_bins


@pytest.mark.parametrize("kind", [0, 1])
def test_first_step_equals_plain_step(orc, kind):
    dim, L, par = 3, 4, 0
    bt = orc.btop(dim, L, par)
    rng = np.random.default_rng(5)
    lnW = rng.normal(0.0, 3.0, bt + 1)
    hist = rng.integers(1, 5000, bt + 1).astype(np.uint32)
    hist[:7] = 0              # bottom never reached
    hist[20] = 0              # an empty bin inside the visited range
    hist[bt - 1] = 0
    e_g = orc.energy_of_bin(dim, L, par, 7)
    plain = orc.update_weights(dim, L, par, kind, -3.6, 96.0, e_g, lnW, hist)
    acc = orc.berg_state(bt + 1)
    berg = orc.update_weights_berg(dim, L, par, kind, -3.6, 96.0, e_g, lnW, hist, acc)
    np.testing.assert_allclose(berg, plain, rtol=0, atol=1e-10 * np.abs(plain).max())
    visited = (hist[:-1] > 0) & (hist[1:] > 0)
    assert np.all((acc[1, :bt] > 0) == visited)


def test_constant_weights_add_no_estimate(orc):
    """From W = const the sequential sweep is deterministic: the step is the plain step and
    the accumulators stay empty."""
    dim, L, par = 3, 4, 1
    bt = orc.btop(dim, L, par)
    hist = np.random.default_rng(6).integers(1, 5000, bt + 1).astype(np.uint32)
    e_g = orc.energy_of_bin(dim, L, par, 3)
    for kind in (0, 1):
        lnW = np.full(bt + 1, 2.5)
        acc = orc.berg_state(bt + 1)
        berg = orc.update_weights_berg(dim, L, par, kind, -3.6, 96.0, e_g, lnW, hist, acc)
        plain = orc.update_weights(dim, L, par, kind, -3.6, 96.0, e_g, lnW, hist)
        np.testing.assert_allclose(berg, plain, rtol=0, atol=1e-10 * np.abs(plain).max())
        assert not acc.any()


def test_fixed_point(orc):
    """Exact weights and noise-free flat histograms leave W unchanged, step after step."""
    dim, L, par = 2, 4, 0
    J = orc.make_disorder(dim, L, 21, 1)
    lnO, par, bt = _exact_lnomega_bins(orc, dim, L, J)
    reach = np.isfinite(lnO)
    lnW = np.where(reach, -(lnO - lnO[bt]), 0.0)
    hist = np.where(reach, 1000, 0).astype(np.uint32)
    acc = orc.berg_state(bt + 1)
    e_g = orc.energy_of_bin(dim, L, par, int(np.argmax(reach)))
    w = lnW
    for _ in range(4):
        w = orc.update_weights_berg(dim, L, par, 0, -3.6, 8.0, e_g, w, hist, acc)
        np.testing.assert_allclose(w[reach], lnW[reach], atol=1e-9)


def test_converges_to_exact_dos(orc):
    """From W = 1 the accumulated recursion drives ln W + ln g - ln P_SH to a constant."""
    dim, L, seed, rid = 2, 4, 21, 1
    J = orc.make_disorder(dim, L, seed, rid)
    lnO, par, bt = _exact_lnomega_bins(orc, dim, L, J)
    reach = np.isfinite(lnO)
    ch = orc.Chain(dim, L, seed, rid, J=J)
    for kind in (orc.FLAT, orc.POWERLAW):
        lnW = np.zeros(bt + 1)
        acc = orc.berg_state(bt + 1)
        for it in range(14):
            ch.hist[:] = 0
            ch.sweeps(20_000, orc.quantize(dim, lnW))
            eg = min(ch.rt.e_min, 0)
            lnW = orc.update_weights_berg(dim, L, par, kind, -3.6, 8.0, eg, lnW, ch.hist, acc)
        bg = int(np.argmax(reach))
        eg = orc.energy_of_bin(dim, L, par, bg)
        lnP = np.array([orc.ln_profile(kind, -3.6, 8.0, eg, orc.energy_of_bin(dim, L, par, b))
                        for b in range(bt + 1)])
        resid = (lnW + lnO - lnP)[reach]
        assert np.ptp(resid) < 0.1, resid
        assert lnW[bt] == 0.0


def test_combination_is_the_inverse_variance_mean(orc):
    """Two iterations of very different statistics on a two-bin system.

    Iteration A sees mean counts (5000, 50) under ln W = (0.5, 0), iteration B about 400 per bin under
    the weights A produced.  ln H has Poisson variance about 1/lambda, so the estimates of
    d = ln Omega(1) - ln Omega(0) have variances vA = 1/5000 + 1/50 and vB about 1/400 + 1/400,
    and their inverse-variance mean has variance 1/(1/vA + 1/vB) -- 20 % below the last
    iteration alone (the plain recursion) and far below a count-weighted mean.
    """
    dim, L, par, bt = 2, 4, 0, 1
    w0 = np.array([0.5, 0.0])
    d_true = np.log(50 / 5000) + w0[0] - w0[1]
    rng = np.random.default_rng(11)
    est, est_plain, vB = [], [], []
    for _ in range(4000):
        acc = orc.berg_state(2)
        hA = rng.poisson([5000.0, 50.0]).astype(np.uint32)
        w1 = orc.update_weights_berg(dim, L, par, 0, 0.0, 1.0, -32, w0, hA, acc)
        p = np.exp(np.array([0.0, d_true]) + w1)
        lam = 800.0 * p / p.sum()
        vB.append(1 / lam[0] + 1 / lam[1])
        hB = rng.poisson(lam).astype(np.uint32)
        w2 = orc.update_weights_berg(dim, L, par, 0, 0.0, 1.0, -32, w1, hB, acc)
        est.append(w2[0] - w2[1])
        plain = orc.update_weights(dim, L, par, 0, 0.0, 1.0, -32, w1, hB)
        est_plain.append(plain[0] - plain[1])
    est, est_plain = np.array(est), np.array(est_plain)
    vA, vB = 1 / 5000 + 1 / 50, float(np.mean(vB))
    v_opt = 1.0 / (1.0 / vA + 1.0 / vB)
    assert abs(np.var(est) / v_opt - 1.0) < 0.1, (np.var(est), v_opt)
    assert np.var(est) < 0.9 * np.var(est_plain)
    assert abs(np.mean(est) - d_true) < 0.01


def test_recovers_from_an_accumulated_trap(orc):
    """An accumulated estimate that over-weights the ground-state bin (by e^25) traps the chain
    there: it then visits that bin only, so no pair estimate arrives that could correct D.  The
    pair the chain stays on one side of must restart from the plain step; the recursion then
    escapes and converges to the exact density of states."""
    dim, L, seed, rid = 2, 4, 21, 1
    J = orc.make_disorder(dim, L, seed, rid)
    lnO, par, bt = _exact_lnomega_bins(orc, dim, L, J)
    reach = np.isfinite(lnO)
    bg = int(np.argmax(reach))
    lnW = np.where(reach, -(lnO - lnO[bt]), 0.0)
    lnW[bg] += 25.0
    acc = orc.berg_state(bt + 1)
    acc[0, :bt] = lnW[:bt] - lnW[1:]          # D consistent with the trapped weights (flat)
    acc[1, :bt] = 50.0
    ch = orc.Chain(dim, L, seed, rid, J=J)
    e_g = orc.energy_of_bin(dim, L, par, bg)
    for it in range(12):
        ch.hist[:] = 0
        ch.sweeps(5000, orc.quantize(dim, lnW))
        lnW = orc.update_weights_berg(dim, L, par, 0, -3.6, 8.0, e_g, lnW, ch.hist, acc)
    ch.hist[:] = 0
    ch.sweeps(20000, orc.quantize(dim, lnW))
    assert (ch.hist[reach] > 0).all(), ch.hist        # no longer confined to one bin
    resid = (lnW + lnO)[reach]
    assert np.ptp(resid) < 0.3, resid


@pytest.mark.parametrize("expected,restart", [(3.0, False), (9.5, False), (10.5, True), (300.0, True)])
def test_one_sided_pair_restarts_only_when_contradicted(orc, expected, restart):
    """A pair visited on one side only keeps its accumulated estimate while that estimate
    predicts few counts on the other side (zero of a Poisson mean of 3 has probability e^-3,
    no evidence against it) and restarts once it predicted at least 10 (probability below
    5e-5): then the plain step applies and the accumulators are empty."""
    dim, L, par, bt = 2, 4, 0, 1
    w0 = np.array([0.5, 0.0])
    for side in (0, 1):
        n = 1000
        hist = np.zeros(2, np.uint32)
        hist[side] = n
        # expected count on the empty side: n * exp(+-D + lnW(other) - lnW(side))
        if side == 0:
            d = np.log(expected / n) - (w0[1] - w0[0])
        else:
            d = -(np.log(expected / n) - (w0[0] - w0[1]))
        acc = orc.berg_state(2)
        acc[0, 0], acc[1, 0] = d, 100.0
        w = orc.update_weights_berg(dim, L, par, 0, 0.0, 1.0, -32, w0, hist, acc)
        plain = orc.update_weights(dim, L, par, 0, 0.0, 1.0, -32, w0, hist)
        if restart:
            assert acc[0, 0] == 0.0 and acc[1, 0] == 0.0
            np.testing.assert_allclose(w, plain, atol=1e-12)
        else:
            assert acc[0, 0] == d and acc[1, 0] == 100.0
            np.testing.assert_allclose(w[0] - w[1], d, atol=1e-12)     # flat target: diff = D
