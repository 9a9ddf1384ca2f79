"""Pins of the oracle's PT protocol: sweeps for odd L and the constant-exchange-rate
temperature adaptation (Sec. II, PT).

The colouring is checked bond by bond; odd-L PT against the exact canonical energies of
lattices small enough to enumerate; the adaptation rule against its fixed point, its end
points and the closed-form solution of a model with known pair stiffnesses; and the whole
protocol (PT runs plus adaptation) against exchange rates computed exactly from the density
of states at the temperatures it settles on.
"""
import numpy as np
import pytest

from tests.test_oracle_pins import _exact_mean_energy


def _coords(dim, L, i):
    return [i % L, (i // L) % L] + ([i // (L * L)] if dim == 3 else [])


def _site(dim, L, c):
    return c[0] + L * c[1] + (L * L * c[2] if dim == 3 else 0)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("L", [3, 4, 5, 6, 7, 9, 11])
def test_colouring_is_proper(orc, dim, L):
    V = L ** dim
    cols = [orc.pt_colour(dim, L, i) for i in range(V)]
    assert set(cols) == set(range(orc.pt_colours(L)))
    for i in range(V):
        c = _coords(dim, L, i)
        for d in range(dim):
            n = list(c)
            n[d] = (n[d] + 1) % L
            assert cols[i] != cols[_site(dim, L, n)], (i, d)
        if L % 2 == 0:
            assert cols[i] == sum(c) % 2          # the checkerboard for even L


def _exact_rates(g, nb, betas):
    """Exchange acceptance of each slot pair from exact canonical distributions."""
    E = 2 * np.arange(g.shape[0]) - nb
    ok = g > 0
    E, lg = E[ok], np.log(g[ok].astype(np.float64))
    P = []
    for b in betas:
        lw = lg - b * E
        w = np.exp(lw - lw.max())
        P.append(w / w.sum())
    rates = []
    for k in range(len(betas) - 1):
        db = betas[k + 1] - betas[k]
        # slot k holds E0, slot k+1 holds E1: accepted with min(1, exp(db (E1 - E0)))
        acc = np.minimum(1.0, np.exp(db * (E[None, :] - E[:, None])))
        rates.append(float(P[k] @ acc @ P[k + 1]))
    return np.array(rates)


@pytest.mark.parametrize("dim,L,rid", [(2, 5, 4), (3, 3, 6)])
def test_odd_L_pt_samples_canonical_distributions(orc, dim, L, rid):
    seed = 8
    betas = [0.2, 0.45, 0.8, 1.3]
    J = orc.make_disorder(dim, L, seed, rid)
    g = orc.dos_bruteforce(dim, L, J)
    nb = dim * L ** dim
    V = L ** dim
    pt = orc.PTRealization(dim, L, seed, rid, betas, J=J)
    pt.sweeps(500)
    sums = np.zeros((10, 4))
    for blk in range(10):
        acc = np.zeros(4)
        for _ in range(600):
            pt.sweeps(1)
            acc += pt.E
        sums[blk] = acc / 600
        for k in range(4):
            assert pt.E[k] == orc.energy(dim, L, J, pt.S[k * V:(k + 1) * V])
    for k, b in enumerate(betas):
        m, se = sums[:, k].mean(), sums[:, k].std(ddof=1) / np.sqrt(10)
        exact = _exact_mean_energy(g, nb, b)
        assert abs(m - exact) < 5 * se + 0.05, (k, m, exact, se)
    # exchange rates against the exact ones
    acc, att = pt.window_rates()
    want = _exact_rates(g, nb, betas)
    got = acc / att
    assert np.all(np.abs(got - want) < 0.03), (got, want)


def test_adapt_fixed_point_and_end_points(orc):
    betas = np.array([0.2, 0.3, 0.5, 0.9, 1.4, 2.5])
    att = np.full(5, 1000, dtype=np.uint64)
    same = orc.pt_adapt(betas, np.full(5, 470, dtype=np.uint64), att, 0.5)
    np.testing.assert_allclose(same, betas, rtol=0, atol=1e-15)
    rng = np.random.default_rng(2)
    for _ in range(20):
        acc = rng.integers(0, 1001, 5).astype(np.uint64)
        new = orc.pt_adapt(betas, acc, att, rng.uniform(0.1, 1.0))
        assert new[0] == betas[0] and new[-1] == betas[-1]
        assert np.all(np.diff(new) > 0)
    # a pair without attempts leaves the temperatures alone
    att0 = att.copy()
    att0[2] = 0
    assert np.array_equal(orc.pt_adapt(betas, np.full(5, 100, dtype=np.uint64), att0, 0.5), betas)


def test_adapt_converges_to_the_closed_form(orc):
    """Model: pair k accepts with exp(-s_k D_k).  Equal rates need D_k proportional to 1/s_k."""
    s = np.array([1.0, 3.0, 0.5, 2.0, 6.0, 1.5])
    M = s.shape[0] + 1
    betas = np.linspace(0.3, 2.8, M)
    span = betas[-1] - betas[0]
    n = 10 ** 12
    for _ in range(60):
        A = np.exp(-s * np.diff(betas))
        betas = orc.pt_adapt(betas, np.round(A * n).astype(np.uint64),
                             np.full(M - 1, n, dtype=np.uint64), 0.5)
    want = span * (1 / s) / np.sum(1 / s)
    np.testing.assert_allclose(np.diff(betas), want, rtol=1e-6)


def test_protocol_reaches_constant_exchange_rates(orc):
    """PT runs plus adaptation on a 4x4 lattice; the exact rates at the final temperatures
    agree with each other far better than at the geometric start."""
    dim, L, seed, rid = 2, 4, 8, 3
    J = orc.make_disorder(dim, L, seed, rid)
    g = orc.dos_bruteforce(dim, L, J)
    betas0 = 0.1 * (25.0 ** (np.arange(6) / 5))      # geometric in [0.1, 2.5]
    pt = orc.PTRealization(dim, L, seed, rid, betas0, J=J)
    pt.sweeps(200)
    pt.adapt(0.0)                                      # start a fresh window
    for _ in range(14):
        pt.sweeps(3000)
        pt.adapt(0.5)
    before = _exact_rates(g, 32, betas0)
    after = _exact_rates(g, 32, pt.betas)
    assert np.ptp(after) < 0.06, after
    assert np.ptp(after) < 0.3 * np.ptp(before), (before, after)
    assert pt.betas[0] == betas0[0] and pt.betas[-1] == betas0[-1]
