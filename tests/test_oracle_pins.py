"""Pins of the CPU oracle against things other than itself.

Each test checks the oracle against a value the paper prints, a published test vector, an
exact result obtained by an independent route (transfer matrices, enumeration), a symmetry
or invariant of the Hamiltonian, or a statistical law that an ensemble must obey.  A
plausible slip in the oracle (a dropped term, a sign, a transposed index, the wrong class
of a move) breaks at least one of them.
"""
from pathlib import Path

import numpy as np
import pytest

from tests.transfer_matrix import partition_function, z_from_dos

GOLDEN = Path(__file__).resolve().parent / "golden"


def _rows(name):
    out = []
    for line in (GOLDEN / name).read_text().splitlines():
        line = line.strip()
        if line and not line.startswith("#"):
            out.append(line.split())
    return out


# ------------------------------------------------------------------ Philox (SC'11 KAT)
def test_philox_known_answers(orc):
    for row in _rows("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in row]
        assert list(orc.philox(v[0:4], v[4:6])) == v[6:10]


# ------------------------------------------------------------------ density of states
def test_dos_ferromagnet_matches_published(orc):
    J = np.ones(32, dtype=np.int8)
    g = orc.dos_bruteforce(2, 4, J)
    want = {int(e): int(c) for e, c in _rows("ising2d_4x4_dos.txt")}
    got = {2 * u - 32: int(c) for u, c in enumerate(g) if c}
    assert got == want


@pytest.mark.parametrize("dim,L,rid", [(2, 4, 0), (2, 4, 7), (3, 3, 1)])
def test_dos_matches_transfer_matrix(orc, dim, L, rid):
    J = orc.make_disorder(dim, L, 11, rid)
    g = orc.dos_bruteforce(dim, L, J)
    nb = orc.nbonds(dim, L)
    assert int(g.sum()) == 2 ** orc.volume(dim, L)
    for beta in (0.05, 0.3, 0.7, 1.3):
        zt = partition_function(dim, L, J, beta)
        zd = z_from_dos(g, nb, beta)
        assert zd == pytest.approx(zt, rel=1e-11)


def test_dos_symmetries(orc):
    # even L: the lattice is bipartite, flipping one sublattice maps E -> -E
    J = orc.make_disorder(2, 4, 3, 5)
    g = orc.dos_bruteforce(2, 4, J)
    assert np.array_equal(g, g[::-1])
    # gauge invariance: J_ij -> t_i J_ij t_j leaves g unchanged
    rng = np.random.default_rng(0)
    tau = rng.choice([-1, 1], size=16).astype(np.int8)
    Jg = _gauge(2, 4, J, tau)
    assert np.array_equal(orc.dos_bruteforce(2, 4, Jg), g)


def _neighbour(dim, L, i, d):
    c = [i % L, (i // L) % L, i // (L * L) if dim == 3 else 0]
    c[d] = (c[d] + 1) % L
    return c[0] + L * c[1] + L * L * c[2]


def _gauge(dim, L, J, tau):
    Jg = J.copy()
    V = L ** dim
    for i in range(V):
        for d in range(dim):
            Jg[i * dim + d] = tau[i] * J[i * dim + d] * tau[_neighbour(dim, L, i, d)]
    return Jg


# ------------------------------------------------------------------ Hamiltonian basics
def test_energy_definitions(orc):
    dim, L = 3, 4
    J = orc.make_disorder(dim, L, 1, 0)
    assert set(np.unique(J)) == {-1, 1}
    assert abs(float((J < 0).mean()) - 0.5) < 0.1
    S = np.ones(64, dtype=np.int8)
    # all spins up: E = -sum J
    assert orc.energy(dim, L, J, S) == -int(J.astype(int).sum())
    # flipping one spin changes E by 2 S_i h_i with dE in {0, +-4, +-8, +-12}
    S2 = orc.make_spins(dim, L, 1, 0)
    E0 = orc.energy(dim, L, J, S2)
    for i in range(64):
        S3 = S2.copy()
        S3[i] = -S3[i]
        dE = orc.energy(dim, L, J, S3) - E0
        assert dE in (-12, -8, -4, 0, 4, 8, 12)
    # bins: E = 2u - 3V and the parity of u is that of the number of negative bonds
    u = (E0 + 192) // 2
    assert u % 2 == orc.parity(dim, L, J)
    b = orc.bin_of_energy(dim, L, E0)
    assert orc.energy_of_bin(dim, L, orc.parity(dim, L, J), b) == E0


def test_top_of_range(orc):
    for dim, L in ((3, 4), (3, 3), (3, 6), (2, 4)):
        nb = orc.nbonds(dim, L)
        for par in (0, 1):
            bt = orc.btop(dim, L, par)
            et = orc.energy_of_bin(dim, L, par, bt)
            assert et <= 0 and et + 4 > 0        # the largest attainable E <= 0
            assert (et + nb) // 2 % 2 == par


# ------------------------------------------------------------------ profile (Eq. power_law)
def test_profile_worked_numbers(orc):
    for alpha, dE, eg, printed, tol in _rows("profile_ratio.txt"):
        alpha, dE, eg, printed, tol = float(alpha), float(dE), int(eg), float(printed), float(tol)
        ratio = np.exp(orc.ln_profile(1, alpha, dE, eg, eg))
        if tol == 0.0:
            assert ratio == 1.0
        else:
            assert abs(ratio / printed - 1.0) < tol
    # normalised to 1 at E = 0, increasing towards E_g for alpha < 0, held below E_g
    assert orc.ln_profile(1, -3.6, 96.0, -100, 0) == 0.0
    assert orc.ln_profile(1, -3.6, 96.0, -100, -50) > 0.0
    assert orc.ln_profile(1, -3.6, 96.0, -100, -120) == orc.ln_profile(1, -3.6, 96.0, -100, -100)
    assert orc.ln_profile(0, -3.6, 96.0, -100, -50) == 0.0


# ------------------------------------------------------------------ quantisation
def test_quantize_special_cases(orc):
    lnW = np.array([0.0, -np.log(2.0), -1000.0, 5.0, 0.0])
    thr = orc.quantize(3, lnW).reshape(5, 8)
    # class n = dim (dE = 0) stays in the bin: always
    assert all(thr[b, 3] == orc.ALWAYS for b in range(5))
    # from bin 1 (lnW=-ln2) to bin 0 (n=4, db=-1): uphill in W -> always
    assert thr[1, 4] == orc.ALWAYS
    # from bin 0 to bin 1 (n=2, db=+1): p = 1/2 -> floor(2^31) within one ulp of exp
    assert thr[0, 2] in (2 ** 31 - 1, 2 ** 31)
    # towards bin 2 (lnW=-1000) p underflows to 0
    assert thr[1, 2] == 0
    # moves leaving [0, b_top] are walls, classes beyond 2*dim are unused
    assert thr[4, 0] == 0 and thr[4, 1] == 0 and thr[4, 2] == 0
    assert thr[0, 6] == 0 and thr[0, 5] == 0 and thr[0, 4] == 0
    assert all(thr[b, 7] == 0 for b in range(5))


# ------------------------------------------------------------------ chain invariants
def _flat_thresholds(orc, ch):
    return orc.quantize(ch.dim, np.zeros(ch.b_top + 1))


def test_descent_reaches_top(orc):
    for rid in range(8):
        ch = orc.Chain(3, 4, 5, rid)
        assert ch.E <= ch.e_top
        assert ch.E == orc.energy(3, 4, ch.J, ch.S)


def test_incremental_energy_equals_recompute(orc):
    ch = orc.Chain(3, 4, 1, 0)
    rng = np.random.default_rng(1)
    lnW = -0.05 * rng.standard_normal(ch.b_top + 1).cumsum()
    thr = orc.quantize(3, lnW)
    for _ in range(5):
        ch.sweeps(20, thr)
        assert ch.E == orc.energy(3, 4, ch.J, ch.S)
        assert ch.E <= ch.e_top


def test_gauge_and_global_flip_invariance(orc):
    dim, L = 3, 4
    ref = orc.Chain(dim, L, 2, 3)
    rng = np.random.default_rng(5)
    tau = rng.choice([-1, 1], size=64).astype(np.int8)
    J0 = orc.make_disorder(dim, L, 2, 3)
    S0 = orc.make_spins(dim, L, 2, 3)
    gauged = orc.Chain(dim, L, 2, 3, J=_gauge(dim, L, J0, tau), S=tau * S0)
    flipped = orc.Chain(dim, L, 2, 3, S=-S0)
    lnW = np.linspace(0.0, -3.0, ref.b_top + 1)[::-1].copy()
    thr = orc.quantize(dim, lnW)
    tr = [c.sweeps(50, thr, trace=True) for c in (ref, gauged, flipped)]
    assert np.array_equal(tr[0], tr[1]) and np.array_equal(tr[0], tr[2])
    assert np.array_equal(gauged.S, tau * ref.S)
    assert np.array_equal(flipped.S, -ref.S)


def test_resume_is_bit_exact(orc):
    a = orc.Chain(3, 4, 9, 1)
    b = orc.Chain(3, 4, 9, 1)
    thr = _flat_thresholds(orc, a)
    ta = a.sweeps(40, thr, trace=True)
    tb = np.concatenate([b.sweeps(15, thr, trace=True), b.sweeps(25, thr, trace=True)])
    assert np.array_equal(ta, tb) and np.array_equal(a.S, b.S)
    assert np.array_equal(a.hist, b.hist)


# ------------------------------------------------------------------ ensembles (statistics)
def _exact_lnomega_bins(orc, dim, L, J):
    g = orc.dos_bruteforce(dim, L, J).astype(np.float64)
    par = orc.parity(dim, L, J)
    bt = orc.btop(dim, L, par)
    lnO = np.full(bt + 1, -np.inf)
    for b in range(bt + 1):
        u = 2 * b + par
        if g[u] > 0:
            lnO[b] = np.log(g[u])
    return lnO, par, bt


def _weights_from(lnW_target):
    lnW = np.where(np.isfinite(lnW_target), lnW_target, 0.0)
    return lnW


@pytest.mark.parametrize("dim,L,rid", [(2, 4, 1), (3, 3, 2)])
def test_flat_histogram_with_exact_weights(orc, dim, L, rid):
    """W = 1/g makes the energy histogram flat (Eq. "muca-weights")."""
    seed = 21
    J = orc.make_disorder(dim, L, seed, rid)
    lnO, par, bt = _exact_lnomega_bins(orc, dim, L, J)
    lnW = _weights_from(-lnO)
    ch = orc.Chain(dim, L, seed, rid, J=J)
    thr = orc.quantize(dim, lnW)
    n = 400_000 if dim == 2 else 60_000
    ch.sweeps(n, thr)
    reach = np.isfinite(lnO)
    h = ch.hist[reach].astype(np.float64)
    rel = h / h.mean() - 1.0
    assert np.abs(rel).max() < 0.12, rel
    assert np.abs(rel).mean() < 0.05, rel


def test_power_law_histogram_follows_profile(orc):
    """W = P_SH/g shapes the histogram as P_SH (the nonflat weight of Sec. II)."""
    dim, L, seed, rid = 2, 4, 21, 1
    J = orc.make_disorder(dim, L, seed, rid)
    lnO, par, bt = _exact_lnomega_bins(orc, dim, L, J)
    reach = np.isfinite(lnO)
    bg = int(np.argmax(reach))
    eg = orc.energy_of_bin(dim, L, par, bg)
    alpha, pole = -3.6, 8.0
    lnP = np.array([orc.ln_profile(1, alpha, pole, eg, orc.energy_of_bin(dim, L, par, b))
                    for b in range(bt + 1)])
    lnW = _weights_from(lnP - lnO)
    ch = orc.Chain(dim, L, seed, rid, J=J)
    ch.sweeps(400_000, orc.quantize(dim, lnW))
    h = ch.hist[reach].astype(np.float64)
    p = np.exp(lnP[reach])
    ratio = (h / h.sum()) / (p / p.sum())
    assert np.abs(ratio - 1.0).max() < 0.12, ratio
    assert p.max() / p.min() > 5.0          # the profile really is nonflat here


def test_one_over_k_histogram(orc):
    """The 1/k ensemble (Eq. "1/k") samples E with probability proportional to g(E)/k(E)."""
    dim, L, seed, rid = 2, 4, 21, 2
    J = orc.make_disorder(dim, L, seed, rid)
    lnO, par, bt = _exact_lnomega_bins(orc, dim, L, J)
    reach = np.isfinite(lnO)
    bg = int(np.argmax(reach))
    eg = orc.energy_of_bin(dim, L, par, bg)
    lnW = orc.build_weights(dim, L, par, orc.ONE_OVER_K, 0.0, 0.0, 0.0, eg,
                            np.where(reach, lnO, -700.0))
    ch = orc.Chain(dim, L, seed, rid, J=J)
    ch.sweeps(400_000, orc.quantize(dim, lnW))
    g = np.exp(lnO[reach])
    k = np.cumsum(g)                          # k(E) = sum_{E_g <= E' <= E} g(E')
    want = g / k
    h = ch.hist[reach].astype(np.float64)
    ratio = (h / h.sum()) / (want / want.sum())
    assert np.abs(ratio - 1.0).max() < 0.12, ratio


def _exact_mean_energy(g, nb, beta, emax=None):
    u = np.arange(len(g))
    E = 2 * u - nb
    w = np.asarray(g, dtype=np.float64) * np.exp(-beta * (E - E.min()))
    if emax is not None:
        w = np.where(E <= emax, w, 0.0)
    return float((w * E).sum() / w.sum())


def test_canonical_special_case(orc):
    """ln W = -beta E reduces the generalized criterion to textbook Metropolis."""
    dim, L, seed, rid = 2, 4, 3, 4
    J = orc.make_disorder(dim, L, seed, rid)
    g = orc.dos_bruteforce(dim, L, J)
    par = orc.parity(dim, L, J)
    bt = orc.btop(dim, L, par)
    beta = 0.6
    lnW = orc.build_weights(dim, L, par, orc.CANON, 0.0, 0.0, beta, 0, np.zeros(bt + 1))
    ch = orc.Chain(dim, L, seed, rid, J=J)
    thr = orc.quantize(dim, lnW)
    ch.sweeps(2000, thr)
    means = []
    for _ in range(20):
        tr = ch.sweeps(10_000, thr, trace=True)
        means.append(tr.mean())
    m, se = np.mean(means), np.std(means, ddof=1) / np.sqrt(len(means))
    exact = _exact_mean_energy(g, 32, beta, emax=orc.energy_of_bin(dim, L, par, bt))
    assert abs(m - exact) < 5 * se + 0.02, (m, exact, se)


def test_weight_iteration_converges_to_dos(orc):
    """Iterating W <- W P/H from W = 1 drives ln W + ln g - ln P to a constant."""
    dim, L, seed, rid = 2, 4, 21, 1
    J = orc.make_disorder(dim, L, seed, rid)
    lnO, par, bt = _exact_lnomega_bins(orc, dim, L, J)
    reach = np.isfinite(lnO)
    ch = orc.Chain(dim, L, seed, rid, J=J)
    for kind in (orc.FLAT, orc.POWERLAW):
        lnW = np.zeros(bt + 1)
        for it in range(14):
            ch.hist[:] = 0
            ch.sweeps(20_000 if it < 10 else 100_000, orc.quantize(dim, lnW))
            eg = min(ch.rt.e_min, 0)
            lnW = orc.update_weights(dim, L, par, kind, -3.6, 8.0, eg, lnW, ch.hist)
        bg = int(np.argmax(reach))
        eg = orc.energy_of_bin(dim, L, par, bg)
        lnP = np.array([orc.ln_profile(kind, -3.6, 8.0, eg, orc.energy_of_bin(dim, L, par, b))
                        for b in range(bt + 1)])
        resid = (lnW + lnO - lnP)[reach]
        assert np.ptp(resid) < 0.15, resid
        assert lnW[bt] == 0.0


def test_round_trip_state_machine(orc):
    """Round trips (Sec. III) are top -> E_g -> top; t_first is the first top visit."""
    dim, L, seed, rid = 2, 4, 21, 1
    J = orc.make_disorder(dim, L, seed, rid)
    lnO, par, bt = _exact_lnomega_bins(orc, dim, L, J)
    reach = np.isfinite(lnO)
    bg = int(np.argmax(reach))
    eg = orc.energy_of_bin(dim, L, par, bg)
    ch = orc.Chain(dim, L, seed, rid, J=J)
    ch.rt.e_g = eg
    tr = ch.sweeps(20_000, orc.quantize(dim, _weights_from(-lnO)), count_rt=True, trace=True)
    rt = ch.rt
    assert rt.n_rt > 50 and rt.requeue == 0
    assert 0 <= rt.t_first <= rt.t_last < 20_000
    assert rt.e_min == eg
    # every round trip needs at least one visit to E_g between two top visits
    assert (tr == eg).sum() >= 1


# ------------------------------------------------------------------ parallel tempering
def test_pt_tables(orc):
    betas = np.array([0.2, 0.5, 1.0])
    thr_k, thr_pair = orc.pt_tables(3, betas, 10)
    thr_k = thr_k.reshape(3, 8)
    for k, b in enumerate(betas):
        for n in range(7):
            dE = 12 - 4 * n
            if dE <= 0:
                assert thr_k[k, n] == orc.ALWAYS
            else:
                assert abs(int(thr_k[k, n]) - np.exp(-b * dE) * 2 ** 32) <= 1.0
    thr_pair = thr_pair.reshape(2, 11)
    for k in range(2):
        for d in range(1, 11):
            p = np.exp(-(betas[k + 1] - betas[k]) * 4 * d)   # Eq. "temperatureexchange"
            assert abs(int(thr_pair[k, d]) - p * 2 ** 32) <= 1.0


def test_pt_samples_canonical_distributions(orc):
    """Each PT slot samples P_k(E) proportional to g(E) exp(-beta_k E)."""
    dim, L, seed, rid = 2, 4, 8, 3
    betas = [0.2, 0.45, 0.8, 1.3]
    J = orc.make_disorder(dim, L, seed, rid)
    g = orc.dos_bruteforce(dim, L, J)
    pt = orc.PTRealization(dim, L, seed, rid, betas, J=J)
    pt.sweeps(1000)
    sums = np.zeros((10, 4))
    for blk in range(10):
        acc = np.zeros(4)
        for _ in range(1000):
            pt.sweeps(1)
            acc += pt.E
        sums[blk] = acc / 1000
        # configurations move between slots but every slot keeps its own energy bookkeeping
        for k in range(4):
            assert pt.E[k] == orc.energy(dim, L, J, pt.S[k * 16:(k + 1) * 16])
    for k, b in enumerate(betas):
        m, se = sums[:, k].mean(), sums[:, k].std(ddof=1) / np.sqrt(10)
        exact = _exact_mean_energy(g, 32, b)
        assert abs(m - exact) < 5 * se + 0.05, (k, m, exact, se)
    assert sorted(pt.label) == [0, 1, 2, 3]
    assert pt.swap_acc.sum() > 0
