"""GPU parallel tempering (a6 + a7) vs the oracle, element by element, through the C ABI.

Spins by slot, energies, replica labels, per-replica round-trip records and exchange counts
must match bit-exact: both sides use the same Philox streams and the same quantised
Metropolis / exchange thresholds (computed on each side in FP64; a threshold can differ by
one unit only where exp(.)*2^32 lies within 1e-6 of an integer, which the chosen betas avoid
and which would matter only if a random word hit that value exactly).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SEED = 11


@pytest.fixture(scope="module")
def eamc():
    import torch
    assert torch.cuda.is_available()
    from paper_2011_08560_gb300 import eamc as m
    m.lib()
    return m


def _compare(orc, ctx, dim, L, n, betas, sweeps_list, e_g, e_hot, rid0=0, J=None, reals=None):
    """betas: one list for every realization, or an array [n][M] of per-realization sets."""
    per = np.ndim(betas) == 2
    M = np.shape(betas)[-1]
    if reals is None:
        reals = [orc.PTRealization(dim, L, SEED, rid0 + r, betas[r] if per else betas,
                                   J=None if J is None else J[r]) for r in range(n)]
    ctx.pt_set_rt_bounds(np.full(n, e_g, np.int32), np.full(n, e_hot, np.int32))
    for sw in sweeps_list:
        ctx.pt_run(sw, count_roundtrips=True)
        for p in reals:
            p.sweeps(sw, count_rt=True, e_g=e_g, e_hot=e_hot)
        S, E, lab, t = ctx.pt_state()
        R = ctx.pt_roundtrips()
        for r, p in enumerate(reals):
            assert np.array_equal(E[r], p.E), (r, E[r], p.E)
            assert np.array_equal(lab[r], p.label), (r, lab[r], p.label)
            assert np.array_equal(S[r].reshape(-1), p.S), r
            for l in range(M):
                want = p.rt[l].as_dict()
                for f in ("phase", "n_rt", "t_first", "t_last", "e_min"):
                    assert R[r][l][f] == want[f], (r, l, f, R[r][l][f], want[f])
        assert t == reals[0].t
    swaps = ctx.pt_swap_counts()
    want = np.sum([p.swap_acc for p in reals], axis=0)
    assert np.array_equal(swaps, want)
    return reals


@pytest.mark.parametrize("dim,L,n,betas,sweeps,eg,ehot", [
    (2, 4, 40, [0.2, 0.5, 0.9, 1.4], [60, 90], -20, -8),
    (3, 3, 40, [0.2, 0.4, 0.7, 1.1, 1.6, 2.2, 3.0], [50, 30], -40, -16),       # odd L: 3 colours
    (3, 5, 33, list(np.geomspace(0.25, 3.0, 12)), [12, 9], -180, -80),
    (2, 5, 35, [0.3, 0.8, 1.5], [40], -40, -15),
    (3, 7, 3, [0.3, 0.6, 1.0, 1.5, 2.2], [4, 3], -500, -200),
    (2, 3, 9, [0.4, 1.2], [30], -10, -2),
    (3, 4, 33, [0.25, 0.4, 0.6, 0.8, 1.0, 1.2, 1.5, 1.9], [30, 20], -90, -40),
    (3, 6, 5, list(np.geomspace(0.2, 3.0, 32)), [6, 4], -300, -150),
    (3, 8, 3, [0.3, 0.9, 1.6, 2.4], [3, 2], -700, -300),
    (2, 6, 70, [0.3, 0.6, 1.0, 1.5, 2.2, 3.0], [40], -55, -20),
])
def test_pt_bit_exact(eamc, orc, dim, L, n, betas, sweeps, eg, ehot):
    ctx = eamc.Context(seed=SEED)
    ctx.pt_init(dim, L, n, betas)
    S0, E0, lab0, _ = ctx.pt_state()
    p0 = orc.PTRealization(dim, L, SEED, 0, betas)
    assert np.array_equal(E0[0], p0.E) and np.array_equal(S0[0].reshape(-1), p0.S)
    reals = _compare(orc, ctx, dim, L, n, betas, sweeps, eg, ehot)
    assert sum(int(p.swap_acc.sum()) for p in reals) > 0


def test_pt_explicit_couplings_and_offset_ids(eamc, orc):
    dim, L, n, betas = 3, 4, 7, [0.3, 0.7, 1.2, 2.0]
    J = np.stack([orc.make_disorder(dim, L, 5, 1000 + r) for r in range(n)])
    ctx = eamc.Context(seed=SEED)
    ctx.pt_init(dim, L, n, betas, rid0=64, couplings=J)
    _compare(orc, ctx, dim, L, n, betas, [25], -90, -40, rid0=64, J=J)


def test_pt_errors(eamc):
    ctx = eamc.Context(seed=SEED)
    with pytest.raises(eamc.EamcError):
        ctx.pt_run(1)                                   # no PT batch
    with pytest.raises(eamc.EamcError):
        ctx.pt_init(3, 13, 4, [0.1, 0.2])               # L out of range
    with pytest.raises(eamc.EamcError):
        ctx.pt_init(3, 4, 4, [0.5, 0.2])                # betas not increasing
    with pytest.raises(eamc.EamcError):
        ctx.pt_init(3, 4, 4, [0.1, 0.2], rid0=3)        # unaligned realization ids


def test_pt_full_size_sampled(eamc, orc):
    """The PT workload (L=8, 1024 realizations x 32 temperatures) at full size: 20 sweeps, then
    60 with round trips counted between per-realization bounds; sampled realizations checked
    against the oracle (spins, energies, labels, per-replica round-trip records, exchange
    counts per pair)."""
    from paper_2011_08560_gb300.workloads import PT, geometric_betas
    betas = geometric_betas(PT["M"], PT["beta_min"], PT["beta_max"])
    n, M = PT["n_real"], PT["M"]
    ctx = eamc.Context(seed=PT["seed"])
    ctx.pt_init(PT["dim"], PT["L"], n, betas)
    ctx.pt_run(20)
    _, E0, _, _ = ctx.pt_state(spins=False)
    # a narrow band around the middle temperature's energy, so that round trips happen within
    # 60 sweeps
    e_hot = E0[:, M // 2].astype(np.int32)
    e_g = (E0[:, M // 2] - 30).astype(np.int32)
    ctx.pt_roundtrips(reset=True)
    ctx.pt_set_rt_bounds(e_g, e_hot)
    ctx.pt_run(60, count_roundtrips=True)
    S, E, lab, t = ctx.pt_state()
    R = ctx.pt_roundtrips()
    acc, att = ctx.pt_exchange_counts()
    total = 0
    for rid in (0, 517, 1023):
        p = orc.PTRealization(PT["dim"], PT["L"], PT["seed"], rid, betas)
        p.sweeps(20)
        for k in range(M):
            p.rt[p.label[k]] = orc.RT(phase=0, n_rt=0, t_first=-1, t_last=-1, e_min=int(p.E[k]),
                                      e_g=0, requeue=0, pad=0)
        p.sweeps(60, count_rt=True, e_g=int(e_g[rid]), e_hot=int(e_hot[rid]))
        assert np.array_equal(E[rid], p.E) and np.array_equal(lab[rid], p.label)
        assert np.array_equal(S[rid].reshape(-1), p.S)
        for l in range(M):
            want = p.rt[l].as_dict()
            for f in ("phase", "n_rt", "t_first", "t_last", "e_min"):
                assert R[rid][l][f] == want[f], (rid, l, f)
            total += want["n_rt"]
        a, tt = p.window_rates()
        assert np.array_equal(acc[rid], a.astype(np.uint32)) and np.array_equal(att, tt)
    assert total > 0


def test_pt_per_realization_temperatures(eamc, orc):
    dim, L, n, M = 3, 4, 45, 6
    rng = np.random.default_rng(3)
    betas = np.sort(rng.uniform(0.15, 2.5, size=(n, M)), axis=1)
    ctx = eamc.Context(seed=SEED)
    ctx.pt_init(dim, L, n, betas[0])
    ctx.pt_set_betas(betas)
    assert np.array_equal(ctx.pt_betas(), betas)
    _compare(orc, ctx, dim, L, n, betas, [40, 25], -90, -40)
    with pytest.raises(eamc.EamcError):
        ctx.pt_set_betas(betas[:, ::-1].copy())          # not increasing


@pytest.mark.parametrize("dim,L,n,M", [(3, 4, 37, 7), (3, 5, 6, 12), (2, 6, 33, 5)])
def test_pt_adaptation_parity(eamc, orc, dim, L, n, M):
    """Counts bit-exact, adapted temperatures to 1e-12, and the runs after each step bit-exact."""
    betas0 = np.geomspace(0.2, 2.8, M)
    ctx = eamc.Context(seed=SEED)
    ctx.pt_init(dim, L, n, betas0)
    reals = [orc.PTRealization(dim, L, SEED, r, betas0) for r in range(n)]
    for step, (sw, eta) in enumerate([(61, 0.5), (40, 0.7), (33, 0.3)]):
        reals = _compare(orc, ctx, dim, L, n, betas0, [sw], -10 ** 6, 10 ** 6, reals=reals)
        acc, att = ctx.pt_exchange_counts()
        for r, p in enumerate(reals):
            a, t = p.window_rates()
            assert np.array_equal(acc[r], a.astype(np.uint32)), (step, r)
            assert np.array_equal(att, t)
        ctx.pt_adapt(eta)
        for p in reals:
            p.adapt(eta)
        got = ctx.pt_betas()
        for r, p in enumerate(reals):
            np.testing.assert_allclose(got[r], p.betas, rtol=1e-12, atol=0)
            assert got[r][0] == betas0[0] and got[r][-1] == betas0[-1]
        assert not ctx.pt_exchange_counts()[0].any()
    assert any(not np.allclose(p.betas, betas0) for p in reals)
