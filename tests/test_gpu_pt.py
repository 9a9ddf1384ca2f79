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


def _compare(orc, ctx, dim, L, n, betas, sweeps_list, e_g, e_hot, rid0=0, J=None):
    M = len(betas)
    V = L ** dim
    reals = [orc.PTRealization(dim, L, SEED, rid0 + r, betas, J=None if J is None else J[r])
             for r in range(n)]
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
        ctx.pt_init(3, 5, 4, [0.1, 0.2])                # odd L: no checkerboard
    with pytest.raises(eamc.EamcError):
        ctx.pt_init(3, 4, 4, [0.5, 0.2])                # betas not increasing
    with pytest.raises(eamc.EamcError):
        ctx.pt_init(3, 4, 4, [0.1, 0.2], rid0=3)        # unaligned realization ids


def test_pt_full_size_sampled(eamc, orc):
    """The PT workload (L=8, 1024 realizations x 32 temperatures) at full size, with sampled
    realizations checked against the oracle."""
    from paper_2011_08560_gb300.workloads import PT, geometric_betas
    betas = geometric_betas(PT["M"], PT["beta_min"], PT["beta_max"])
    ctx = eamc.Context(seed=PT["seed"])
    ctx.pt_init(PT["dim"], PT["L"], PT["n_real"], betas)
    ctx.pt_run(3)
    S, E, lab, t = ctx.pt_state()
    for rid in (0, 517, 1023):
        p = orc.PTRealization(PT["dim"], PT["L"], PT["seed"], rid, betas)
        p.sweeps(3)
        assert np.array_equal(E[rid], p.E) and np.array_equal(lab[rid], p.label)
        assert np.array_equal(S[rid].reshape(-1), p.S)
