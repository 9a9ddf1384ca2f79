"""GPU MUCA path vs the oracle, element by element, through the C ABI.

Integer state (spins, energies, histograms, round-trip records) must match bit-exact when
both sides use the same acceptance thresholds.  FP64 weights must agree to 1e-12 relative
(the two sides call different exp/log implementations); thresholds quantised from them may
differ by one unit only where p*2^32 lies within 1e-6 of an integer.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SEED = 7


@pytest.fixture(scope="module")
def eamc():
    import torch
    assert torch.cuda.is_available()
    from paper_2011_08560_gb300 import eamc as m
    m.lib()
    return m


def _oracle_chains(orc, dim, L, n, rid0=0, stream=0, seed=SEED, J=None, S=None):
    out = []
    for k in range(n):
        out.append(orc.Chain(dim, L, seed, rid0 + k, stream,
                             J=None if J is None else J[k], S=None if S is None else S[k]))
    return out


def _random_lnw(rng, b_top, scale):
    # a rough, non-monotone weight profile that still favours low energies
    steps = rng.normal(0.3 * scale, scale, size=b_top + 1)
    lnW = np.cumsum(steps[::-1])[::-1].copy()
    return lnW - lnW[b_top]


def _pad(rows, width):
    out = np.zeros((len(rows), width), dtype=rows[0].dtype)
    for k, r in enumerate(rows):
        out[k, :len(r)] = r
    return out


def _compare_state(ctx, chains, chain0=0, hist=True, rt=True):
    n = len(chains)
    S, E, t = ctx.state(chain0, n)
    for k, c in enumerate(chains):
        assert np.array_equal(S[k, :c.V], c.S), f"chain {k}: spins differ"
        assert E[k] == c.E, f"chain {k}: E {E[k]} vs {c.E}"
        assert t[k] == c.t
    if hist:
        H = ctx.histograms(chain0, n)
        for k, c in enumerate(chains):
            assert np.array_equal(H[k, :c.b_top + 1], c.hist), f"chain {k}: histogram differs"
    if rt:
        R = ctx.roundtrips(chain0, n)
        for k, c in enumerate(chains):
            want = c.rt.as_dict()
            got = R[k]
            for f in ("phase", "n_rt", "t_first", "t_last", "e_min", "requeue"):
                assert got[f] == want[f], f"chain {k}: rt.{f} {got[f]} vs {want[f]}"


@pytest.mark.parametrize("dim,L,n", [(3, 4, 40), (3, 3, 33), (3, 5, 7), (3, 6, 64), (2, 4, 35),
                                     (2, 6, 5), (3, 8, 3), (3, 12, 2), (3, 4, 1)])
def test_init_matches_oracle(eamc, orc, dim, L, n):
    ctx = eamc.Context(seed=SEED)
    first = ctx.init_disorder(dim, L, n, rid0=3)
    assert first == 0 and ctx.num_chains() == n
    chains = _oracle_chains(orc, dim, L, n, rid0=3)
    desc = ctx.describe()
    for k, c in enumerate(chains):
        assert desc[k]["b_top"] == c.b_top and desc[k]["parity"] == c.parity
        assert desc[k]["rid"] == 3 + k
    _compare_state(ctx, chains, hist=False, rt=False)


@pytest.mark.parametrize("dim,L,n,sweeps", [(3, 4, 40, 120), (3, 3, 33, 100), (3, 5, 7, 40),
                                            (3, 6, 64, 30), (2, 4, 35, 300), (3, 8, 3, 20),
                                            (3, 12, 2, 4), (3, 4, 1, 200)])
def test_sweeps_bit_exact_with_injected_thresholds(eamc, orc, dim, L, n, sweeps):
    rng = np.random.default_rng(L * 100 + n)
    ctx = eamc.Context(seed=SEED)
    ctx.init_disorder(dim, L, n, rid0=11, stream=2)
    chains = _oracle_chains(orc, dim, L, n, rid0=11, stream=2)
    thr = [orc.quantize(dim, _random_lnw(rng, c.b_top, 0.4)) for c in chains]
    ctx.set_thresholds(0, _pad(thr, max(len(t) for t in thr)))
    # E_g for round trips: a few bins above the lowest energy the descent found
    eg = np.array([c.E - 8 for c in chains], dtype=np.int32)
    ctx.set_eg(0, n, eg)
    for c, e in zip(chains, eg):
        c.rt.e_g = int(e)
    for part in (sweeps // 3, sweeps - sweeps // 3):
        ctx.run_sweeps(part, count_roundtrips=True)
        for c, th in zip(chains, thr):
            c.sweeps(part, th, count_rt=True)
        _compare_state(ctx, chains)


def _injected_run(eamc, orc, ctx, chains, chain0, thr, sweeps, parts=2):
    """Inject thresholds, set E_g a little below the start and sweep both sides in parts."""
    n = len(chains)
    ctx.set_thresholds(chain0, _pad(thr, max(len(t) for t in thr)))
    eg = np.array([c.E - 8 for c in chains], dtype=np.int32)
    ctx.set_eg(chain0, n, eg)
    for c, e in zip(chains, eg):
        c.rt.e_g = int(e)
    done = 0
    for k in range(parts):
        part = sweeps // parts if k < parts - 1 else sweeps - done
        ctx.run_sweeps(part, count_roundtrips=True)
        for c, th in zip(chains, thr):
            c.sweeps(part, th, count_rt=True)
        done += part
        _compare_state(ctx, chains, chain0)


@pytest.mark.parametrize("L,n,sweeps", [(8, 32, 200), (9, 32, 200), (10, 32, 200), (11, 32, 200),
                                        (12, 32, 200)])
def test_large_lattices_full_tile(eamc, orc, L, n, sweeps):
    """Full tiles at the sizes with thresholds read through L1 (L >= 7) and 64-bit row words
    (L >= 9), with round-trip counting."""
    rng = np.random.default_rng(1000 + L)
    ctx = eamc.Context(seed=SEED)
    ctx.init_disorder(3, L, n, rid0=200, stream=1)
    chains = _oracle_chains(orc, 3, L, n, rid0=200, stream=1)
    thr = [orc.quantize(3, _random_lnw(rng, c.b_top, 0.4)) for c in chains]
    _injected_run(eamc, orc, ctx, chains, 0, thr, sweeps)
    assert sum(c.rt.n_rt for c in chains) > 0 or L >= 11   # round trips exercised


@pytest.mark.parametrize("L,n,sweeps", [(7, 19, 150), (8, 33, 200), (8, 16, 60)])
def test_narrow_tiles_bit_exact(eamc, orc, L, n, sweeps):
    """Tiles of 16 chains (thresholds in shared memory at L = 7, 8): ragged last tiles, the
    same trajectories as the oracle."""
    info = eamc.tile_width_info(3, L, 16)
    assert info is not None and info[1], "width 16 keeps the thresholds in shared memory"
    assert eamc.tile_width_info(3, L, 32)[1] is False
    rng = np.random.default_rng(2000 + L + n)
    ctx = eamc.Context(seed=SEED)
    ctx.set_tile_width(L, 16)
    ctx.init_disorder(3, L, n, rid0=300, stream=4)
    chains = _oracle_chains(orc, 3, L, n, rid0=300, stream=4)
    desc = ctx.describe()
    for k, c in enumerate(chains):
        assert desc[k]["rid"] == 300 + k and desc[k]["b_top"] == c.b_top
    thr = [orc.quantize(3, _random_lnw(rng, c.b_top, 0.4)) for c in chains]
    _injected_run(eamc, orc, ctx, chains, 0, thr, sweeps, parts=3)
    ctx.check()


@pytest.mark.parametrize("persistent", [False, True])
def test_mixed_widths_in_one_context(eamc, orc, persistent):
    """Narrow L = 8 tiles beside full L = 6 tiles and caller couplings, one launch; then the
    plain weight iteration (thresholds requantised on the device)."""
    ctx = eamc.Context(seed=SEED)
    ctx.set_tile_width(8, 16)
    J8 = np.stack([orc.make_disorder(3, 8, 5, 40 + k) for k in range(21)])
    ctx.init_disorder(3, 8, 21, rid0=40, couplings=J8)
    ctx.init_disorder(3, 6, 35, rid0=70, stream=2)
    ctx.set_ensemble(0, 21, eamc.EA_POWERLAW, -3.6, 96.0)
    ctx.set_launch(persistent, 0, 0)
    chains = _oracle_chains(orc, 3, 8, 21, rid0=40, J=J8) + _oracle_chains(orc, 3, 6, 35, rid0=70, stream=2)
    kinds = [orc.POWERLAW] * 21 + [orc.FLAT] * 35
    lnW = [np.zeros(c.b_top + 1) for c in chains]
    for _ in range(3):
        ctx.run_sweeps(40)
        ctx.update_weights()
        for k, c in enumerate(chains):
            c.sweeps(40, orc.quantize(3, lnW[k]))
            lnW[k] = orc.update_weights(3, c.L, c.parity, kinds[k], -3.6, 96.0, c.rt.e_min, lnW[k], c.hist)
            c.hist[:] = 0
        _compare_state(ctx, chains, hist=True, rt=False)
        G = ctx.get_weights()
        for k, c in enumerate(chains):
            assert _close(G[k, :c.b_top + 1], lnW[k])
    ctx.check()


def test_tile_width_rejects_unavailable(eamc):
    ctx = eamc.Context(seed=SEED)
    for L, w in ((12, 16), (6, 4), (3, 8), (8, 4), (8, 64)):
        with pytest.raises(eamc.EamcError):
            ctx.set_tile_width(L, w)
    assert eamc.tile_width_info(3, 6, 16) is None
    assert eamc.narrow_width(3, 8) == 16 and eamc.narrow_width(3, 6) == 32


def test_zero_sweeps_and_errors(eamc, orc):
    ctx = eamc.Context(seed=SEED)
    with pytest.raises(eamc.EamcError):
        ctx.run_sweeps(1)                       # no chains yet
    with pytest.raises(eamc.EamcError):
        ctx.init_disorder(4, 4, 1)              # bad dim
    with pytest.raises(eamc.EamcError):
        ctx.init_disorder(3, 2, 1)              # L too small
    with pytest.raises(eamc.EamcError):
        ctx.init_disorder(3, 4, 0)              # empty batch
    ctx.init_disorder(3, 4, 3)
    with pytest.raises(eamc.EamcError):
        ctx.init_disorder(2, 4, 3)              # one dim per context
    with pytest.raises(eamc.EamcError):
        ctx.histograms(2, 5)                    # range beyond the chains
    S0, E0, _ = ctx.state()
    ctx.run_sweeps(0)
    S1, E1, t1 = ctx.state()
    assert np.array_equal(S0, S1) and np.array_equal(E0, E1) and t1.max() == 0


def test_explicit_couplings_and_spins(eamc, orc):
    """Caller-provided couplings (here gauge-transformed) give the oracle's trajectory."""
    dim, L, n = 3, 4, 5
    rng = np.random.default_rng(3)
    J = np.stack([orc.make_disorder(dim, L, 99, k) for k in range(n)])
    S = rng.choice([-1, 1], size=(n, 64)).astype(np.int8)
    ctx = eamc.Context(seed=SEED)
    ctx.init_disorder(dim, L, n, rid0=50, couplings=J, spins=S)
    chains = _oracle_chains(orc, dim, L, n, rid0=50, J=J, S=S)
    thr = [orc.quantize(dim, np.zeros(c.b_top + 1)) for c in chains]
    ctx.set_thresholds(0, _pad(thr, max(len(t) for t in thr)))
    ctx.run_sweeps(50)
    for c, th in zip(chains, thr):
        c.sweeps(50, th)
    _compare_state(ctx, chains, rt=False)


def _oracle_iteration(orc, c, kind, alpha, pole, sweeps, lnW):
    c.sweeps(sweeps, orc.quantize(c.dim, lnW))
    new = orc.update_weights(c.dim, c.L, c.parity, kind, alpha, pole, c.rt.e_min, lnW, c.hist)
    c.hist[:] = 0
    return new


def _close(a, b, rel=1e-12):
    scale = max(1.0, float(np.max(np.abs(b))))
    return float(np.max(np.abs(a - b))) <= rel * scale


def _thresholds_agree(orc, dim, got, lnW_oracle):
    want = orc.quantize(dim, lnW_oracle)
    got = got[:len(want)]
    bad = np.nonzero(got != want)[0]
    for idx in bad:
        b, nn = divmod(int(idx), 8)
        bn = b + dim - nn
        x = lnW_oracle[bn] - lnW_oracle[b]
        q = np.exp(x) * 2.0 ** 32
        assert abs(int(got[idx]) - int(want[idx])) <= 1
        assert min(q - np.floor(q), np.ceil(q) - q) < 1e-6, (b, nn, q)
    return len(bad)


@pytest.mark.parametrize("kind", [0, 1])
def test_weight_iteration_parity(eamc, orc, kind):
    dim, L, n = 3, 4, 33
    alpha, pole = -3.6, 96.0
    ctx = eamc.Context(seed=SEED)
    ctx.init_disorder(dim, L, n, rid0=200)
    ctx.set_ensemble(0, n, kind, alpha, pole)
    chains = _oracle_chains(orc, dim, L, n, rid0=200)
    lnW = [np.zeros(c.b_top + 1) for c in chains]
    for it in range(6):
        ctx.run_sweeps(150)
        ctx.update_weights()
        lnW = [_oracle_iteration(orc, c, kind, alpha, pole, 150, w) for c, w in zip(chains, lnW)]
        G = ctx.get_weights()
        T = ctx.get_thresholds()
        for k, c in enumerate(chains):
            assert _close(G[k, :c.b_top + 1], lnW[k]), (it, k)
            _thresholds_agree(orc, dim, T[k], lnW[k])
        _compare_state(ctx, chains, hist=True, rt=False)
    ctx.check()


@pytest.mark.parametrize("kind", [0, 1])
def test_berg_recursion_parity(eamc, orc, kind):
    """Berg's accumulated recursion on every other chain, the plain step on the rest."""
    dim, L, n = 3, 4, 37
    alpha, pole = -3.6, 96.0
    ctx = eamc.Context(seed=SEED)
    ctx.init_disorder(dim, L, n, rid0=500)
    ctx.set_ensemble(0, n, kind, alpha, pole)
    berg = [k % 2 == 0 for k in range(n)]
    for k in range(n):
        if berg[k]:
            ctx.set_recursion(k, 1, eamc.EA_REC_BERG)
    chains = _oracle_chains(orc, dim, L, n, rid0=500)
    lnW = [np.zeros(c.b_top + 1) for c in chains]
    acc = [orc.berg_state(c.b_top + 1) for c in chains]
    for it in range(6):
        ctx.run_sweeps(150)
        ctx.update_weights()
        for k, c in enumerate(chains):
            c.sweeps(150, orc.quantize(dim, lnW[k]))
            if berg[k]:
                lnW[k] = orc.update_weights_berg(dim, L, c.parity, kind, alpha, pole, c.rt.e_min,
                                                 lnW[k], c.hist, acc[k])
            else:
                lnW[k] = orc.update_weights(dim, L, c.parity, kind, alpha, pole, c.rt.e_min,
                                            lnW[k], c.hist)
            c.hist[:] = 0
        G = ctx.get_weights()
        T = ctx.get_thresholds()
        A = ctx.recursion_state()
        for k, c in enumerate(chains):
            assert _close(G[k, :c.b_top + 1], lnW[k]), (it, k)
            _thresholds_agree(orc, dim, T[k], lnW[k])
            want = acc[k] if berg[k] else np.zeros_like(acc[k])
            assert _close(A[k, :c.b_top + 1, 0], want[0]), (it, k, "D")
            assert _close(A[k, :c.b_top + 1, 1], want[1]), (it, k, "G")
        _compare_state(ctx, chains, hist=True, rt=False)
    assert np.any(A[0, :, 1] > 0)


def test_berg_subset_update_and_reset(eamc, orc):
    dim, L, n = 3, 5, 6
    ctx = eamc.Context(seed=SEED)
    ctx.init_disorder(dim, L, n, rid0=600)
    ctx.set_recursion(0, n, eamc.EA_REC_BERG)
    chains = _oracle_chains(orc, dim, L, n, rid0=600)
    lnW = [np.zeros(c.b_top + 1) for c in chains]
    acc = [orc.berg_state(c.b_top + 1) for c in chains]
    sel = [1, 4]
    for it in range(3):
        ctx.run_sweeps(80)
        for c, w in zip(chains, lnW):
            c.sweeps(80, orc.quantize(dim, w))
        ctx.update_weights_subset(sel)
        for k in sel:
            c = chains[k]
            lnW[k] = orc.update_weights_berg(dim, L, c.parity, 0, -3.6, 96.0, c.rt.e_min, lnW[k],
                                             c.hist, acc[k])
            c.hist[:] = 0
    G = ctx.get_weights()
    for k, c in enumerate(chains):
        assert _close(G[k, :c.b_top + 1], lnW[k]), k
    # re-setting the recursion empties the accumulators; a lane reset returns it to plain
    ctx.set_recursion(1, 1, eamc.EA_REC_BERG)
    assert not ctx.recursion_state(1, 1).any()
    assert ctx.recursion_state(4, 1)[0, :, 1].any()
    with pytest.raises(eamc.EamcError):
        ctx.set_recursion(0, 1, 7)


@pytest.mark.parametrize("kind", [0, 1, 2, 3])
def test_build_ensemble_parity(eamc, orc, kind):
    dim, L, n = 3, 4, 6
    ctx = eamc.Context(seed=SEED)
    ctx.init_disorder(dim, L, n, rid0=300)
    ctx.set_ensemble(0, n, 1, -3.6, 96.0)          # current weights are a power-law iteration
    chains = _oracle_chains(orc, dim, L, n, rid0=300)
    rng = np.random.default_rng(kind)
    lnW = [_random_lnw(rng, c.b_top, 0.5) for c in chains]
    ctx.set_weights(0, _pad(lnW, max(len(w) for w in lnW)))
    ctx.set_eg(0, n, np.array([c.E - 12 for c in chains], dtype=np.int32))
    ctx.build_ensemble(0, n, kind, alpha=-2.5, pole=50.0, beta=0.7)
    G = ctx.get_weights()
    for k, c in enumerate(chains):
        eg = c.E - 12
        lnP = np.array([orc.ln_profile(1, -3.6, 96.0, eg, orc.energy_of_bin(dim, L, c.parity, b))
                        for b in range(c.b_top + 1)])
        lnO = lnP - lnW[k]
        want = orc.build_weights(dim, L, c.parity, kind, -2.5, 50.0, 0.7, eg, lnO)
        assert _close(G[k, :c.b_top + 1], want), k
    assert [d["kind"] for d in ctx.describe()] == [kind] * n


def test_roundtrip_reset_and_requeue(eamc, orc):
    dim, L, n = 3, 4, 4
    ctx = eamc.Context(seed=SEED)
    ctx.init_disorder(dim, L, n, rid0=400)
    chains = _oracle_chains(orc, dim, L, n, rid0=400)
    thr = [orc.quantize(dim, np.zeros(c.b_top + 1)) for c in chains]
    ctx.set_thresholds(0, _pad(thr, max(len(t) for t in thr)))
    # an E_g above the reachable minimum forces the requeue flag
    eg = np.array([c.E + 20 for c in chains], dtype=np.int32)
    ctx.set_eg(0, n, eg)
    for c, e in zip(chains, eg):
        c.rt.e_g = int(e)
    ctx.run_sweeps(300, count_roundtrips=True)
    for c, th in zip(chains, thr):
        c.sweeps(300, th, count_rt=True)
    R = ctx.roundtrips(reset=True)
    for k, c in enumerate(chains):
        assert R[k]["requeue"] == c.rt.requeue == 1
        assert R[k]["n_rt"] == c.rt.n_rt
    R2 = ctx.roundtrips()
    S, E, _ = ctx.state()
    for k in range(n):
        assert R2[k]["n_rt"] == 0 and R2[k]["phase"] == 0 and R2[k]["requeue"] == 0
        assert R2[k]["e_min"] == E[k]


def test_reset_chains_match_fresh_oracle_chains(eamc, orc):
    """ea_reset_chains (a lane taking a new job) gives exactly a fresh oracle chain of the new
    realization and stream, and leaves the other chains of the tile on their trajectories."""
    dim, L, n = 3, 5, 40
    ctx = eamc.Context(seed=SEED)
    ctx.init_disorder(dim, L, n, rid0=60, stream=1)
    ctx.set_ensemble(0, n, eamc.EA_POWERLAW, -3.6, 96.0)
    chains = _oracle_chains(orc, dim, L, n, rid0=60, stream=1)
    lnW = [np.zeros(c.b_top + 1) for c in chains]
    for _ in range(2):
        ctx.run_sweeps(30)
        ctx.update_weights()
        for k, c in enumerate(chains):
            c.sweeps(30, orc.quantize(dim, lnW[k]))
            lnW[k] = orc.update_weights(dim, L, c.parity, orc.POWERLAW, -3.6, 96.0, c.rt.e_min, lnW[k], c.hist)
            c.hist[:] = 0
    picked = [3, 17, 38]
    new_rid, new_stream = [901, 902, 903], [7, 0, 5]
    ctx.reset_chains(picked, new_rid, new_stream)
    for k, r, s in zip(picked, new_rid, new_stream):
        chains[k] = orc.Chain(dim, L, SEED, r, s)      # a fresh chain: flat weights, t = 0
        lnW[k] = np.zeros(chains[k].b_top + 1)
    desc = ctx.describe()
    for k, r, s in zip(picked, new_rid, new_stream):
        assert desc[k]["rid"] == r and desc[k]["stream"] == s and desc[k]["t"] == 0
        assert desc[k]["kind"] == eamc.EA_FLAT
    W = ctx.get_weights()
    for k in picked:
        assert not W[k, :chains[k].b_top + 1].any()
    _compare_state(ctx, chains, hist=True, rt=True)
    # every chain continues exactly (the reset ones as fresh flat chains)
    ctx.run_sweeps(25, count_roundtrips=False)
    for k, c in enumerate(chains):
        c.sweeps(25, orc.quantize(dim, lnW[k]))
    _compare_state(ctx, chains, hist=True, rt=False)
