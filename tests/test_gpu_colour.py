"""The colour-order sweep kernels against the oracle's colour order, element by element: spins,
energies, histograms and round-trip records bit-exact, weights to 1e-12.  One kernel, one lane
per chain, for every L: even L two colour passes, odd L three with rows padded to the most
colour sites of a row; records of two to eight rows or a plane, one or two records of look-ahead,
padded last records, 2D and 3D, full and narrow tiles; launch splitting, captured graphs,
contexts holding both parities and the weight recursions (the chains-per-CTA argument has no
effect)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SEED = 13


@pytest.fixture(scope="module")
def eamc():
    import torch
    assert torch.cuda.is_available()
    from paper_2011_08560_gb300 import eamc as m
    m.lib()
    return m


def _chains(orc, dim, L, n, rid0, stream=0):
    return [orc.Chain(dim, L, SEED, rid0 + k, stream, order=1) for k in range(n)]


def _random_lnw(rng, b_top, scale):
    steps = rng.normal(0.3 * scale, scale, size=b_top + 1)
    lnW = np.cumsum(steps[::-1])[::-1].copy()
    return lnW - lnW[b_top]


def _pad(rows):
    w = max(len(r) for r in rows)
    out = np.zeros((len(rows), w), dtype=rows[0].dtype)
    for k, r in enumerate(rows):
        out[k, :len(r)] = r
    return out


def _compare(ctx, chains, chain0=0, hist=True, rt=True):
    n = len(chains)
    S, E, t = ctx.state(chain0, n)
    for k, c in enumerate(chains):
        assert np.array_equal(S[k, :c.V], c.S), f"chain {k}: spins differ"
        assert E[k] == c.E, (k, E[k], c.E)
        assert t[k] == c.t
    if hist:
        H = ctx.histograms(chain0, n)
        for k, c in enumerate(chains):
            assert np.array_equal(H[k, :c.b_top + 1], c.hist), f"chain {k}: histogram differs"
    if rt:
        R = ctx.roundtrips(chain0, n)
        for k, c in enumerate(chains):
            want = c.rt.as_dict()
            for f in ("phase", "n_rt", "t_first", "t_last", "e_min", "requeue"):
                assert R[k][f] == want[f], (k, f, R[k][f], want[f])


@pytest.mark.parametrize("dim,L,n,sweeps,cpc", [
    (3, 4, 40, 120, 0), (3, 3, 33, 100, 4), (3, 5, 7, 40, 2), (3, 6, 64, 40, 8), (2, 4, 35, 300, 8),
    (2, 5, 9, 200, 1), (3, 7, 19, 40, 0), (3, 8, 32, 30, 4), (3, 9, 5, 12, 0), (3, 10, 33, 8, 2),
    (3, 11, 3, 6, 1), (3, 12, 3, 5, 0), (3, 4, 1, 200, 0),
    (2, 6, 33, 200, 0), (2, 8, 5, 150, 0), (2, 10, 9, 100, 0), (2, 12, 40, 60, 0),
    (3, 10, 40, 24, 0), (3, 12, 33, 16, 0)])
def test_colour_sweeps_bit_exact(eamc, orc, dim, L, n, sweeps, cpc):
    rng = np.random.default_rng(L * 100 + n)
    ctx = eamc.Context(seed=SEED)
    ctx.init_disorder(dim, L, n, rid0=11, stream=2)
    ctx.set_sweep_order(eamc.EA_ORDER_COLOUR, cpc)
    chains = _chains(orc, dim, L, n, 11, 2)
    thr = [orc.quantize(dim, _random_lnw(rng, c.b_top, 0.4)) for c in chains]
    ctx.set_thresholds(0, _pad(thr))
    eg = np.array([c.E - 8 for c in chains], dtype=np.int32)
    ctx.set_eg(0, n, eg)
    for c, e in zip(chains, eg):
        c.rt.e_g = int(e)
    for part in (sweeps // 3, sweeps - sweeps // 3):
        ctx.run_sweeps(part, count_roundtrips=True)
        for c, th in zip(chains, thr):
            c.sweeps(part, th, count_rt=True)
        _compare(ctx, chains)
    ctx.check()
    assert sum(c.rt.n_rt for c in chains) > 0 or L >= 9


def test_block_sizes_split_launches_and_graph_agree(eamc, orc):
    """Every chains-per-CTA choice, launches split into pieces and a captured graph of
    (sweeps + weight update) iterations give the oracle's trajectories."""
    import torch
    dim, L, n = 3, 6, 45
    results = []
    for cpc, spl, graph in ((1, 0, False), (2, 7, False), (4, 0, True), (8, 0, False), (8, 5, True), (0, 0, False)):
        stream = torch.cuda.Stream()
        ctx = eamc.Context(seed=SEED, stream=stream.cuda_stream)
        ctx.init_disorder(dim, L, n, rid0=70)
        ctx.set_ensemble(0, n, eamc.EA_POWERLAW, -3.6, 96.0)
        ctx.set_sweep_order(eamc.EA_ORDER_COLOUR, cpc)
        ctx.set_launch(False, spl, 0)
        if graph:
            ctx.graph_capture(n_iter=3, sweeps_per_iter=20, count_roundtrips=True, update_weights=True)
            ctx.graph_launch(1)
        else:
            for _ in range(3):
                ctx.run_sweeps(20, count_roundtrips=True)
                ctx.update_weights()
        ctx.synchronize()
        S, E, t = ctx.state()
        results.append((S, E, ctx.get_weights(), [r["n_rt"] for r in ctx.roundtrips()]))
        ctx.close()
    chains = _chains(orc, dim, L, n, 70)
    lnW = [np.zeros(c.b_top + 1) for c in chains]
    for _ in range(3):
        for k, c in enumerate(chains):
            c.sweeps(20, orc.quantize(dim, lnW[k]), count_rt=True)
            lnW[k] = orc.update_weights(dim, L, c.parity, orc.POWERLAW, -3.6, 96.0, c.rt.e_min, lnW[k], c.hist)
            c.hist[:] = 0
            c.rt.e_g = c.rt.e_min
    for S, E, W, nrt in results:
        for k, c in enumerate(chains):
            assert np.array_equal(S[k, :c.V], c.S) and E[k] == c.E
            np.testing.assert_allclose(W[k, :c.b_top + 1], lnW[k], rtol=0, atol=1e-11)
            assert nrt[k] == c.rt.n_rt


def test_colour_berg_mixed_sizes_and_narrow_tiles(eamc, orc):
    """Berg's recursion with the colour order, chains of two sizes in one context, one of them in
    16-chain tiles."""
    ctx = eamc.Context(seed=SEED)
    ctx.set_tile_width(8, 16)
    ctx.init_disorder(3, 8, 20, rid0=5)
    ctx.init_disorder(3, 5, 34, rid0=40, stream=3)
    n = 54
    ctx.set_ensemble(0, n, eamc.EA_POWERLAW, -3.6, 96.0)
    ctx.set_recursion(0, n, eamc.EA_REC_BERG)
    ctx.set_sweep_order(eamc.EA_ORDER_COLOUR)
    chains = _chains(orc, 3, 8, 20, 5) + _chains(orc, 3, 5, 34, 40, 3)
    lnW = [np.zeros(c.b_top + 1) for c in chains]
    acc = [orc.berg_state(c.b_top + 1) for c in chains]
    for _ in range(4):
        ctx.run_sweeps(25)
        ctx.update_weights()
        for k, c in enumerate(chains):
            c.sweeps(25, orc.quantize(3, lnW[k]))
            lnW[k] = orc.update_weights_berg(3, c.L, c.parity, orc.POWERLAW, -3.6, 96.0, c.rt.e_min, lnW[k],
                                             c.hist, acc[k])
            c.hist[:] = 0
    _compare(ctx, chains, hist=True, rt=False)
    W = ctx.get_weights()
    for k, c in enumerate(chains):
        np.testing.assert_allclose(W[k, :c.b_top + 1], lnW[k], rtol=0, atol=1e-11)
    ctx.check()


def test_sweep_order_rejects_bad_arguments(eamc):
    ctx = eamc.Context(seed=SEED)
    for order, cpc in ((2, 0), (1, 3), (1, 16), (-1, 0)):
        with pytest.raises(eamc.EamcError):
            ctx.set_sweep_order(order, cpc)


def test_colour_snapshot_resume_and_narrow_tiles(eamc, orc):
    """The colour order continues a snapshot bit-exactly (the order is the caller's setting, not
    part of the snapshot): 2 x 30 sweeps straight == 30, snapshot, restore, 30; chains of an even
    (16-chain tiles) and an odd size (three colour passes) in one context;
    the oracle's colour order agrees."""
    def make():
        ctx = eamc.Context(seed=SEED)
        ctx.set_sweep_order(eamc.EA_ORDER_COLOUR)
        ctx.set_tile_width(8, 16)
        ctx.init_disorder(3, 8, 18, rid0=3)
        ctx.init_disorder(3, 7, 5, rid0=30, stream=1)
        ctx.set_ensemble(0, 23, eamc.EA_POWERLAW, -3.6, 96.0)
        return ctx

    def run(ctx, steps):
        for _ in range(steps):
            ctx.run_sweeps(30, count_roundtrips=True)
            ctx.update_weights()

    straight = make()
    run(straight, 2)
    first = make()
    run(first, 1)
    blob = first.snapshot()
    resumed = eamc.Context(seed=999)
    resumed.restore(blob)
    resumed.set_sweep_order(eamc.EA_ORDER_COLOUR)
    run(resumed, 1)
    S1, E1, t1 = straight.state()
    S2, E2, t2 = resumed.state()
    assert np.array_equal(S1, S2) and np.array_equal(E1, E2) and np.array_equal(t1, t2)
    assert np.array_equal(straight.get_weights(), resumed.get_weights())
    chains = _chains(orc, 3, 8, 18, 3) + _chains(orc, 3, 7, 5, 30, 1)
    lnW = [np.zeros(c.b_top + 1) for c in chains]
    for _ in range(2):
        for k, c in enumerate(chains):
            c.sweeps(30, orc.quantize(3, lnW[k]), count_rt=True)
            lnW[k] = orc.update_weights(3, c.L, c.parity, orc.POWERLAW, -3.6, 96.0, c.rt.e_min, lnW[k], c.hist)
            c.hist[:] = 0
            c.rt.e_g = c.rt.e_min
    for k, c in enumerate(chains):
        assert np.array_equal(S2[k, :c.V], c.S) and E2[k] == c.E
    resumed.check()


@pytest.mark.parametrize("L,width,n,sweeps", [(4, 16, 37, 40), (4, 8, 13, 40), (5, 16, 20, 30), (5, 8, 11, 30),
                                              (6, 16, 18, 20), (6, 8, 21, 20), (7, 16, 21, 10), (7, 8, 9, 10),
                                              (8, 16, 35, 10), (8, 8, 19, 10), (9, 8, 13, 6),
                                              (10, 8, 9, 6), (11, 4, 6, 6), (12, 4, 5, 6)])
def test_narrow_colour_tiles_bit_exact(eamc, orc, L, width, n, sweeps):
    """Tiles of 16 (L = 4..8), 8 (L = 4..10) and 4 chains (L = 11, 12), each chain on 32 / width
    lanes with its thresholds in shared memory and the producers' rows dealt to the lane groups:
    the colour order's trajectories, a partly filled last tile."""
    info = eamc.tile_width_info(3, L, width, order=1)
    assert info is not None and info[1], info           # thresholds in shared memory
    lex_has_width = eamc.tile_width_info(3, L, width, order=0) is not None
    assert lex_has_width == (width == 16 and L in (7, 8))
    rng = np.random.default_rng(L * 7 + width)
    ctx = eamc.Context(seed=SEED)
    ctx.set_sweep_order(eamc.EA_ORDER_COLOUR)
    ctx.set_tile_width(L, width)
    ctx.init_disorder(3, L, n, rid0=21, stream=1)
    chains = _chains(orc, 3, L, n, 21, 1)
    thr = [orc.quantize(3, _random_lnw(rng, c.b_top, 0.4)) for c in chains]
    ctx.set_thresholds(0, _pad(thr))
    eg = np.array([c.E - 8 for c in chains], dtype=np.int32)
    ctx.set_eg(0, n, eg)
    for c, e in zip(chains, eg):
        c.rt.e_g = int(e)
    ctx.run_sweeps(sweeps, count_roundtrips=True)
    for c, th in zip(chains, thr):
        c.sweeps(sweeps, th, count_rt=True)
    _compare(ctx, chains)
    ctx.check()
    if not lex_has_width:  # the lexicographic kernel has no tiles of this width
        ctx.set_sweep_order(eamc.EA_ORDER_LEX)
        with pytest.raises(eamc.EamcError):
            ctx.run_sweeps(1)


@pytest.mark.parametrize("shapes", [((4, 8, 11), (6, 16, 18), (8, 8, 10)), ((5, 8, 9), (6, 8, 12), (8, 16, 7))])
def test_small_narrow_tiles_in_mixed_contexts(eamc, orc, shapes):
    """Narrow tiles of the small even sizes beside other sizes in one context: with even sizes
    only they run in a kernel form of their own, with an odd size in the form for both parities;
    every chain's trajectory is the oracle's."""
    rng = np.random.default_rng(sum(L * w for L, w, _ in shapes))
    ctx = eamc.Context(seed=SEED)
    ctx.set_sweep_order(eamc.EA_ORDER_COLOUR)
    chains, rid = [], 31
    for L, w, n in shapes:
        ctx.set_tile_width(L, w)
        ctx.init_disorder(3, L, n, rid0=rid, stream=2)
        chains += _chains(orc, 3, L, n, rid, 2)
        rid += n
    thr = [orc.quantize(3, _random_lnw(rng, c.b_top, 0.4)) for c in chains]
    ctx.set_thresholds(0, _pad(thr))
    ctx.run_sweeps(12, count_roundtrips=True)
    for c, th in zip(chains, thr):
        c.sweeps(12, th, count_rt=True)
    _compare(ctx, chains)
    ctx.check()
