"""Batched uneven-L launches (a8): persistent work queue, split launches and the captured
iteration graph give exactly the results of the plain launch and of the oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SEED = 13
MIX = [(3, 4, 5), (4, 3, 33), (5, 2, 3), (6, 1, 40), (8, 2, 2), (10, 5, 1), (12, 3, 2)]  # (L, stream, n)


@pytest.fixture(scope="module")
def eamc():
    import torch
    assert torch.cuda.is_available()
    from paper_2011_08560_gb300 import eamc as m
    m.lib()
    return m


def _mixed(eamc, stream_ptr=None):
    ctx = eamc.Context(seed=SEED, stream=stream_ptr)
    rid = 0
    for L, st, n in MIX:
        ctx.init_disorder(3, L, n, rid0=rid, stream=st)
        rid += n
    n_all = ctx.num_chains()
    ctx.set_ensemble(0, n_all // 2, eamc.EA_POWERLAW, -3.6, 96.0)
    return ctx


def _state(ctx):
    S, E, t = ctx.state()
    return S, E, t, ctx.histograms(), ctx.get_weights(), [tuple(r.values()) for r in ctx.roundtrips()]


def _same(a, b):
    for x, y in zip(a, b):
        if isinstance(x, np.ndarray):
            assert np.array_equal(x, y)
        else:
            assert x == y


def _run(ctx, iters, sweeps):
    for _ in range(iters):
        ctx.run_sweeps(sweeps, count_roundtrips=True)
        ctx.update_weights()


def test_persistent_and_split_launches_match_plain(eamc):
    ref = _mixed(eamc)
    _run(ref, 3, 40)
    for persistent, spl in ((True, 0), (False, 7), (True, 13)):
        ctx = _mixed(eamc)
        ctx.set_launch(persistent, spl, 2 if persistent else 0)
        _run(ctx, 3, 40)
        _same(_state(ref), _state(ctx))


def test_mixed_batch_matches_oracle(eamc, orc):
    ctx = _mixed(eamc)
    ctx.set_launch(True, 0)
    ctx.run_sweeps(6, count_roundtrips=False)
    S, E, t = ctx.state()
    H = ctx.histograms()
    chain = 0
    rid = 0
    for L, st, n in MIX:
        for k in (0, n - 1):
            c = orc.Chain(3, L, SEED, rid + k, st)
            c.sweeps(6, orc.quantize(3, np.zeros(c.b_top + 1)))
            idx = chain + k
            assert np.array_equal(S[idx, :c.V], c.S) and E[idx] == c.E
            assert np.array_equal(H[idx, :c.b_top + 1], c.hist)
        chain += n
        rid += n


def test_graph_replay_matches_direct_calls(eamc):
    import torch
    st = torch.cuda.Stream()
    ref = _mixed(eamc, st.cuda_stream)
    ctx = _mixed(eamc, st.cuda_stream)
    for c in (ref, ctx):
        c.set_recursion(30, 20, eamc.EA_REC_BERG)
    ctx.set_launch(True, 0)
    ctx.graph_capture(n_iter=2, sweeps_per_iter=25, count_roundtrips=True, update_weights=True)
    ctx.graph_launch(3)
    ctx.synchronize()
    _run(ref, 6, 25)
    ref.synchronize()
    _same(_state(ref), _state(ctx))
    assert np.array_equal(ref.recursion_state(), ctx.recursion_state())
    ctx.graph_release()
    with pytest.raises(eamc.EamcError):
        ctx.graph_launch(1)
    # adding chains may move the arenas: the captured graph is released
    ctx.graph_capture(n_iter=1, sweeps_per_iter=5)
    ctx.init_disorder(3, 4, 3, rid0=900)
    with pytest.raises(eamc.EamcError):
        ctx.graph_launch(1)


def test_snapshot_resume_is_bit_exact(eamc):
    """Run 2S sweeps straight vs S, snapshot, restore into a new context, S more."""
    straight = _mixed(eamc)
    straight.set_recursion(0, 40, eamc.EA_REC_BERG)
    _run(straight, 4, 30)
    first = _mixed(eamc)
    first.set_recursion(0, 40, eamc.EA_REC_BERG)
    _run(first, 2, 30)
    blob = first.snapshot()
    resumed = eamc.Context(seed=999)          # the seed comes from the snapshot
    resumed.restore(blob)
    assert resumed.num_chains() == first.num_chains()
    _run(resumed, 2, 30)
    _same(_state(straight), _state(resumed))
    assert np.array_equal(straight.recursion_state(), resumed.recursion_state())
    with pytest.raises(eamc.EamcError):
        resumed.restore(blob)                 # only into a context without chains
    with pytest.raises(eamc.EamcError):
        eamc.Context(seed=1).restore(blob[:100])
