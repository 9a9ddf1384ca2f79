"""Parity at the benchmark's full sizes and launch configurations, on sampled chains.

The headline batch (L=8, 1024 power-law chains: Berg weight iteration, E_g fixed, then a
production step with round-trip counting), the L=6 batch (1024 realizations x {flat, power
law} = 2048 chains) and the uneven
batch (4096 realizations of L in {4..12} x {power law, flat, 1/k} = 12288 chains, autotuned
launch, graph-captured iteration loop) are built by the same functions bench.py times; the
oracle then replays chosen chains one by one through the same steps.  Spins, energies, round-
trip records must match exactly, the weights to 1e-12 relative.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eamc():
    import torch
    assert torch.cuda.is_available()
    from paper_2011_08560_gb300 import eamc as m
    m.lib()
    return m


def _close(a, b, rel=1e-12):
    return float(np.max(np.abs(a - b))) <= rel * max(1.0, float(np.max(np.abs(b))))


def _rt_equal(got, rt):
    want = rt.as_dict()
    for f in ("phase", "n_rt", "t_first", "t_last", "e_min", "requeue"):
        assert got[f] == want[f], (f, got[f], want[f])


def _check(ctx, orc, c, ch, lnW):
    S, E, t = ctx.state(c, 1)
    assert np.array_equal(S[0, :ch.V], ch.S) and E[0] == ch.E and t[0] == ch.t
    W = ctx.get_weights(c, 1)[0, :ch.b_top + 1]
    assert _close(W, lnW)
    _rt_equal(ctx.roundtrips(c, 1)[0], ch.rt)


@pytest.mark.parametrize("order", ["colour", "lex"])
def test_headline_full_size_sampled(eamc, orc, order):
    """The headline as bench.py builds and launches it: 1024 power-law chains of L=8 with Berg's
    recursion, a (shortened) iteration phase, E_g fixed and records reset, then one production
    step of 10^4 sweeps with round-trip counting; sampled chains replayed by the oracle.  In the
    headline's sweep order (the checkerboard) and in the lexicographic order."""
    import dataclasses

    import torch

    import bench
    from paper_2011_08560_gb300.workloads import HEADLINE, order_code
    W = dataclasses.replace(HEADLINE, iter_steps=4, iter_sweeps=1000, order=order)
    stream = torch.cuda.Stream()
    ctx = bench.build_context(eamc, 0, stream.cuda_stream, W)
    assert ctx.num_chains() == W.n_real == 1024
    bench.iterate_weights(ctx, W, stream)
    with torch.cuda.stream(stream):
        ctx.run_sweeps(W.sweeps, count_roundtrips=True)
    ctx.synchronize()
    H = ctx.histograms()
    for rid in (0, 511, 1023):
        ch = orc.Chain(W.dim, W.L, W.seed, rid, 0, order=order_code(W.order))
        lnW = np.zeros(ch.b_top + 1)
        acc = orc.berg_state(ch.b_top + 1)
        for _ in range(W.iter_steps):
            ch.sweeps(W.iter_sweeps, orc.quantize(W.dim, lnW))
            lnW = orc.update_weights_berg(W.dim, W.L, ch.parity, orc.POWERLAW, W.alpha, W.pole,
                                          ch.rt.e_min, lnW, ch.hist, acc)
            ch.hist[:] = 0
        # E_g fixed at the lowest energy; the record restarts at the current energy
        ch.rt = orc.RT(phase=0, n_rt=0, t_first=-1, t_last=-1, e_min=ch.E, e_g=ch.rt.e_min,
                       requeue=0, pad=0)
        ch.sweeps(W.sweeps, orc.quantize(W.dim, lnW), count_rt=True)
        _check(ctx, orc, rid, ch, lnW)
        assert np.array_equal(H[rid, :ch.b_top + 1], ch.hist)
    ctx.check()                       # no chain left its energy range on the device
    ctx.close()


def test_l6_full_size_sampled(eamc, orc):
    """Two steps (10^4 sweeps with round-trip counting, then a weight update) of the L=6 batch
    of 2048 chains; chains of both ensembles at both ends of the realization range."""
    import torch

    from paper_2011_08560_gb300.workloads import L6_FLAT_PL as W
    stream = torch.cuda.Stream()
    ctx = eamc.Context(seed=W.seed, device=0, stream=stream.cuda_stream)
    ctx.init_disorder(W.dim, W.L, W.n_real, rid0=0, stream=0)
    ctx.init_disorder(W.dim, W.L, W.n_real, rid0=0, stream=1)
    ctx.set_ensemble(0, W.n_real, eamc.EA_FLAT)
    ctx.set_ensemble(W.n_real, W.n_real, eamc.EA_POWERLAW, W.alpha, W.pole)
    S = W.sweeps
    with torch.cuda.stream(stream):
        for _ in range(2):
            ctx.run_sweeps(S, count_roundtrips=True)
            ctx.update_weights()
    ctx.synchronize()
    n = W.n_real
    for rid, stream_id in ((0, 0), (1023, 0), (0, 1), (517, 1), (1023, 1)):
        kind = orc.POWERLAW if stream_id else orc.FLAT
        ch = orc.Chain(W.dim, W.L, W.seed, rid, stream_id)
        lnW = np.zeros(ch.b_top + 1)
        for _ in range(2):
            ch.sweeps(S, orc.quantize(W.dim, lnW), count_rt=True)
            lnW = orc.update_weights(W.dim, W.L, ch.parity, kind, W.alpha, W.pole, ch.rt.e_min, lnW, ch.hist)
            ch.hist[:] = 0
            ch.rt.e_g = ch.rt.e_min          # the update takes E_g = the lowest energy seen
        _check(ctx, orc, stream_id * n + rid, ch, lnW)
    ctx.check()
    ctx.close()


def test_uneven_full_size_sampled(eamc, orc):
    """The uneven batch with its autotuned launch: one iteration step, 1/k weights for the 1/k
    chains, then a captured graph of two (sweeps + update) iterations replayed once; the first
    and last chain of every (ensemble, L) group."""
    import torch

    import bench
    from paper_2011_08560_gb300 import autotune
    from paper_2011_08560_gb300.workloads import UNEVEN
    S = 20
    stream = torch.cuda.Stream()
    ctx, groups, _ = bench.build_uneven(eamc, autotune, stream.cuda_stream, S)
    ctx.graph_capture(n_iter=2, sweeps_per_iter=S, count_roundtrips=True, update_weights=True)
    ctx.graph_launch(1)
    ctx.synchronize()
    first = 0
    for kind_idx, L, rid0, n in bench.uneven_groups():
        for k in (0, n - 1):
            ch = orc.Chain(3, L, UNEVEN["seed"], rid0 + k, kind_idx)
            kind = orc.POWERLAW if kind_idx == 0 else orc.FLAT
            lnW = np.zeros(ch.b_top + 1)
            ch.sweeps(S, orc.quantize(3, lnW))
            lnW = orc.update_weights(3, L, ch.parity, kind, -3.6, 96.0, ch.rt.e_min, lnW, ch.hist)
            ch.hist[:] = 0
            ch.rt.e_g = ch.rt.e_min
            if kind_idx == 2:
                lnW = orc.build_weights(3, L, ch.parity, orc.ONE_OVER_K, -3.6, 96.0, 1.0, ch.rt.e_g, -lnW)
            for _ in range(2):
                ch.sweeps(S, orc.quantize(3, lnW), count_rt=True)
                if kind_idx != 2:
                    lnW = orc.update_weights(3, L, ch.parity, kind, -3.6, 96.0, ch.rt.e_min, lnW, ch.hist)
                    ch.rt.e_g = ch.rt.e_min
                ch.hist[:] = 0
            _check(ctx, orc, first + k, ch, lnW)
        first += n
    ctx.check()
    ctx.close()
