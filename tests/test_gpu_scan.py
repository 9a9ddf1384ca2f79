"""Profile-parameter scan (power-law alpha, Delta E) and the weight copy it relies on, against
the oracle run through the same stages: density of states from a flat chain with Berg's
recursion, the ensembles built from it, production with round-trip counting."""
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


def test_copy_weights(eamc):
    ctx = eamc.Context(seed=3)
    ctx.init_disorder(3, 4, 4, rid0=10, stream=0)
    ctx.init_disorder(3, 4, 4, rid0=10, stream=1)
    ctx.init_disorder(3, 5, 2, rid0=10, stream=2)
    ctx.set_ensemble(0, 4, eamc.EA_POWERLAW, -2.5, 50.0)
    ctx.run_sweeps(50)
    ctx.update_weights()
    ctx.set_eg(0, 4, None)
    ctx.copy_weights([0, 1, 2, 3], [4, 5, 6, 7])
    W, T = ctx.get_weights(), ctx.get_thresholds()
    D, R = ctx.describe(), ctx.roundtrips()
    for a, b in zip(range(4), range(4, 8)):
        assert np.array_equal(W[a], W[b]) and np.array_equal(T[a], T[b])
        assert D[b]["kind"] == eamc.EA_POWERLAW and R[b]["e_g"] == R[a]["e_g"]
    with pytest.raises(eamc.EamcError):
        ctx.copy_weights([0], [8])          # other L
    with pytest.raises(eamc.EamcError):
        ctx.copy_weights([0, 1], [4, 4])    # a destination twice
    with pytest.raises(eamc.EamcError):
        ctx.copy_weights([0, 4], [4, 5])    # 4 is source and destination


@pytest.mark.parametrize("order", [0, 1])
def test_profile_scan_matches_oracle(eamc, orc, order):
    """In both sweep orders (order 1: the checkerboard kernel at L = 4)."""
    from paper_2011_08560_gb300 import scan
    dim, L, n, seed = 3, 4, 5, 13
    iters, S, P = 6, 400, 2500
    res = scan.profile_scan(dim, L, n, (-3.6, -2.0), (96.0, 30.0), seed=seed, dos_iters=iters,
                            dos_sweeps=S, prod_sweeps=P, recursion=eamc.EA_REC_BERG, order=order)
    assert res.labels[0] == "flat" and res.labels[-1] == "1/k" and len(res.labels) == 6
    for r in range(n):
        dos = orc.Chain(dim, L, seed, r, 0, order=order)
        lnW = np.zeros(dos.b_top + 1)
        acc = orc.berg_state(dos.b_top + 1)
        for _ in range(iters):
            dos.hist[:] = 0
            dos.sweeps(S, orc.quantize(dim, lnW))
            lnW = orc.update_weights_berg(dim, L, dos.parity, 1, -3.6, 96.0, dos.rt.e_min, lnW,
                                          dos.hist, acc)
        e_g = int(dos.rt.e_min)
        assert res.e_g[r] == e_g
        lnP = np.array([orc.ln_profile(1, -3.6, 96.0, e_g, orc.energy_of_bin(dim, L, dos.parity, b))
                        for b in range(dos.b_top + 1)])
        lnO = lnP - lnW
        for k, (kind, a, p) in enumerate(res.params):
            ch = orc.Chain(dim, L, seed, r, stream=1 + k, order=order)
            if kind != 1:
                a, p = -3.6, 96.0
            w = orc.build_weights(dim, L, ch.parity, kind, a, p, 1.0, e_g, lnO)
            ch.rt = orc.RT(phase=0, n_rt=0, t_first=-1, t_last=-1, e_min=ch.E, e_g=e_g, requeue=0, pad=0)
            ch.sweeps(P, orc.quantize(dim, w), count_rt=True)
            assert res.n_rt[k, r] == ch.rt.n_rt, (k, r)
            assert bool(res.requeue[k, r]) == bool(ch.rt.requeue), (k, r)
            if ch.rt.n_rt:
                assert res.tau[k, r] == (ch.rt.t_last - ch.rt.t_first) / ch.rt.n_rt
    rows = res.summary()
    assert rows[0]["ensemble"] == "flat" and "tau_over_flat" not in rows[0]


def test_pt_arm_matches_oracle(eamc, orc):
    """The scan's PT arm (adapted temperatures, E_hot from the hottest slot, round trips between
    E_g and E_hot per replica, replicas pooled per realization) against the oracle run through
    the same steps, on sampled realizations of one 32-realization group."""
    from paper_2011_08560_gb300 import scan
    from paper_2011_08560_gb300.workloads import geometric_betas
    dim, L, n, M, seed = 3, 4, 32, 4, 17
    windows, window, prod = 2, 100, 600
    e_g = np.array([-76 + 4 * (r % 3) for r in range(n)], dtype=np.int32)
    tau, below = scan.pt_round_trips(dim, L, n, M, e_g, seed=seed, windows=windows, window=window,
                                     prod_sweeps=prod)
    for r in (0, 13, 31):
        p = orc.PTRealization(dim, L, seed, r, geometric_betas(M, 0.3, 2.15))
        hot = []
        for _ in range(windows):
            for _ in range(10):
                p.sweeps(window // 10)
                hot.append(int(p.E[0]))
            p.adapt(0.5)
        e_hot = int(np.floor(np.mean(hot)))
        for k in range(M):
            p.rt[p.label[k]] = orc.RT(phase=0, n_rt=0, t_first=-1, t_last=-1, e_min=int(p.E[k]),
                                      e_g=0, requeue=0, pad=0)
        p.sweeps(prod, count_rt=True, e_g=int(e_g[r]), e_hot=e_hot)
        n_rt = sum(p.rt[m].n_rt for m in range(M))
        span = sum(p.rt[m].t_last - p.rt[m].t_first for m in range(M) if p.rt[m].n_rt > 0)
        want = span / n_rt if n_rt else np.inf
        assert tau[r] == want, (r, tau[r], want)
        assert bool(below[r]) == (min(p.rt[m].e_min for m in range(M)) < e_g[r])
    assert np.isfinite(tau).sum() > 0
