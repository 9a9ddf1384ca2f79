"""Pins of the oracle's round-trip counter (Sec. III of the paper).

A round trip runs from the top of the energy range (E >= E_top, the paper's "E approx 0")
down to the lowest energy E_g and back to the top; the clock starts at the first top visit
and tau_i = (t_last - t_first) / n_rt, in sweeps.  For parallel tempering the paper counts
the same trips per replica between E_g and an energy typical of a temperature well above
freezing.

The counter is pinned three ways, none of which re-types the oracle's state machine:
  * hand-made energy sequences with expected records derived by hand from the definition
    (tests/golden/roundtrip_sequences.txt), fed through the counter alone;
  * real oracle chains (MUCA, per attempt; PT, per replica label and sweep) whose energy
    traces are re-counted by a run-length formulation: the sequence of top / bottom events
    after the first top visit, with runs of equal events merged, alternates T, B, T, ...,
    and every T run after the first completes one round trip at its first element;
  * the requeue flag of the paper (a lower energy than E_g found while counting).
"""
from itertools import groupby
from pathlib import Path

import numpy as np
import pytest

GOLDEN = Path(__file__).resolve().parent / "golden"


def _cases():
    out = []
    for line in (GOLDEN / "roundtrip_sequences.txt").read_text().splitlines():
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, e_top, e_bot, seq, phase, n_rt, t_first, t_last = line.split()
        pairs = [p.split(":") for p in seq.split(",")]
        t = [int(a) for a, _ in pairs]
        E = [int(b) for _, b in pairs]
        out.append((name, int(e_top), int(e_bot), t, E,
                    (int(phase), int(n_rt), int(t_first), int(t_last))))
    return out


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_hand_made_sequences(orc, case):
    _, e_top, e_bot, t, E, want = case
    rt = orc.rt_replay(E, t, e_top, e_bot)
    assert (rt.phase, rt.n_rt, rt.t_first, rt.t_last) == want


def test_replay_continues_a_record(orc):
    """Counting in pieces (a record carried over between calls) equals counting at once."""
    _, e_top, e_bot, t, E, want = [c for c in _cases() if c[0] == "long_gaps"][0]
    rt = orc.rt_replay(E[:3], t[:3], e_top, e_bot)
    rt = orc.rt_replay(E[3:], t[3:], e_top, e_bot, rt=rt)
    assert (rt.phase, rt.n_rt, rt.t_first, rt.t_last) == want


def _runs(E, t, e_top, e_bot):
    """Run-length count of round trips from (E, t) checks with e_bot < e_top: returns
    (phase, n_rt, t_first, t_last)."""
    assert e_bot < e_top
    events = [("T" if e >= e_top else "B", tt) for e, tt in zip(E, t) if e >= e_top or e <= e_bot]
    k = next((i for i, (ev, _) in enumerate(events) if ev == "T"), None)
    if k is None:
        return 0, 0, -1, -1
    runs = [(ev, [tt for _, tt in grp]) for ev, grp in groupby(events[k:], key=lambda x: x[0])]
    t_first = runs[0][1][0]
    later_tops = [times[0] for ev, times in runs[1:] if ev == "T"]
    n_rt = len(later_tops)
    return (2 if runs[-1][0] == "B" else 1), n_rt, t_first, (later_tops[-1] if n_rt else -1)


def _exact_flat_thresholds(orc, dim, L, J):
    """Thresholds of W = 1/g from the enumerated density of states (many round trips)."""
    g = orc.dos_bruteforce(dim, L, J)
    par, nb = orc.parity(dim, L, J), orc.nbonds(dim, L)
    bt = orc.btop(dim, L, par)
    lnO = np.full(bt + 1, -np.inf)
    for b in range(bt + 1):
        u = 2 * b + par
        if g[u] > 0:
            lnO[b] = np.log(float(g[u]))
    reach = np.isfinite(lnO)
    lnW = np.where(reach, -np.where(reach, lnO, 0.0), 50.0)
    lnW -= lnW[bt]
    e_g = orc.energy_of_bin(dim, L, par, int(np.argmax(reach)))
    assert e_g == min(2 * u - nb for u in range(nb + 1) if g[u] > 0)
    return orc.quantize(dim, lnW), e_g


@pytest.mark.parametrize("dim,L,seed,rid", [(2, 4, 21, 1), (3, 3, 5, 2)])
def test_muca_chain_matches_run_length_count(orc, dim, L, seed, rid):
    """Per-attempt checks of a real chain (Sec. III; the oracle checks after every attempt)."""
    J = orc.make_disorder(dim, L, seed, rid)
    thr, e_g = _exact_flat_thresholds(orc, dim, L, J)
    ch = orc.Chain(dim, L, seed, rid, J=J)
    ch.rt.e_g = e_g
    at = ch.sweeps(3000, thr, count_rt=True, attempt_trace=True)
    t = np.repeat(np.arange(3000), ch.V)
    want = _runs(at.ravel(), t, ch.e_top, e_g)
    rt = ch.rt
    assert (rt.phase, rt.n_rt, rt.t_first, rt.t_last) == want
    assert rt.n_rt > 30
    # the same checks through the counter alone give the same record
    rr = orc.rt_replay(at.ravel(), t, ch.e_top, e_g)
    assert (rr.phase, rr.n_rt, rr.t_first, rr.t_last) == want


def test_muca_chain_in_pieces_and_requeue(orc):
    """Counting across calls continues the record; the requeue flag is raised exactly when
    the chain went below E_g while counting (the paper's requeue on a lower energy)."""
    dim, L, seed, rid = 2, 4, 21, 1
    J = orc.make_disorder(dim, L, seed, rid)
    thr, e_g = _exact_flat_thresholds(orc, dim, L, J)
    a = orc.Chain(dim, L, seed, rid, J=J)
    b = orc.Chain(dim, L, seed, rid, J=J)
    a.rt.e_g = b.rt.e_g = e_g
    a.sweeps(900, thr, count_rt=True)
    for n in (1, 299, 600):
        b.sweeps(n, thr, count_rt=True)
    assert a.rt.as_dict() == b.rt.as_dict()
    assert a.rt.requeue == 0                      # nothing lies below the exact ground state
    # E_g set above the true ground state: the chain finds lower energies -> requeue
    c = orc.Chain(dim, L, seed, rid, J=J)
    c.rt.e_g = e_g + 8
    at = c.sweeps(900, thr, count_rt=True, attempt_trace=True)
    assert at.min() < e_g + 8 and c.rt.requeue == 1
    # without counting, no requeue is raised
    d = orc.Chain(dim, L, seed, rid, J=J)
    d.rt.e_g = e_g + 8
    d.sweeps(900, thr, count_rt=False)
    assert d.rt.requeue == 0 and d.rt.n_rt == 0


def test_pt_replicas_match_run_length_count(orc):
    """PT: one check per replica label after each sweep's exchanges, between E_g (bottom) and
    E_hot (top)."""
    dim, L, seed, rid = 2, 4, 8, 3
    betas = [0.2, 0.45, 0.8, 1.3, 2.0]
    J = orc.make_disorder(dim, L, seed, rid)
    g = orc.dos_bruteforce(dim, L, J)
    nb = orc.nbonds(dim, L)
    e_g = min(2 * u - nb for u in range(nb + 1) if g[u] > 0)
    e_hot = -8
    pt = orc.PTRealization(dim, L, seed, rid, betas, J=J)
    pt.sweeps(50)
    t0 = pt.t
    lt = pt.sweeps(4000, count_rt=True, e_g=e_g, e_hot=e_hot, label_trace=True)
    t = np.arange(t0, t0 + 4000)
    total = 0
    for m in range(pt.M):
        want = _runs(lt[:, m], t, e_hot, e_g)
        r = pt.rt[m]
        assert (r.phase, r.n_rt, r.t_first, r.t_last) == want, m
        total += r.n_rt
    assert total > 20
    # labels are a permutation, and the trace's last row is the current energy by label
    assert sorted(pt.label) == list(range(pt.M))
    for k in range(pt.M):
        assert lt[-1, pt.label[k]] == pt.E[k]
