"""Serving loop (a9, ea_srv_*): a job gives the same result alone and among other jobs, the
result equals the oracle's replay of the job's schedule (reset lane, weight steps, E_g fixed,
production, requeue), admission respects the memory budget, cancellation frees lanes for exact
newcomers, and a short Poisson run accounts for every job."""
import copy

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def serve():
    import torch
    assert torch.cuda.is_available()
    from paper_2011_08560_gb300 import serve as s
    return s


def _job(serve, jid, L, rid, target, **kw):
    kw.setdefault("iter_steps", 3)
    kw.setdefault("ticks_per_step", 4)
    kw.setdefault("max_prod_ticks", 3000)
    return serve.Job(jid=jid, L=L, rid=rid, rt_target=target, **kw)


RESULT_KEYS = ("n_rt", "t_first", "t_last", "e_g", "e_min", "sweeps", "requeues")


def _same(a, b):
    return a.phase == b.phase and all(a.result[k] == b.result[k] for k in RESULT_KEYS)


def test_same_result_alone_and_in_mix(serve):
    probe = _job(serve, 0, 4, 12345, 6)
    alone = serve.Server(seed=21, Ls=(4, 5, 6), base_sweeps=4)
    a = copy.deepcopy(probe)
    alone.submit(a)
    alone.run_until(a)
    alone.close()

    mix = serve.Server(seed=21, Ls=(4, 5, 6), base_sweeps=4, mem_budget=1 << 30)
    rng = np.random.default_rng(3)
    others = [_job(serve, 100 + k, int(rng.choice([4, 5, 6])), 500 + k, int(rng.integers(2, 20)))
              for k in range(60)]
    for j in others[:40]:
        mix.submit(j)
    mix.step(7)                           # the probe arrives while others are mid-flight
    b = copy.deepcopy(probe)
    mix.submit(b)
    for j in others[40:]:
        mix.submit(j)
    mix.run_until(b)
    mix.close()
    assert a.phase == b.phase == "done"
    assert _same(a, b), (a.result, b.result)
    assert a.result["n_rt"] >= 6


def _oracle_replay(orc, seed, job, spt, order=0):
    """The job's schedule in the oracle, tick by tick (the device's job control)."""
    ch = orc.Chain(3, job.L, seed, job.rid, job.stream, order=order)
    lnW = np.zeros(ch.b_top + 1)
    acc = orc.berg_state(ch.b_top + 1)
    kind = orc.POWERLAW if job.kind == 1 else orc.FLAT

    def step():
        nonlocal lnW
        if job.recursion == 1:
            lnW = orc.update_weights_berg(3, job.L, ch.parity, kind, job.alpha, job.pole, ch.rt.e_min,
                                          lnW, ch.hist, acc)
        else:
            lnW = orc.update_weights(3, job.L, ch.parity, kind, job.alpha, job.pole, ch.rt.e_min, lnW, ch.hist)
        ch.hist[:] = 0
        ch.rt.e_g = ch.rt.e_min

    def restart():
        ch.rt = orc.RT(phase=0, n_rt=0, t_first=-1, t_last=-1, e_min=ch.E, e_g=ch.rt.e_g, requeue=0, pad=0)

    ticks = steps = prod = requeues = 0
    phase = "iterate"
    while True:
        ch.sweeps(spt, orc.quantize(3, lnW), count_rt=True)
        ticks += 1
        if phase == "iterate":
            if ticks % job.ticks_per_step == 0:
                step()
                steps += 1
                if steps >= job.iter_steps:
                    restart()
                    phase, prod = "produce", 0
            continue
        prod += 1
        if ch.rt.requeue and requeues < job.max_requeues:
            step()
            restart()
            requeues += 1
            prod = 0
        elif ch.rt.n_rt >= job.rt_target:
            status = "done"
            break
        elif prod >= job.max_prod_ticks:
            status = "censored"
            break
    return status, {"n_rt": ch.rt.n_rt, "t_first": ch.rt.t_first, "t_last": ch.rt.t_last, "e_g": ch.rt.e_g,
                    "e_min": ch.rt.e_min, "sweeps": ch.t, "requeues": requeues}


@pytest.mark.parametrize("L,recursion,target,order", [(4, 1, 5, 0), (5, 0, 4, 0), (6, 1, 3, 0),
                                                     (4, 1, 5, 1), (5, 0, 4, 1), (6, 1, 3, 1)])
def test_served_job_matches_oracle_replay(serve, orc, L, recursion, target, order):
    """Power-law jobs whose weight steps leave E_g above the ground state, so that production
    finds lower energies and requeues (new E_g, one more step, counting restarts); served in
    the lexicographic and in the colour order (even and odd L)."""
    srv = serve.Server(seed=41, Ls=(4, 5, 6), base_sweeps=2, order=order)
    jobs = [_job(serve, k, L, 300 + k, target, recursion=recursion, iter_steps=1, ticks_per_step=2,
                 max_prod_ticks=4000, max_requeues=3) for k in range(6)]
    for j in jobs:
        srv.submit(j)
    for j in jobs:
        srv.run_until(j)
    spt = srv.sweeps_per_tick(L)
    srv.close()
    requeued = 0
    for j in jobs:
        status, want = _oracle_replay(orc, 41, j, spt, order)
        assert j.phase == status, (j.jid, j.phase, status)
        for k in RESULT_KEYS:
            assert j.result[k] == want[k], (j.jid, k, j.result[k], want[k])
        requeued += want["requeues"] > 0
    assert requeued > 0                      # the requeue path was exercised


def test_memory_budget_admission(serve):
    L = 4
    server = serve.Server(seed=5, Ls=(L,), base_sweeps=4, mem_budget=serve.tile_bytes(3, L))
    jobs = [_job(serve, k, L, 10 + k, 2, iter_steps=1, ticks_per_step=2) for k in range(40)]
    for j in jobs:
        server.submit(j)
    server.step(1)
    st = server.stats()
    assert st["lanes"] == 32                 # one tile fits the budget
    assert st["queued"] == 8 and st["running"] == 32   # the rest wait for a free lane
    for _ in range(20000):
        if all(j.phase in ("done", "censored") for j in jobs):
            break
        server.step(4)
        server.poll()
    server.poll(wait=True)
    assert all(j.phase in ("done", "censored") for j in jobs)
    st = server.stats()
    assert st["lanes"] == 32 and st["mem_used"] <= server.mem_budget
    assert st["done"] + st["censored"] == 40
    server.close()


def test_cancel_frees_the_lane_for_an_exact_newcomer(serve):
    """Cancelling a queued and a running job; the freed lane is reused by a job whose result
    equals the one it gets alone (the in-place reset leaves nothing behind)."""
    probe = _job(serve, 0, 5, 777, 5)
    alone = serve.Server(seed=31, Ls=(5,), base_sweeps=4)
    a = copy.deepcopy(probe)
    alone.submit(a)
    alone.run_until(a)
    alone.close()

    srv = serve.Server(seed=31, Ls=(5,), base_sweeps=4, mem_budget=serve.tile_bytes(3, 5))  # one tile
    jobs = [_job(serve, 10 + k, 5, 900 + k, 10 ** 6) for k in range(34)]    # never finish
    for j in jobs:
        srv.submit(j)
    srv.step(5)
    st = srv.stats()
    assert st["running"] == 32 and st["queued"] == 2       # one tile of lanes, two waiting
    assert srv.cancel(jobs[-1]) and srv.cancel(jobs[0])    # a queued and a running job
    assert not srv.cancel(jobs[0])
    srv.step(1)                                              # the waiting job takes the lane
    st = srv.stats()
    assert st["running"] == 32 and st["queued"] == 0 and st["cancelled"] == 2
    assert srv.cancel(jobs[-2])                              # give it back once more
    b = copy.deepcopy(probe)
    srv.submit(b)
    srv.run_until(b)
    assert srv.stats()["lanes"] == 32
    srv.close()
    assert _same(a, b), (a.result, b.result)


def test_submit_rejects_bad_jobs(serve):
    from paper_2011_08560_gb300 import eamc
    srv = serve.Server(seed=1, Ls=(4,), base_sweeps=4)
    for bad in (dict(L=5), dict(kind=eamc.EA_ONE_OVER_K), dict(rt_target=0), dict(recursion=7),
                dict(max_prod_ticks=10 ** 9, max_requeues=10 ** 6)):
        kw = dict(L=4)
        kw.update(bad)
        L = kw.pop("L")
        with pytest.raises(eamc.EamcError):
            srv.submit(_job(serve, 0, L, 1, kw.pop("rt_target", 3), **kw))
    srv.close()


def test_poisson_run_reports_latency(serve):
    jobs = serve.poisson_jobs(200.0, 1.0, (4, 5, 6), 10, 1000, seed=5,
                              iter_steps=2, ticks_per_step=4, max_prod_ticks=50)
    server = serve.Server(seed=5, Ls=(4, 5, 6), base_sweeps=4)
    stats = serve.run_poisson(server, jobs, duration_s=1.0, drain_s=20.0)
    server.close()
    assert stats["jobs"] == len(jobs) > 100
    assert stats["completed"] + stats["censored"] + stats["failed"] + stats["unfinished"] == stats["jobs"]
    assert stats["completed"] > 0 and stats["p99_s"] >= stats["p50_s"] > 0
    assert stats["attempts_per_ns"] > 0
