"""Serving loop (a9): continuous batching gives every job the same result alone and in a mix,
admission respects the memory budget, and a short Poisson run completes with latency stats."""
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


def _run_until(server, job, max_ticks=100000):
    for _ in range(max_ticks):
        if job.phase in ("done", "censored"):
            return
        server.tick()
    raise AssertionError("job did not finish")


def test_same_result_alone_and_in_mix(serve):
    probe = _job(serve, 0, 4, 12345, 6)
    alone = serve.Server(seed=21, Ls=(4, 5, 6), base_sweeps=4)
    a = copy.deepcopy(probe)
    alone.submit(a)
    _run_until(alone, a)
    alone.close()

    mix = serve.Server(seed=21, Ls=(4, 5, 6), base_sweeps=4, mem_budget=1 << 30)
    rng = np.random.default_rng(3)
    others = [_job(serve, 100 + k, int(rng.choice([4, 5, 6])), 500 + k, int(rng.integers(2, 20)))
              for k in range(60)]
    for j in others[:40]:
        mix.submit(j)
    for _ in range(7):
        mix.tick()                          # the probe arrives while others are mid-flight
    b = copy.deepcopy(probe)
    mix.submit(b)
    for j in others[40:]:
        mix.submit(j)
    _run_until(mix, b)
    mix.close()
    assert a.phase == b.phase == "done"
    assert a.result == b.result, (a.result, b.result)
    assert a.result["n_rt"] >= 6


def test_memory_budget_admission(serve):
    L = 4
    server = serve.Server(seed=5, Ls=(L,), base_sweeps=4, mem_budget=serve.tile_bytes(3, L))
    jobs = [_job(serve, k, L, 10 + k, 2, iter_steps=1, ticks_per_step=2) for k in range(40)]
    for j in jobs:
        server.submit(j)
    server.tick()
    assert server.lanes[L] == 32                 # one tile fits the budget
    assert len(server.queue) == 8                # the rest wait for a free lane
    for _ in range(20000):
        if all(j.phase in ("done", "censored") for j in jobs):
            break
        server.tick()
    assert all(j.phase in ("done", "censored") for j in jobs)
    assert server.lanes[L] == 32 and server.mem_used <= server.mem_budget
    server.close()


def test_poisson_run_reports_latency(serve):
    jobs = serve.poisson_jobs(200.0, 1.0, (4, 5, 6), 10, 1000, seed=5,
                              iter_steps=2, ticks_per_step=4, max_prod_ticks=50)
    server = serve.Server(seed=5, Ls=(4, 5, 6), base_sweeps=4)
    stats = serve.run_poisson(server, jobs, duration_s=1.0, drain_s=20.0)
    server.close()
    assert stats["jobs"] == len(jobs) > 100
    assert stats["completed"] + stats["censored"] + stats["unfinished"] == stats["jobs"]
    assert stats["completed"] > 0 and stats["p99_s"] >= stats["p50_s"] > 0


def test_cancel_frees_the_lane_for_an_exact_newcomer(serve):
    """Cancelling a queued and a running job; the running job's lane is reused by a job whose
    result equals the one it gets alone (the in-place reset leaves nothing behind)."""
    probe = _job(serve, 0, 5, 777, 5)
    alone = serve.Server(seed=31, Ls=(5,), base_sweeps=4)
    a = copy.deepcopy(probe)
    alone.submit(a)
    _run_until(alone, a)
    alone.close()

    srv = serve.Server(seed=31, Ls=(5,), base_sweeps=4, mem_budget=serve.tile_bytes(3, 5))  # one tile
    jobs = [_job(serve, 10 + k, 5, 900 + k, 10 ** 6) for k in range(34)]    # never finish
    for j in jobs:
        srv.submit(j)
    for _ in range(5):
        srv.tick()
    assert len(srv.active) == 32 and len(srv.queue) == 2      # one tile of lanes, two waiting
    running = next(iter(srv.active.values()))
    lane = running.chain
    assert srv.cancel(jobs[-1].jid) and srv.cancel(running.jid)
    assert not srv.cancel(running.jid) and not srv.cancel(12345)
    srv.tick()                                                # the waiting job takes the lane
    assert jobs[-2].chain == lane and jobs[-2].phase == "iterate"
    assert srv.cancel(jobs[-2].jid)                           # give it back once more
    b = copy.deepcopy(probe)
    srv.submit(b)
    _run_until(srv, b)
    srv.close()
    assert b.chain == lane
    assert {j.jid for j in srv.cancelled} == {jobs[-1].jid, running.jid, jobs[-2].jid}
    assert a.result == b.result, (a.result, b.result)
