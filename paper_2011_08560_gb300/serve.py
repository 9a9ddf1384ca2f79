"""Continuous-batching request loop for realization jobs (a9): a thin client of ea_srv_*.

A job is one disorder realization simulated with power-law (or flat) MUCA (Sec. II): a number
of weight-iteration steps, then production until it has completed its target number of round
trips (Sec. III), with the paper's requeue when a lower energy turns up.  The loop itself --
admission into free lanes by memory, one tick after another over all lanes, per-job control
on the device, asynchronous read-back of finished jobs -- runs in the CUDA library
(csrc/serve.cu); this module only marshals jobs and results and drives the clock of a Poisson
arrival process.
"""
from __future__ import annotations

import collections
import ctypes
import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import eamc

LANE = 32


def rows_of(dim: int, L: int) -> int:
    V = L ** dim
    return ((dim * V) // 2 >> 1) + 1


def tile_bytes(dim: int, L: int) -> int:
    """Device bytes one tile of 32 lanes of linear size L takes from the memory budget."""
    return int(eamc.lib().ea_srv_tile_bytes(dim, L))


@dataclass
class Job:
    jid: int
    L: int
    rid: int
    rt_target: int
    arrival: float = 0.0
    stream: int = 0
    kind: int = eamc.EA_POWERLAW
    recursion: int = eamc.EA_REC_BERG
    alpha: float = -3.6
    pole: float = 96.0
    iter_steps: int = 6            # weight-iteration steps before production
    ticks_per_step: int = 8        # ticks per weight-iteration step
    max_prod_ticks: int = 4000     # production cap (the job is then reported as censored)
    max_requeues: int = 4
    # filled in by the server
    server_id: int = 0
    phase: str = "new"             # queued, done, censored, failed, cancelled
    result: dict = field(default_factory=dict)

    def as_c(self) -> eamc.ea_job:
        return eamc.ea_job(L=self.L, rid=self.rid, stream=self.stream, kind=self.kind,
                           recursion=self.recursion, alpha=self.alpha, pole=self.pole,
                           rt_target=self.rt_target, iter_steps=self.iter_steps,
                           ticks_per_step=self.ticks_per_step, max_prod_ticks=self.max_prod_ticks,
                           max_requeues=self.max_requeues, pad=0)


_STATUS = {eamc.EA_JOB_DONE: "done", eamc.EA_JOB_CENSORED: "censored", eamc.EA_JOB_FAILED: "failed"}


class Server:
    """One device, one ea_srv; jobs of any L in `Ls` are served concurrently."""

    def __init__(self, seed: int, Ls=(4, 5, 6, 7, 8, 9, 10, 11, 12), dim: int = 3,
                 mem_budget: int = 2 << 30, base_sweeps: int = 8, poll_ticks: int = 8,
                 max_ahead: int = 64, stream=None, device: int = 0, order: int = 0):
        """order: the sites' order within a sweep for every served chain (eamc.EA_ORDER_LEX or
        eamc.EA_ORDER_COLOUR)."""
        import torch
        self.stream = stream or torch.cuda.Stream(device=device)
        self.dim, self.Ls, self.base_sweeps, self.order = dim, tuple(Ls), base_sweeps, order
        self.mem_budget = mem_budget
        cfg = eamc.ea_srv_config(dim=dim, n_L=len(self.Ls), mem_budget=mem_budget, base_sweeps=base_sweeps,
                                 poll_ticks=poll_ticks, max_ahead=max_ahead, sweep_order=order)
        for k, L in enumerate(self.Ls):
            cfg.Ls[k] = L
        self._h = ctypes.c_void_p()
        eamc.check(eamc.lib().ea_srv_create(ctypes.byref(self._h), device,
                                            ctypes.c_void_p(self.stream.cuda_stream), seed, ctypes.byref(cfg)))
        self.jobs = {}                 # server id -> Job
        self.done = []                 # finished jobs (done, censored, failed) in completion order
        self.cancelled = []
        self._buf = (eamc.ea_srv_result * 4096)()

    def sweeps_per_tick(self, L: int) -> int:
        return self.base_sweeps * max(1, int((max(self.Ls) / L) ** self.dim + 0.5))

    # ---------------------------------------------------------------- jobs
    def submit(self, job: Job) -> int:
        jid = ctypes.c_uint64(0)
        eamc.check(eamc.lib().ea_srv_submit(self._h, ctypes.byref(job.as_c()), ctypes.byref(jid)))
        job.server_id, job.phase = jid.value, "queued"
        self.jobs[jid.value] = job
        return jid.value

    def cancel(self, job: Job) -> bool:
        """Withdraws a waiting or running job; False when it is unknown or already finished."""
        rc = eamc.lib().ea_srv_cancel(self._h, job.server_id)
        if rc == eamc.EA_ESTATE:
            return False
        eamc.check(rc)
        job.phase = "cancelled"
        self.cancelled.append(job)
        self.jobs.pop(job.server_id, None)
        return True

    def step(self, ticks: int = 1):
        eamc.check(eamc.lib().ea_srv_step(self._h, ticks))

    def poll(self, wait: bool = False) -> list:
        """Finished jobs since the last poll (their Job objects, result filled in)."""
        out = []
        while True:
            n = ctypes.c_int(0)
            eamc.check(eamc.lib().ea_srv_poll(self._h, self._buf, len(self._buf), ctypes.byref(n), int(wait)))
            for r in self._buf[:n.value]:
                job = self.jobs.pop(r.job_id, None)
                if job is None:
                    continue
                tau = (r.t_last - r.t_first) / r.n_rt if r.n_rt > 0 else math.inf
                job.phase = _STATUS[r.status]
                job.result = {"n_rt": r.n_rt, "tau_sweeps": tau, "t_first": r.t_first, "t_last": r.t_last,
                              "e_g": r.e_g, "e_min": r.e_min, "sweeps": r.sweeps, "requeues": r.requeues,
                              "t_submit": r.t_submit, "t_admit": r.t_admit, "t_done": r.t_done}
                out.append(job)
            if n.value < len(self._buf):
                break
            wait = False
        self.done.extend(out)
        return out

    def stats(self) -> dict:
        c = eamc.ea_srv_counters()
        eamc.check(eamc.lib().ea_srv_stats(self._h, ctypes.byref(c)))
        return {f: getattr(c, f) for f, _ in eamc.ea_srv_counters._fields_ if f != "pad"}

    def run_until(self, job: Job, max_steps: int = 200000, ticks: int = 8):
        """Steps until `job` has finished (tests)."""
        for _ in range(max_steps):
            if job.phase in ("done", "censored", "failed"):
                return
            self.step(ticks)
            self.poll(wait=True)
        raise AssertionError("job did not finish")

    def close(self):
        if self._h:
            eamc.lib().ea_srv_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def poisson_jobs(rate_hz: float, duration_s: float, Ls, rt_min: int, rt_max: int, seed: int,
                 **job_kw):
    """Seeded Poisson arrivals: uniform L, log-uniform integer round-trip target."""
    rng = np.random.default_rng(seed)
    t, jid, out = 0.0, 0, []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            return out
        L = int(rng.choice(Ls))
        target = int(round(math.exp(rng.uniform(math.log(rt_min), math.log(rt_max)))))
        out.append(Job(jid=jid, L=L, rid=jid, rt_target=target, arrival=t, **job_kw))
        jid += 1


def run_poisson(server: Server, jobs, duration_s: float, drain_s: float, ticks_per_call: int = 4):
    """Feeds jobs at their arrival times for duration_s, then drains for at most drain_s.

    Latency is time to result: from submission to the read-back that reports the job.  A
    censored job counts at its censoring time and a job still unfinished at the end of the drain
    at the end time (both right-censored), so the percentiles cover every job."""
    t0 = time.perf_counter()
    pending = collections.deque(sorted(jobs, key=lambda j: j.arrival))
    submitted_at = {}
    while True:
        now = time.perf_counter() - t0
        while pending and pending[0].arrival <= now:
            j = pending.popleft()
            server.submit(j)
            submitted_at[j.jid] = time.perf_counter() - t0
        if now >= duration_s and not pending:
            break
        if server.jobs:
            server.step(ticks_per_call)
            server.poll()
        else:
            time.sleep(0.0005)
    t_end = time.perf_counter() + drain_s
    while server.jobs and time.perf_counter() < t_end:
        server.step(ticks_per_call)
        server.poll()
    server.poll(wait=True)
    wall = time.perf_counter() - t0
    st = server.stats()
    lat_all, lat_done = [], []
    for j in jobs:
        if j.phase == "done":
            lat = j.result["t_done"] - j.result["t_submit"]
            lat_done.append(lat)
            lat_all.append(lat)
        elif j.phase in ("censored", "failed"):
            lat_all.append(j.result["t_done"] - j.result["t_submit"])
    unfinished = [j for j in jobs if j.phase in ("queued", "new")]
    for j in unfinished:                      # right-censored at the end of the run
        lat_all.append(wall - submitted_at.get(j.jid, j.arrival))
    lat_all, lat_done = np.array(lat_all), np.array(lat_done)
    by_L = {}
    for L in sorted({j.L for j in jobs}):
        js = [j for j in jobs if j.L == L]
        d = [j for j in js if j.phase == "done"]
        by_L[L] = {"jobs": len(js), "done": len(d),
                   "p50_s_done": float(np.percentile([j.result["t_done"] - j.result["t_submit"] for j in d], 50))
                   if d else None}
    return {
        "jobs": len(jobs), "completed": int(sum(j.phase == "done" for j in jobs)),
        "censored": int(sum(j.phase == "censored" for j in jobs)),
        "failed": int(sum(j.phase == "failed" for j in jobs)),
        "unfinished": len(unfinished),
        "p50_s": float(np.percentile(lat_all, 50)) if lat_all.size else None,
        "p99_s": float(np.percentile(lat_all, 99)) if lat_all.size else None,
        "p50_s_completed": float(np.percentile(lat_done, 50)) if lat_done.size else None,
        "p99_s_completed": float(np.percentile(lat_done, 99)) if lat_done.size else None,
        "censored_fraction": float((len(jobs) - len(lat_done)) / max(1, len(jobs))),
        "round_trips_per_s": st["round_trips"] / wall, "wall_s": wall,
        "attempts_per_ns": st["attempts"] / (wall * 1e9), "ticks": st["ticks"],
        "lanes": st["lanes"], "mem_used": st["mem_used"], "by_L": by_L,
    }
