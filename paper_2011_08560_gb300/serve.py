"""Continuous-batching request loop for realization jobs (a9).

A job is one disorder realization to be simulated with power-law MUCA (Sec. II): a fixed
number of weight-iteration steps, then production until it has completed its target number
of round trips (Sec. III), with the paper's requeue when a lower energy turns up (E_g moves
down, the weights take one more iteration step with the new profile, counting restarts).

All state stays on the device in one context: a pool of lanes (tiles of 32 chains) per L.
Every tick is one batched launch over all tiles (small-L tiles get proportionally more
sweeps, so a tick costs about the same for every L); between ticks the loop reaps finished
jobs, frees their lanes, admits waiting jobs into free lanes (resetting a lane in place never
disturbs the other lanes), and grows the pool of an L while the device-memory budget allows
(admission by memory).  Because every random number of a chain is keyed by (realization,
stream, the chain's own sweep count) and a job's schedule is counted in its own ticks, a
job's result does not depend on which other jobs share the device.
"""
from __future__ import annotations

import collections
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
    """Device bytes one tile of 32 chains of linear size L occupies."""
    V = L ** dim
    B = rows_of(dim, L)
    per_lane = B * (8 + 4 + 32)            # ln W (f64), H (u32), thresholds (8 x u32)
    return LANE * per_lane + 4 * (V + dim * V) + LANE * 96


@dataclass
class Job:
    jid: int
    L: int
    rid: int
    rt_target: int
    arrival: float = 0.0
    stream: int = 0
    # schedule, in this job's own ticks
    iter_steps: int = 6            # weight-iteration steps before production
    ticks_per_step: int = 8        # ticks of sweeps per weight-iteration step
    max_prod_ticks: int = 4000     # production cap (the job is then reported as censored)
    max_requeues: int = 4
    # progress
    chain: int = -1
    phase: str = "queued"          # queued, iterate, produce, done, censored
    ticks: int = 0
    steps_done: int = 0
    prod_ticks: int = 0
    requeues: int = 0
    t_admit: float = 0.0
    t_done: float = 0.0
    result: dict = field(default_factory=dict)


class Server:
    """One device, one context; jobs of any L in `Ls` are served concurrently."""

    def __init__(self, seed: int, Ls=(4, 5, 6, 7, 8, 9, 10, 11, 12), dim: int = 3,
                 mem_budget: int = 2 << 30, base_sweeps: int = 8, alpha: float = -3.6,
                 pole: float = 96.0, stream=None, device: int = 0):
        import torch
        self.torch = torch
        self.stream = stream or torch.cuda.Stream(device=device)
        self.ctx = eamc.Context(seed=seed, device=device, stream=self.stream.cuda_stream)
        self.dim, self.Ls, self.alpha, self.pole = dim, tuple(Ls), alpha, pole
        self.mem_budget, self.mem_used = mem_budget, 0
        self.base_sweeps = base_sweeps
        self.lmax = max(self.Ls)
        self.free = {L: collections.deque() for L in self.Ls}
        self.lanes = {L: 0 for L in self.Ls}
        self.queue = collections.deque()
        self.active = {}              # chain -> Job
        self.done = []
        self.cancelled = []
        self.ticks = 0
        self.attempts = 0
        self.n_rt_total = 0
        self._placeholder = 1 << 31   # realization ids of idle lanes

    # ---------------------------------------------------------------- capacity
    def sweeps_per_tick(self, L: int) -> int:
        """Small lattices run more sweeps per tick: about equal attempts per tick for all L."""
        return self.base_sweeps * max(1, round((self.lmax / L) ** self.dim))

    def _grow(self, L: int) -> bool:
        need = tile_bytes(self.dim, L)
        if self.mem_used + need > self.mem_budget:
            return False
        first = self.ctx.init_disorder(self.dim, L, LANE, rid0=self._placeholder, stream=0)
        self._placeholder += LANE
        self.ctx.set_sweep_multiplier(L, self.sweeps_per_tick(L) // self.base_sweeps)
        for c in range(first, first + LANE):
            self.free[L].append(c)
        self.lanes[L] += LANE
        self.mem_used += need
        return True

    # ---------------------------------------------------------------- jobs
    def submit(self, job: Job):
        if job.L not in self.free:
            raise ValueError(f"L={job.L} not served")
        job.phase = "queued"
        self.queue.append(job)

    def cancel(self, jid: int) -> bool:
        """Withdraws a job.  A waiting job leaves the queue; an admitted one gives its lane back
        (the lane's chain keeps sweeping as an idle placeholder until the next admitted job
        resets it in place, which leaves every other lane untouched).  Returns False when the
        job is unknown or already finished."""
        for j in list(self.queue):
            if j.jid == jid:
                self.queue.remove(j)
                j.phase = "cancelled"
                self.cancelled.append(j)
                return True
        for chain, j in list(self.active.items()):
            if j.jid == jid:
                del self.active[chain]
                self.free[j.L].append(chain)
                j.phase = "cancelled"
                self.cancelled.append(j)
                return True
        return False

    def _admit(self, now: float):
        waiting = collections.deque()
        resets = []
        while self.queue:
            job = self.queue.popleft()
            if not self.free[job.L] and not self._grow(job.L):
                waiting.append(job)          # backpressure: no lane and no memory
                continue
            job.chain = self.free[job.L].popleft()
            job.phase, job.t_admit = "iterate", now
            job.ticks = job.steps_done = job.prod_ticks = job.requeues = 0
            resets.append(job)
        self.queue = waiting
        if resets:
            self.ctx.reset_chains([j.chain for j in resets], [j.rid for j in resets],
                                  [j.stream for j in resets])
            for j in resets:
                self.ctx.set_ensemble(j.chain, 1, eamc.EA_POWERLAW, self.alpha, self.pole)
                self.active[j.chain] = j

    def _finish(self, job: Job, rt, now: float, censored: bool):
        n = int(rt["n_rt"])
        tau = int(rt["t_last"] - rt["t_first"]) / n if n > 0 else math.inf
        job.result = {"n_rt": n, "tau_sweeps": tau, "e_g": int(rt["e_g"]), "e_min": int(rt["e_min"]),
                      "sweeps": job.ticks * self.sweeps_per_tick(job.L), "requeues": job.requeues}
        job.phase = "censored" if censored else "done"
        job.t_done = now
        self.n_rt_total += n
        del self.active[job.chain]
        self.free[job.L].append(job.chain)
        self.done.append(job)

    def tick(self, now: float | None = None):
        now = time.perf_counter() if now is None else now
        self._admit(now)
        if not self.active:
            return
        with self.torch.cuda.stream(self.stream):
            self.ctx.run_sweeps(self.base_sweeps, count_roundtrips=True)
        self.ticks += 1
        for L in self.Ls:
            self.attempts += self.lanes[L] * self.sweeps_per_tick(L) * L ** self.dim
        jobs = list(self.active.values())
        for j in jobs:
            j.ticks += 1
        # weight-iteration steps of the jobs that reached a step boundary
        step = [j for j in jobs if j.phase == "iterate" and j.ticks % j.ticks_per_step == 0]
        if step:
            self.ctx.update_weights_subset([j.chain for j in step])
            for j in step:
                j.steps_done += 1
                if j.steps_done >= j.iter_steps:
                    j.phase = "produce"
                    self.ctx.set_eg(j.chain, 1, None)           # E_g = lowest energy seen
                    self.ctx.roundtrips(j.chain, 1, reset=True)
        prod = [j for j in jobs if j.phase == "produce"]
        if not prod:
            return
        rts = self.ctx.roundtrips_array()
        done_now = time.perf_counter()
        for j in prod:
            j.prod_ticks += 1
            rt = rts[j.chain]
            if rt["requeue"] and j.requeues < j.max_requeues:
                # a lower energy: new E_g, one more weight step with the new profile, restart
                j.requeues += 1
                self.ctx.set_eg(j.chain, 1, None)
                self.ctx.update_weights_subset([j.chain])
                self.ctx.roundtrips(j.chain, 1, reset=True)
                j.prod_ticks = 0
            elif rt["n_rt"] >= j.rt_target:
                self._finish(j, rt, done_now, censored=False)
            elif j.prod_ticks >= j.max_prod_ticks:
                self._finish(j, rt, done_now, censored=True)

    def drain(self, deadline: float):
        while (self.active or self.queue) and time.perf_counter() < deadline:
            self.tick()

    def close(self):
        self.ctx.close()


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


def run_poisson(server: Server, jobs, duration_s: float, drain_s: float):
    """Feeds jobs at their arrival times, then drains; returns latency / throughput stats."""
    t0 = time.perf_counter()
    pending = collections.deque(sorted(jobs, key=lambda j: j.arrival))
    while True:
        now = time.perf_counter() - t0
        while pending and pending[0].arrival <= now:
            j = pending.popleft()
            j.arrival += t0
            server.submit(j)
        if now >= duration_s and not pending:
            break
        if server.active or server.queue:
            server.tick()
        else:
            time.sleep(0.0005)
    server.drain(time.perf_counter() + drain_s)
    wall = time.perf_counter() - t0
    lat = np.array([j.t_done - j.arrival for j in server.done if j.phase == "done"])
    return {
        "jobs": len(jobs), "completed": int((np.array([j.phase for j in server.done]) == "done").sum()),
        "censored": sum(j.phase == "censored" for j in server.done),
        "unfinished": len(server.active) + len(server.queue),
        "p50_s": float(np.percentile(lat, 50)) if lat.size else None,
        "p99_s": float(np.percentile(lat, 99)) if lat.size else None,
        "round_trips_per_s": server.n_rt_total / wall, "wall_s": wall,
        "attempts_per_ns": server.attempts / (wall * 1e9), "ticks": server.ticks,
        "lanes": dict(server.lanes), "mem_used": server.mem_used,
    }
