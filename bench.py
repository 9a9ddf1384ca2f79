"""Benchmark: batched power-law MUCA on the 3D +-J EA spin glass, one JSON line.

Headline workload: L=8, 1024 disorder realizations, each a power-law MUCA chain (alpha=-3.6,
Delta E=96, Sec. II) packed into multi-spin-coded tiles.  Before timing, the weights iterate
with Berg's accumulated recursion (the iteration phase, timed and reported on its own); then
E_g is fixed at each chain's lowest energy, the round-trip records are reset and the weights
are frozen (Sec. III: round trips are measured with weights determined beforehand).  One step
= one production pass over the batch: `sweeps_per_step` sweeps of generalized Metropolis with
histogram, lowest-energy and round-trip measurement (muca_run_sweeps).  Metric: spin-flip
attempts per ns (whole job), with round trips per second and the mean round-trip time in
sweeps beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the CPU oracle (plain C, one chain at a time, all host cores) on a
bounded sample of the same workload.  Under torchrun every rank runs its own 1024
realizations (disjoint realization ids, no data-path collective): weak scaling.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

from paper_2011_08560_gb300.workloads import HEADLINE, L6_FLAT_PL, SMALL, order_code  # noqa: E402

METRIC = "spin-flip attempts/ns (L=8, power-law ensemble)"
UNIT = "attempts/ns"
# algorithmic integer lane-operations per spin-flip attempt, the count of the hot-path scope:
# 20 (a quarter of a Philox4x32-10 call: 10 rounds of two 32x32->64 products, the xors and the
# key bumps, about 80 operations for four words) + 10 for the rest (bit-sliced local field of
# 32 chains per word with extraction 3.5, threshold fetch and compare 3, flip and energy update
# 2, lowest energy and round-trip check 1.5); the midpoint of the scope's 25-35
ALG_OPS_PER_ATTEMPT = 30.0
# per-chain latency floor of one MUCA attempt in SM cycles: the next attempt's threshold is a
# shared-memory load whose address depends on the current decision (the bin moves only if the
# attempt is accepted), loaded for both outcomes one attempt ahead and selected.  That minimal
# dependent pattern (select the address, load, select the threshold, compare), timed alone in one
# warp with clock64 over 4096 steps on the GB300, takes 35.4 cycles per step (a chain of
# dependent shared-memory loads: 34.0; compare -> select: 8.6; the same loads at independent
# addresses pipeline at 9.2): the load's latency is not hidden once its address depends on the
# decision it feeds, also with the loads issued two attempts ahead (32.4)
LATENCY_FLOOR_CYCLES = 35.4
# PT, per site word of 32 lattices (32 attempts): 12 word loads + 14 bit ops for the
# unsatisfied counts + 4 for the classes, about 8 compared bit planes (2 Philox4x32-10 calls of
# 40 ops, 5 ops per plane) and the flip: about 150 lane-operations per 32 attempts
PT_ALG_OPS = 4.7
# dram__bytes_read.sum + dram__bytes_write.sum of one production launch of the headline workload
# (L=8, 1024 chains in tiles of 8, checkerboard kernel), ncu capture of this kernel version:
# 14.20 MB + 0 B for a 2000-sweep launch.  It is the one-time staging of the threshold tables and
# lattices, so it does not grow with the sweeps of a launch: a 10^4-sweep launch moves the same
# bytes.
SWEEP_TRAFFIC_BYTES = 14.20e6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--sweeps-per-step", type=int, default=10_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the PT / uneven / serving lines")
    ap.add_argument("--only", choices=["pt", "pt_protocol", "uneven", "serving", "serving_saturated",
                                       "recursion", "scan", "small", "flat", "l6", "table_one_l8",
                                       "paper_samples", "lex", "uneven_checkerboard",
                                       "table_one_l8_checkerboard", "scan_checkerboard", "serving_colour",
                                       "serving_lex"],
                    default=None,
                    help="run one secondary workload alone and print its record (profiling)")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the autotuner: narrow tiles where available, one launch per call "
                         "(a fixed launch sequence, for profiling)")
    ap.add_argument("--order", choices=["lex", "colour"], default=None,
                    help="sweep order of the headline chains (default: the workload's, colour)")
    ap.add_argument("--iter-steps", type=int, default=None,
                    help="weight-iteration steps before timing (default: the workload's)")
    ap.add_argument("--iter-sweeps", type=int, default=None,
                    help="sweeps per weight-iteration step (default: the workload's)")
    ap.add_argument("--pt-sweeps", type=int, default=100_000,
                    help="timed PT sweeps with round-trip counting (the workload names 10^6)")
    ap.add_argument("--scan-L", type=int, default=6, help="lattice size of the profile scan")
    ap.add_argument("--scan-prod-sweeps", type=int, default=100_000,
                    help="production sweeps of the profile scan")
    return ap.parse_args()


# ------------------------------------------------------------------------------ oracle (CPU)
def _oracle_worker(args):
    """One headline chain in the oracle: two short plain iteration steps (untimed) give it
    power-law-shaped weights, then `sweeps` production sweeps with frozen weights and
    round-trip counting are timed."""
    import numpy as np

    import oracle
    dim, L, seed, rid, stream, kind, sweeps, order = args
    c = oracle.Chain(dim, L, seed, rid, stream, order=order)
    lnW = np.zeros(c.b_top + 1)
    for _ in range(2):
        c.sweeps(200, oracle.quantize(dim, lnW))
        lnW = oracle.update_weights(dim, L, c.parity, kind, HEADLINE.alpha, HEADLINE.pole,
                                    c.rt.e_min, lnW, c.hist)
        c.hist[:] = 0
    c.rt.e_g = c.rt.e_min
    thr = oracle.quantize(dim, lnW)
    t0 = time.perf_counter()
    c.sweeps(sweeps, thr, count_rt=True)
    dt = time.perf_counter() - t0
    return c.V * sweeps, dt, c.rt.n_rt


def oracle_sample(target_s: float = 15.0, cores: int | None = None, W=HEADLINE):
    """Times the oracle on all host cores on a bounded sample of the headline workload (in the
    workload's sweep order)."""
    import oracle
    oracle.build()
    cores = cores or os.cpu_count() or 1
    order = order_code(W.order)
    # calibrate one chain
    calib = _oracle_worker((W.dim, W.L, W.seed, 0, 0, 1, 50, order))
    per_sweep = calib[1] / 50
    chains = 2 * cores
    sweeps = max(20, int(target_s * cores / (chains * per_sweep)))
    jobs = [(W.dim, W.L, W.seed, k, 0, 1, sweeps, order) for k in range(chains)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_worker, jobs)
    # the timed production sweeps of all chains, run side by side on `cores` processes
    busy = sum(r[1] for r in res)
    wall = busy / min(cores, chains) if chains else 0.0
    attempts = sum(r[0] for r in res)
    return {"value": attempts / (wall * 1e9), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{chains} power-law chains of L={W.L} (realizations 0..{chains - 1}), "
                      f"{sweeps} production sweeps each with frozen weights and round-trip counting, "
                      f"sites in the {'colour (checkerboard)' if order else 'lexicographic'} order, "
                      f"{busy:.1f} s of CPU time on {cores} processes",
            "round_trips": sum(r[2] for r in res), "wall_s": wall}


# ------------------------------------------------------------------------------ clocks
class ClockSampler:
    def __init__(self, device: int):
        self.device = device
        self.proc = None
        # the samples are kept in EAMC_CLOCKS_DIR when it is set, else in the temp directory
        base = os.environ.get("EAMC_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = Path(base) / f"clocks_{os.getpid()}.csv"

    def __enter__(self):
        self.path.parent.mkdir(exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            self.proc.wait(timeout=5)
            self.f.close()

    def summary(self):
        if not self.proc or not self.path.exists():
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.path.read_text().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------ GPU arm
def shard_rid0(rank: int, n_per_rank: int) -> int:
    """Realizations of a rank: ids rank*n .. rank*n + n - 1 (disjoint; no data-path exchange)."""
    return rank * n_per_rank


def reduce_max_ms(t_ms: float, world: int, device=None) -> float:
    """The job's time is the slowest rank's (max over ranks of the timed interval)."""
    if world <= 1:
        return t_ms
    import torch
    t = torch.tensor([t_ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def headline(args):
    """The headline workload, with the iteration schedule overridden from the command line."""
    import dataclasses
    kw = {}
    if args.iter_steps is not None:
        kw["iter_steps"] = args.iter_steps
    if args.iter_sweeps is not None:
        kw["iter_sweeps"] = args.iter_sweeps
    if getattr(args, "order", None) is not None:
        kw["order"] = args.order
    return dataclasses.replace(HEADLINE, **kw)


def build_context(eamc, rank: int, stream_ptr: int, W=HEADLINE, ensembles=None, tuned=True):
    """The chains of workload W (one per realization and ensemble, stream = ensemble index),
    with W's weight recursion and the autotuned tile width and launch (tuned=False: narrow tiles
    where available, one launch per call); realizations of this rank only."""
    from paper_2011_08560_gb300 import autotune
    ens_list = ensembles or W.ensembles
    n = W.n_real
    if tuned:
        best = autotune.tune([(W.dim, W.L, n)] * len(ens_list), order=order_code(W.order))
    else:
        best = {"widths": {str(W.L): eamc.narrow_width(W.dim, W.L, order_code(W.order))}, "persistent": False,
                "blocks_per_sm": 0, "sweeps_per_launch": 0}
    ctx = eamc.Context(seed=W.seed, device=0, stream=stream_ptr)
    ctx.set_sweep_order(order_code(W.order))
    if best:
        autotune.prepare(ctx, best)
    rid0 = shard_rid0(rank, n)
    for s, ens in enumerate(ens_list):
        first = ctx.init_disorder(W.dim, W.L, n, rid0=rid0, stream=s)
        kind = eamc.EA_POWERLAW if ens == "powerlaw" else eamc.EA_FLAT
        ctx.set_ensemble(first, n, kind, W.alpha, W.pole)
        if W.recursion == "berg":
            ctx.set_recursion(first, n, eamc.EA_REC_BERG)
    if best:
        autotune.launch(ctx, best)
        ctx.tuned = best
    return ctx


def iterate_weights(ctx, W, stream):
    """The iteration phase (Sec. II): W.iter_steps x (W.iter_sweeps sweeps, then one weight
    update); then E_g = each chain's lowest energy, and histograms and round-trip records start
    afresh for production.  Returns (device ms of the sweeps, device ms of the updates)."""
    import torch
    sw, up = [], []
    for _ in range(W.iter_steps):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        ctx.run_sweeps(W.iter_sweeps)
        e1.record(stream)
        ctx.update_weights()
        e2.record(stream)
        sw.append((e0, e1))
        up.append((e1, e2))
    stream.synchronize()
    ctx.set_eg(0, ctx.num_chains(), None)
    ctx.roundtrips(reset=True)
    ctx.histograms(reset=True)
    return sum(a.elapsed_time(b) for a, b in sw), sum(a.elapsed_time(b) for a, b in up)


def total_rt(ctx):
    return sum(r["n_rt"] for r in ctx.roundtrips())


def tau_stats(records):
    """Sec. III: tau_i = (t_last - t_first) / n_rt per chain with a round trip, in sweeps."""
    taus = [(r["t_last"] - r["t_first"]) / r["n_rt"] for r in records if r["n_rt"] > 0]
    return {"mean": statistics.mean(taus) if taus else None,
            "median": statistics.median(taus) if taus else None,
            "chains_with_round_trip": len(taus), "chains": len(records),
            "round_trips": sum(r["n_rt"] for r in records),
            "requeued": sum(1 for r in records if r["requeue"])}


def run_gpu(args, rank, world):
    import numpy as np
    import torch

    from paper_2011_08560_gb300 import eamc

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    W = headline(args)
    S = args.sweeps_per_step
    stream = torch.cuda.Stream()
    ctx = build_context(eamc, rank, stream.cuda_stream, W, tuned=not args.no_tune)
    n_chains = ctx.num_chains()
    V = W.L ** W.dim
    attempts_per_step = n_chains * V * S
    iter_sweep_ms, iter_update_ms = iterate_weights(ctx, W, stream)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            ctx.run_sweeps(S, count_roundtrips=True)
    stream.synchronize()
    rt0 = total_rt(ctx)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    with ClockSampler(int(os.environ.get("LOCAL_RANK", 0))) as clk:
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(k))                       # evict L2 between steps
                starts[k].record(stream)
                ctx.run_sweeps(S, count_roundtrips=True)    # one launch of the sweep kernel
                ends[k].record(stream)
        stream.synchronize()
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    t_ms = sum(step_ms)
    if world > 1:
        t_ms = reduce_max_ms(t_ms, world, device="cuda")
        torch.distributed.barrier()
    rts = total_rt(ctx) - rt0
    try:
        ctx.check()                       # device-side invariants held during the timed steps
        invariants = "ok"
    except eamc.EamcError as err:
        invariants = str(err)
    taus = tau_stats(ctx.roundtrips())
    value = world * attempts_per_step * args.steps / (t_ms * 1e6)
    kern_avg_s = statistics.mean(step_ms) / 1e3
    achieved_ops = attempts_per_step * ALG_OPS_PER_ATTEMPT / kern_avg_s
    props = torch.cuda.get_device_properties(0)
    peaks = json.loads((ROOT / "MEASURED_PEAKS.json").read_text()) if (ROOT / "MEASURED_PEAKS.json").exists() else {}
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = props.multi_processor_count * 4 * 32 * sm_max * 1e6   # lane-instr/s issue limit

    # end to end through the C ABI with host buffers in pinned memory: the frozen weights in,
    # histograms and round-trip records out, every step
    from paper_2011_08560_gb300.eamc import RT_DTYPE
    rows = max(d["b_top"] for d in ctx.describe()) + 1

    def pinned(shape, dtype):
        nbytes = int(np.prod(shape)) * np.dtype(dtype).itemsize
        return torch.empty(nbytes, dtype=torch.uint8, pin_memory=True).numpy().view(dtype).reshape(shape)

    lnW_host = pinned((n_chains, rows), np.float64)
    hist = pinned((n_chains, rows), np.uint32)
    rt = pinned((n_chains,), RT_DTYPE)
    ctx.get_weights(rows=rows, out=lnW_host)
    e2e_ms = []
    for k in range(max(2, min(args.steps, 5))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            ctx.set_weights(0, lnW_host)
            ctx.run_sweeps(S, count_roundtrips=True)
            ctx.histograms(rows=rows, out=hist)
            ctx.roundtrips_array(out=rt)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    h2d = lnW_host.nbytes
    d2h = hist.nbytes + rt.nbytes
    ctx.close()

    plain = None
    if not args.no_plain and rank == 0:
        plain = plain_form(eamc, stream, S=200)

    return {
        "value": value, "t_ms": t_ms, "step_ms": step_ms, "wall": wall,
        "rts": rts, "attempts_per_step": attempts_per_step, "n_chains": n_chains,
        "achieved_ops": achieved_ops, "alu_peak": alu_peak, "clocks": clk.summary(),
        "e2e_ms": statistics.median(e2e_ms), "h2d": h2d, "d2h": d2h, "plain": plain,
        "sm_count": props.multi_processor_count, "taus": taus, "sm_max_mhz": sm_max,
        "invariants": invariants, "launch": getattr(ctx, "tuned", None),
        "iteration": {"steps": W.iter_steps, "sweeps_per_step": W.iter_sweeps, "recursion": W.recursion,
                      "sweep_ms": iter_sweep_ms, "update_ms": iter_update_ms,
                      "attempts_per_ns": n_chains * V * W.iter_steps * W.iter_sweeps / (iter_sweep_ms * 1e6),
                      "update_share": iter_update_ms / (iter_sweep_ms + iter_update_ms)},
    }


def launches_per_run(launch, sweeps: int) -> int:
    """Sweep-kernel launches of one muca_run_sweeps call under a launch configuration."""
    spl = (launch or {}).get("sweeps_per_launch", 0)
    return 1 if not spl else -(-sweeps // spl)


def rt_roofline(r, world):
    tau = r["taus"]["mean"]
    if not tau:
        return None
    V = HEADLINE.L ** HEADLINE.dim
    peak = world * r["alu_peak"] / ALG_OPS_PER_ATTEMPT / (V * tau)
    achieved = world * r["rts"] / (r["t_ms"] / 1e3)
    return {"achieved": achieved, "peak": peak, "unit": "round trips/s", "frac": achieved / peak,
            "basis": "ALU peak / ops per attempt / (V x mean round-trip time in sweeps)"}


def plain_form(eamc, stream, S: int, W=HEADLINE):
    """One realization per launch: the same kernel with a single chain in the context."""
    import torch
    ctx = eamc.Context(seed=W.seed, device=0, stream=stream.cuda_stream)
    ctx.init_disorder(W.dim, W.L, 1, rid0=0)
    ctx.set_ensemble(0, 1, eamc.EA_POWERLAW, W.alpha, W.pole)
    with torch.cuda.stream(stream):
        ctx.run_sweeps(S)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        ctx.run_sweeps(S)
        e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1)
    ctx.close()
    return {"value": W.L ** W.dim * S / (ms * 1e6), "unit": UNIT,
            "what": f"one realization per launch, {S} sweeps, L={W.L}, power law"}


def bench_flat_same_schedule(S: int = 10_000, steps: int = 10):
    """The headline's realizations as flat-MUCA chains under the same schedule (Berg iteration,
    frozen weights, E_g fixed), for the paper's comparison of round-trip times (Table I)."""
    import torch

    from paper_2011_08560_gb300 import eamc
    W = HEADLINE
    stream = torch.cuda.Stream()
    ctx = build_context(eamc, 0, stream.cuda_stream, ensembles=("flat",))
    iterate_weights(ctx, W, stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        ctx.run_sweeps(S, count_roundtrips=True)
    e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1)
    recs = ctx.roundtrips()
    ctx.close()
    st = tau_stats(recs)
    return {"workload": f"3D L={W.L}, {W.n_real} realizations, flat MUCA, Berg iteration "
                        f"{W.iter_steps} x {W.iter_sweeps}, {steps} x {S} production sweeps",
            "attempts_per_ns": W.n_real * W.L ** 3 * S * steps / (ms * 1e6),
            "round_trips_per_s": st["round_trips"] / (ms / 1e3), "round_trip_time_sweeps": st}


def bench_l6_flat_pl(S: int = 10_000, steps: int = 5):
    """L=6, 1024 realizations x {flat, power law} = 2048 chains; a step is S sweeps with
    measurement plus one weight update (plain recursion)."""
    import torch

    from paper_2011_08560_gb300 import eamc
    W = L6_FLAT_PL
    stream = torch.cuda.Stream()
    ctx = eamc.Context(seed=W.seed, device=0, stream=stream.cuda_stream)
    ctx.init_disorder(W.dim, W.L, W.n_real, rid0=0, stream=0)
    ctx.init_disorder(W.dim, W.L, W.n_real, rid0=0, stream=1)
    ctx.set_ensemble(0, W.n_real, eamc.EA_FLAT)
    ctx.set_ensemble(W.n_real, W.n_real, eamc.EA_POWERLAW, W.alpha, W.pole)
    for _ in range(2):
        ctx.run_sweeps(S, count_roundtrips=True)
        ctx.update_weights()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        ctx.run_sweeps(S, count_roundtrips=True)
        ctx.update_weights()
    e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1)
    ctx.close()
    return {"workload": W.name, "chains": 2 * W.n_real, "steps": steps,
            "attempts_per_ns": 2 * W.n_real * W.L ** 3 * S * steps / (ms * 1e6)}


def _small_oracle_full():
    """Config 1 in the oracle, in full: the same schedule as bench_small."""
    import numpy as np

    import oracle
    W = SMALL
    c = oracle.Chain(W.dim, W.L, W.seed, 0, 0)
    lnW = np.zeros(c.b_top + 1)
    t0 = time.perf_counter()
    for _ in range(W.iter_steps):
        c.sweeps(W.iter_sweeps, oracle.quantize(W.dim, lnW))
        lnW = oracle.update_weights(W.dim, W.L, c.parity, oracle.FLAT, 0.0, 0.0, c.rt.e_min, lnW, c.hist)
        c.hist[:] = 0
    c.rt.e_g = c.rt.e_min
    t1 = time.perf_counter()
    c.sweeps(W.prod_sweeps, oracle.quantize(W.dim, lnW), count_rt=True)
    t2 = time.perf_counter()
    return {"seconds": t2 - t0, "production_seconds": t2 - t1, "n_rt": c.rt.n_rt,
            "t_first": c.rt.t_first, "t_last": c.rt.t_last, "E": c.E, "e_g": c.rt.e_g}


def _small_gpu(order: int):
    """Config 1 on the GPU in sweep order `order`: device ms of the iteration and production
    phases, the round-trip record and the final energy."""
    import torch

    from paper_2011_08560_gb300 import eamc
    W = SMALL
    stream = torch.cuda.Stream()
    ctx = eamc.Context(seed=W.seed, device=0, stream=stream.cuda_stream)
    ctx.set_sweep_order(order)
    ctx.init_disorder(W.dim, W.L, 1, rid0=0, stream=0)
    ctx.set_ensemble(0, 1, eamc.EA_FLAT)
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record(stream)
    for _ in range(W.iter_steps):
        ctx.run_sweeps(W.iter_sweeps)
        ctx.update_weights()
    e1.record(stream)
    stream.synchronize()
    ctx.set_eg(0, 1, None)
    ctx.roundtrips(reset=True)
    e1.record(stream)
    ctx.run_sweeps(W.prod_sweeps, count_roundtrips=True)
    e2.record(stream)
    stream.synchronize()
    it_ms, prod_ms = e0.elapsed_time(e1), e1.elapsed_time(e2)
    rec = ctx.roundtrips()[0]
    _, E, _ = ctx.state(spins=False)
    ctx.close()
    return it_ms, prod_ms, rec, int(E[0])


def bench_small():
    """Config 1: L=4, one realization, flat MUCA, 20 x 10^4 iteration sweeps then 10^5
    production sweeps, on the GPU and (in full, one core) in the oracle; same trajectory.  Also
    timed on the GPU in the checkerboard order (a different trajectory of the same ensemble)."""
    W = SMALL
    it_ms, prod_ms, rec, E = _small_gpu(0)
    it_c, prod_c, rec_c, _ = _small_gpu(1)
    orc = _small_oracle_full()
    same = (rec["n_rt"], rec["t_first"], rec["t_last"], E, rec["e_g"]) == \
        (orc["n_rt"], orc["t_first"], orc["t_last"], orc["E"], orc["e_g"])
    V = W.L ** W.dim
    total = V * (W.iter_steps * W.iter_sweeps + W.prod_sweeps)
    return {"workload": W.name, "gpu_ms": it_ms + prod_ms,
            "gpu_attempts_per_ns": total / ((it_ms + prod_ms) * 1e6),
            "gpu_production_round_trips_per_s": rec["n_rt"] / (prod_ms / 1e3),
            "round_trips": rec["n_rt"], "tau_sweeps": (rec["t_last"] - rec["t_first"]) / rec["n_rt"] if rec["n_rt"] else None,
            "oracle_seconds_one_core": orc["seconds"], "oracle_attempts_per_ns": total / (orc["seconds"] * 1e9),
            "oracle_production_round_trips_per_s": orc["n_rt"] / orc["production_seconds"],
            "same_trajectory_as_oracle": same,
            "checkerboard": {"gpu_ms": it_c + prod_c, "gpu_attempts_per_ns": total / ((it_c + prod_c) * 1e6),
                             "round_trips": rec_c["n_rt"],
                             "gpu_production_round_trips_per_s": rec_c["n_rt"] / (prod_c / 1e3)}}


def bench_pt(S: int = 100_000, equil: int = 10_000, sample_every: int = 100):
    """Config 3, PT: L=8, 1024 realizations x 32 temperatures (geometric beta in [0.2, 3]);
    `equil` sweeps of equilibration, in which E_g = the lowest energy any replica of a
    realization reached and E_hot = the mean energy at the hottest slot (sampled every
    `sample_every` sweeps of the second half); then S timed sweeps with round trips counted per
    replica (Sec. III, PT variant)."""
    import numpy as np
    import torch

    from paper_2011_08560_gb300 import eamc
    from paper_2011_08560_gb300.workloads import PT, geometric_betas
    stream = torch.cuda.Stream()
    ctx = eamc.Context(seed=PT["seed"], device=0, stream=stream.cuda_stream)
    betas = geometric_betas(PT["M"], PT["beta_min"], PT["beta_max"])
    ctx.pt_init(PT["dim"], PT["L"], PT["n_real"], betas)
    ctx.pt_run(equil // 2)
    hot = []
    for _ in range(equil // 2 // sample_every):
        ctx.pt_run(sample_every)
        _, E, _, _ = ctx.pt_state(spins=False)
        hot.append(E[:, 0].astype(np.int64))
    e_hot = np.floor(np.mean(hot, axis=0)).astype(np.int32)
    recs = ctx.pt_roundtrips(reset=True)
    e_g = np.array([min(r["e_min"] for r in rr) for rr in recs], dtype=np.int32)
    ctx.pt_set_rt_bounds(e_g, e_hot)
    sw0 = ctx.pt_swap_counts()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.pt_run(S, count_roundtrips=True)
    e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1)
    attempts = PT["n_real"] * PT["M"] * PT["L"] ** 3 * S
    swaps = ctx.pt_swap_counts() - sw0
    recs = ctx.pt_roundtrips()
    ctx.close()
    flat = [r for rr in recs for r in rr]
    taus = [(r["t_last"] - r["t_first"]) / r["n_rt"] for r in flat if r["n_rt"] > 0]
    n_rt = sum(r["n_rt"] for r in flat)
    return {"workload": "PT: 3D L=8, 1024 realizations x 32 temperatures, beta geometric in [0.2, 3], "
                        f"{equil} equilibration + {S} timed sweeps with round trips per replica",
            "sweeps": S, "ms": ms, "attempts_per_ns": attempts / (ms * 1e6),
            "alg_ops_per_attempt": PT_ALG_OPS, "achieved_Tops": attempts * PT_ALG_OPS / (ms * 1e9),
            "round_trips_per_s": n_rt / (ms / 1e3), "round_trips": n_rt,
            "round_trip_time_sweeps": {"mean": statistics.mean(taus) if taus else None,
                                       "median": statistics.median(taus) if taus else None,
                                       "replicas_with_round_trip": len(taus), "replicas": len(flat)},
            "e_hot_mean": float(e_hot.mean()), "e_g_mean": float(e_g.mean()),
            "swap_acceptance_mean": float(swaps.sum() / max(1, (PT["M"] - 1) * PT["n_real"] * S / 2))}


def bench_pt_protocol(rounds: int = 12, window: int = 1000, S: int = 4000):
    """The paper's PT protocol (Sec. II, PT) on L=8: M=20 replicas per realization, 1024
    realizations, T_max = 3.33 (above 3, as the paper requires) down to T_min = 0.465 (the paper
    gives none: chosen so that 20 replicas give exchange rates near its 40-60 % band),
    temperatures adapted per realization towards constant exchange rates (`rounds` windows of
    `window` sweeps), then S production sweeps timed."""
    import numpy as np
    import torch

    from paper_2011_08560_gb300 import eamc
    from paper_2011_08560_gb300.workloads import PT, geometric_betas
    M, beta_min, beta_max = 20, 0.3, 2.15
    stream = torch.cuda.Stream()
    ctx = eamc.Context(seed=PT["seed"], device=0, stream=stream.cuda_stream)
    ctx.pt_init(PT["dim"], PT["L"], PT["n_real"], geometric_betas(M, beta_min, beta_max))

    def rates():
        acc, att = ctx.pt_exchange_counts()
        return acc / att[None, :], att

    ctx.pt_run(window)
    r0, _ = rates()
    ctx.pt_adapt(0.0)                      # new window, temperatures unchanged
    for _ in range(rounds):
        ctx.pt_run(window)
        ctx.pt_adapt(0.5)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.pt_run(S)
    e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1)
    r1, att1 = rates()
    ctx.close()
    # spread that counting noise alone gives equal true rates (each realization's mean rate)
    rng = np.random.default_rng(0)
    pm = r1.mean(axis=1, keepdims=True)
    sim = rng.binomial(att1[None, :].astype(np.int64), np.repeat(pm, M - 1, axis=1)) / att1[None, :]
    noise_spread = float(np.median(sim.max(axis=1) - sim.min(axis=1)))
    attempts = PT["n_real"] * M * PT["L"] ** 3 * S

    def summary(r):
        spread = r.max(axis=1) - r.min(axis=1)
        return {"mean_rate": float(r.mean()), "median_spread": float(np.median(spread)),
                "realizations_all_pairs_in_40_60pct": float(np.mean(np.all((r >= 0.4) & (r <= 0.6), axis=1)))}

    return {"workload": f"PT protocol: 3D L=8, {PT['n_real']} realizations x {M} temperatures, "
                        f"beta in [{beta_min}, {beta_max}], {rounds} adaptation windows of "
                        f"{window} sweeps", "sweeps": S, "ms": ms, "attempts_per_ns": attempts / (ms * 1e6),
            "exchange_rates_geometric": summary(r0), "exchange_rates_adapted": summary(r1),
            "adapted_spread_from_counting_noise_alone": noise_spread}


def uneven_groups():
    """(kind index, L, first realization id, count) of the uneven batch: realization ids with
    L = Ls[id % 5], one contiguous id block per L; kind 0 power law, 1 flat, 2 1/k."""
    from paper_2011_08560_gb300.workloads import UNEVEN
    Ls = UNEVEN["Ls"]
    out = []
    for kind_idx in range(3):
        for L in Ls:
            n = sum(1 for r in range(UNEVEN["n_real"]) if Ls[r % len(Ls)] == L)
            out.append((kind_idx, L, Ls.index(L) * UNEVEN["n_real"], n))
    return out


def build_uneven(eamc, autotune, stream_ptr, S: int, order: int = 0):
    """The uneven batch as the bench runs it: chains, autotuned launch, one iteration step, then
    the 1/k chains take 1/k weights built from their estimate."""
    from paper_2011_08560_gb300.workloads import UNEVEN
    groups = [(3, L, n) for _, L, _, n in uneven_groups()]
    best = autotune.tune(groups, sweeps=20, order=order)
    ctx = eamc.Context(seed=UNEVEN["seed"], device=0, stream=stream_ptr)
    ctx.set_sweep_order(order)
    autotune.prepare(ctx, best)
    one_over_k = []
    for kind_idx, L, rid0, n in uneven_groups():
        first = ctx.init_disorder(3, L, n, rid0=rid0, stream=kind_idx)
        ctx.set_ensemble(first, n, eamc.EA_POWERLAW if kind_idx == 0 else eamc.EA_FLAT)
        if kind_idx == 2:
            one_over_k.append((first, n))
    autotune.launch(ctx, best)
    ctx.run_sweeps(S, count_roundtrips=False)
    ctx.update_weights()
    for first, n in one_over_k:
        ctx.build_ensemble(first, n, eamc.EA_ONE_OVER_K)
    return ctx, groups, best


def bench_uneven(S: int = 100, iters: int = 3, order: int = 0):
    """Uneven batch: 4096 realizations, L uniform over {4,6,8,10,12} (round robin by id), each
    as a power-law, a flat and a 1/k chain, in one launch per step (lexicographic order: the
    persistent work-queue kernel; checkerboard order: one block per tile); the
    weight-iteration loop is a captured CUDA graph."""
    import torch

    from paper_2011_08560_gb300 import autotune, eamc
    stream = torch.cuda.Stream()
    ctx, groups, best = build_uneven(eamc, autotune, stream.cuda_stream, S, order)
    attempts_per_sweep = sum(n * L ** 3 for _, L, n in groups)
    ctx.graph_capture(n_iter=iters, sweeps_per_iter=S, count_roundtrips=True, update_weights=True)
    ctx.graph_launch(1)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.graph_launch(1)
    e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1)
    ctx.close()
    return {"workload": "4096 realizations, L in {4,6,8,10,12} round robin, x3 ensembles "
                        "(power law, flat, 1/k), graph-captured iteration loop, sweep order "
                        + ("checkerboard" if order else "lexicographic"),
            "chains": sum(n for _, _, n in groups), "graph": f"{iters} x ({S} sweeps + weight update)",
            "ms": ms, "attempts_per_ns": attempts_per_sweep * S * iters / (ms * 1e6), "launch": best}


def bench_recursion(L: int = 8, n: int = 256, iters: int = 24, S: int = 2000, P: int = 20000):
    """Weight recursions side by side: the plain step and Berg's accumulated error-weighted one,
    flat and power-law ensembles, n chains of L^3, `iters` iterations of S sweeps, then P
    production sweeps with frozen weights.  Reported per variant: round trips in production
    (the paper's figure of merit), chains without one, mean lowest energy, median spread
    ln(max H / min H) of the production histogram between the lowest visited bin and E_top,
    and the device time of one weight update over all chains."""
    import numpy as np
    import torch

    from paper_2011_08560_gb300 import eamc
    out = {"workload": f"3D L={L}, {n} realizations (seed 3), {iters} x {S} iteration sweeps, "
                       f"{P} production sweeps"}
    stream = torch.cuda.Stream()
    for kind, kname in ((eamc.EA_FLAT, "flat"), (eamc.EA_POWERLAW, "power_law")):
        for mode, mname in ((eamc.EA_REC_PLAIN, "plain"), (eamc.EA_REC_BERG, "berg")):
            ctx = eamc.Context(seed=3, device=0, stream=stream.cuda_stream)
            ctx.init_disorder(3, L, n, rid0=0)
            ctx.set_ensemble(0, n, kind, -3.6, 96.0)
            ctx.set_recursion(0, n, mode)
            upd_ms = []
            for it in range(iters):
                ctx.run_sweeps(S)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx.update_weights()
                e1.record(stream)
                stream.synchronize()
                upd_ms.append(e0.elapsed_time(e1))
            ctx.set_eg(0, n, None)
            ctx.roundtrips(reset=True)
            ctx.histograms(reset=True)
            ctx.run_sweeps(P, count_roundtrips=True)
            H, R, D = ctx.histograms(), ctx.roundtrips(), ctx.describe()
            spread = []
            for k in range(n):
                h = H[k, :D[k]["b_top"] + 1]
                seg = h[np.nonzero(h)[0].min():].astype(float)
                spread.append(float(np.log(seg.max() / max(seg.min(), 1.0))))
            nrt = np.array([r["n_rt"] for r in R])
            out[f"{kname}_{mname}"] = {
                "round_trips": int(nrt.sum()), "chains_without_rt": int((nrt == 0).sum()),
                "e_min_mean": float(np.mean([r["e_min"] for r in R])),
                "spread_median": float(np.median(spread)),
                "update_ms": float(np.median(upd_ms[1:]))}
            ctx.close()
    return out


# the paper's number of PT replicas per lattice size (Sec. II, PT)
PT_REPLICAS = {3: 7, 4: 7, 5: 12, 6: 14, 8: 20}
# the paper's Table I: (r_pop, r_eps) of flat MUCA, the 1/k ensemble and PT relative to PL
PAPER_TABLE_ONE = {3: {"flat": (1.160, 1.174), "1/k": (1.0146, 1.0193), "PT": (1.637, 1.640)},
                   4: {"flat": (1.622, 1.68), "1/k": (1.288, 1.328), "PT": (1.175, 1.25)},
                   5: {"flat": (2.28, 2.44), "1/k": (1.63, 1.75), "PT": (1.136, 1.185)},
                   6: {"flat": (3.8, 3.9), "1/k": (2.59, 2.6), "PT": (2.8, 3.4)},
                   8: {"flat": (10.5, 14.2), "1/k": (6.9, 9.4), "PT": (2.1, 2.62)}}


def bench_profile_scan(L: int = 6, n_real: int = 128, dos_iters: int = 100, dos_sweeps: int = 10000,
                       prod_sweeps: int = 100000, pt: bool = True, order: int = 0):
    """Profile-parameter scan (Sec. II): power-law alpha x Delta E grid, flat and 1/k beside
    it, n_real realizations of L^3, density of states once per realization (power-law target,
    Berg's recursion), production with round-trip counting in one batched launch; PT with the
    paper's replica count on the same realizations.  Reports the mean round-trip time per
    ensemble, its ratio to flat, and the Table I analog: r_pop and r_eps (eps = 1e-4) of flat,
    1/k and PT relative to the power law (-3.6, 96), with jackknife errors, beside the paper's
    values (other disorder sets: context, not a target).  The MUCA chains sweep in `order`."""
    import time

    import numpy as np
    import torch

    from paper_2011_08560_gb300 import eamc, scan
    alphas, poles = (-1.5, -2.5, -3.6, -5.0), (24.0, 48.0, 96.0, 192.0)
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    res = scan.profile_scan(3, L, n_real, alphas, poles, seed=6, dos_iters=dos_iters,
                            dos_sweeps=dos_sweeps, prod_sweeps=prod_sweeps,
                            recursion=eamc.EA_REC_BERG, stream=stream.cuda_stream, order=order)
    wall = time.perf_counter() - t0
    pt_tau = pt_below = None
    M = PT_REPLICAS.get(L)
    if pt and M:
        pt_tau, pt_below = scan.pt_round_trips(3, L, n_real, M, res.e_g, seed=6, prod_sweeps=prod_sweeps,
                                               stream=stream.cuda_stream)
    wall_pt = time.perf_counter() - t0 - wall
    rows = res.summary()
    out = {"workload": f"3D L={L}, {n_real} realizations (seed 6), power law alpha in {list(alphas)} x "
                       f"Delta E in {list(poles)}, flat and 1/k; density of states {dos_iters} x "
                       f"{dos_sweeps} sweeps (Berg), {prod_sweeps} production sweeps; PT with M = {M} "
                       f"replicas, beta in [0.3, 2.15] adapted over 8 x 1000 sweeps, {prod_sweeps} sweeps; "
                       f"MUCA sites in the {'checkerboard' if order else 'lexicographic'} order",
           "wall_s": wall, "pt_wall_s": wall_pt, "best_power_law": res.best(),
           "ensembles": {r["ensemble"]: {k: v for k, v in r.items() if k != "ensemble"} for r in rows},
           "table_one": res.table_one(pt_tau, pt_below),
           "paper_table_one": PAPER_TABLE_ONE.get(L)}
    if pt_tau is not None:
        ok = np.isfinite(pt_tau)
        out["pt"] = {"mean_tau": float(np.mean(pt_tau[ok])) if ok.any() else None,
                     "without_rt": int((~ok).sum()), "below_eg": int(pt_below.sum())}
    return out


def bench_table_one_l8(n_real: int = 1024, prod_sweeps: int = 300_000, order: int = 0):
    """Table I analog at the headline's size, L=8, on its 1024 realizations: one density of
    states per realization from the headline's power-law Berg iteration, shared by flat MUCA,
    the power law (-3.6, 96) and the 1/k ensemble (each a chain of its own), and PT with the
    paper's M = 20 on the same realizations; production with round-trip counting.  The MUCA
    chains sweep in `order` (0 lexicographic, 1 checkerboard)."""
    import time

    import numpy as np
    import torch

    from paper_2011_08560_gb300 import eamc, scan
    W = HEADLINE
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    res = scan.profile_scan(3, W.L, n_real, (W.alpha,), (W.pole,), seed=W.seed, dos_iters=W.iter_steps,
                            dos_sweeps=W.iter_sweeps, prod_sweeps=prod_sweeps, recursion=eamc.EA_REC_BERG,
                            stream=stream.cuda_stream, tile_width=eamc.narrow_width(3, W.L, order),
                            order=order)
    wall = time.perf_counter() - t0
    pt_tau, pt_below = scan.pt_round_trips(3, W.L, n_real, PT_REPLICAS[W.L], res.e_g, seed=W.seed,
                                           prod_sweeps=prod_sweeps, stream=stream.cuda_stream)
    rows = {r["ensemble"]: {k: v for k, v in r.items() if k != "ensemble"} for r in res.summary()}
    ok = np.isfinite(pt_tau)
    rows["PT"] = {"mean_tau": float(np.mean(pt_tau[ok])) if ok.any() else None,
                  "median_tau": float(np.median(pt_tau[ok])) if ok.any() else None,
                  "without_rt": int((~ok).sum()), "requeued": int(pt_below.sum())}
    return {"workload": f"3D L={W.L}, {n_real} realizations (seed {W.seed}), density of states from "
                        f"{W.iter_steps} x {W.iter_sweeps} power-law Berg sweeps, flat / power law "
                        f"(-3.6, 96) / 1/k chains from it, PT with M = {PT_REPLICAS[W.L]}; {prod_sweeps} "
                        f"production sweeps each; MUCA sites in the "
                        f"{'checkerboard' if order else 'lexicographic'} order",
            "wall_s": time.perf_counter() - t0, "muca_wall_s": wall, "ensembles": rows,
            "table_one": res.table_one(pt_tau, pt_below), "paper_table_one": PAPER_TABLE_ONE[W.L]}


def bench_order(order: str = "lex", n_real: int = 1024, S: int = 10_000, steps: int = 3,
                iter_steps: int = 4, iter_sweeps: int = 2000):
    """The headline workload with the sites of a sweep in another order (the paper fixes none):
    same chains, same weight recursion (short iteration: the throughput of a production sweep
    does not depend on how far the weights converged), autotuned tile width and launch."""
    import dataclasses

    import torch

    from paper_2011_08560_gb300 import eamc
    W = dataclasses.replace(HEADLINE, n_real=n_real, iter_steps=iter_steps, iter_sweeps=iter_sweeps,
                            order=order)
    stream = torch.cuda.Stream()
    ctx = build_context(eamc, 0, stream.cuda_stream, W)
    iterate_weights(ctx, W, stream)
    ctx.run_sweeps(S // 10, count_roundtrips=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        ctx.run_sweeps(S, count_roundtrips=True)
    e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1)
    launch = getattr(ctx, "tuned", None)
    ctx.check()
    ctx.close()
    return {"workload": f"3D L={W.L}, {n_real} realizations, power law (-3.6, 96), sweep order {order}, "
                        f"{steps} x {S} production sweeps after {iter_steps} x {iter_sweeps} Berg iteration sweeps",
            "attempts_per_ns": n_real * W.L ** 3 * S * steps / (ms * 1e6), "launch": launch}


def bench_paper_samples(n_real: int = 4096, S: int = 10_000, steps: int = 3, iter_steps: int = 4,
                        iter_sweeps: int = 2000):
    """The headline ensemble (L=8, power law, production with frozen weights) at the paper's
    sample count for L=8 (4000 realizations; 4096 here): a batch large enough to fill the GPU.
    Short Berg iteration (the throughput of a production sweep does not depend on how far the
    weights converged), autotuned tile width and launch."""
    import dataclasses

    import torch

    from paper_2011_08560_gb300 import eamc
    W = dataclasses.replace(HEADLINE, n_real=n_real, iter_steps=iter_steps, iter_sweeps=iter_sweeps)
    stream = torch.cuda.Stream()
    ctx = build_context(eamc, 0, stream.cuda_stream, W)
    iterate_weights(ctx, W, stream)
    ctx.run_sweeps(S // 10, count_roundtrips=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        ctx.run_sweeps(S, count_roundtrips=True)
    e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1)
    launch = getattr(ctx, "tuned", None)
    ctx.close()
    return {"workload": f"3D L={W.L}, {n_real} realizations, power law (-3.6, 96), {steps} x {S} production "
                        f"sweeps after {iter_steps} x {iter_sweeps} Berg iteration sweeps",
            "attempts_per_ns": n_real * W.L ** 3 * S * steps / (ms * 1e6), "launch": launch}


def bench_serving(window_s: float = 10.0, drain_s: float = 30.0, order: int = 0):
    """Serving (config 5): Poisson arrivals (200 jobs/s) of realization jobs, L in {4..12},
    round-trip targets log-uniform in [10, 1000]; power-law MUCA with Berg's recursion; state
    resident on the device, admission by memory, job control on the device, asynchronous
    read-back.  Latency percentiles cover every job: censored jobs count at their cap.  The
    served chains sweep in `order` (0 lexicographic, 1 colour order)."""
    from paper_2011_08560_gb300 import serve
    from paper_2011_08560_gb300.workloads import SERVING
    jobs = serve.poisson_jobs(SERVING["rate_hz"], window_s, SERVING["Ls"], SERVING["rt_min"],
                              SERVING["rt_max"], seed=SERVING["seed"], iter_steps=8, ticks_per_step=8,
                              max_prod_ticks=2000, max_requeues=4)
    server = serve.Server(seed=SERVING["seed"], Ls=SERVING["Ls"], base_sweeps=16, mem_budget=8 << 30,
                          poll_ticks=8, max_ahead=64, order=order)
    stats = serve.run_poisson(server, jobs, duration_s=window_s, drain_s=drain_s)
    server.close()
    stats["workload"] = (f"Poisson {SERVING['rate_hz']:.0f} jobs/s for {window_s:.0f} s, L in 4..12, "
                         f"round-trip targets log-uniform [10, 1000], power law + Berg, 8 x 8 iteration "
                         f"ticks, production cap 2000 ticks (16 sweeps per tick at L=12, (12/L)^3 times "
                         f"more at smaller L), sites in the {'colour' if order else 'lexicographic'} order")
    return stats


def bench_serving_saturated(n_jobs: int = 4096, window_s: float = 5.0, base: int = 16):
    """The serving loop under saturation: n_jobs jobs of L uniform in {4..12} submitted at once
    (long targets: all stay running), served for window_s after admission; against the plain
    batched launch of the same chains (same tiles, same sweeps per tick).  The ratio is the
    share of the sweep kernel's throughput the loop keeps (its per-tick control, weight steps
    and read-backs)."""
    import time

    import torch

    from paper_2011_08560_gb300 import eamc, serve
    from paper_2011_08560_gb300.workloads import SERVING
    Ls = SERVING["Ls"]
    server = serve.Server(seed=SERVING["seed"], Ls=Ls, base_sweeps=base, mem_budget=8 << 30)
    jobs = [serve.Job(jid=k, L=Ls[k % len(Ls)], rid=k, rt_target=10 ** 6, iter_steps=8, ticks_per_step=8,
                      max_prod_ticks=10 ** 5, max_requeues=4) for k in range(n_jobs)]
    for j in jobs:
        server.submit(j)
    server.step(80)                       # admission and the jobs' iteration phases
    server.poll(wait=True)
    a0, t0 = server.stats()["attempts"], time.perf_counter()
    while time.perf_counter() - t0 < window_s:
        server.step(8)
        server.poll()
    server.poll(wait=True)
    t1 = time.perf_counter()
    st = server.stats()
    served = (st["attempts"] - a0) / ((t1 - t0) * 1e9)
    server.close()
    # the same chains as one batch: per L, n_jobs / 9 chains with the server's sweeps per tick
    stream = torch.cuda.Stream()
    ctx = eamc.Context(seed=SERVING["seed"], device=0, stream=stream.cuda_stream)
    attempts_per_tick = 0
    for i, L in enumerate(Ls):
        n = sum(1 for k in range(n_jobs) if k % len(Ls) == i)
        ctx.init_disorder(3, L, n, rid0=i * n_jobs)
        mul = max(1, int((max(Ls) / L) ** 3 + 0.5))
        ctx.set_sweep_multiplier(L, mul)
        attempts_per_tick += n * L ** 3 * base * mul
    ctx.run_sweeps(base)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.run_sweeps(base * 100)
    e1.record(stream)
    stream.synchronize()
    batch = attempts_per_tick * 100 / (e0.elapsed_time(e1) * 1e6)
    ctx.close()
    return {"workload": f"{n_jobs} jobs, L uniform in 4..12, all running (power law, Berg), {window_s:.0f} s "
                        f"window after admission; batch = the same chains in one muca_run_sweeps",
            "served_attempts_per_ns": served, "batch_attempts_per_ns": batch,
            "served_over_batch": served / batch, "ticks": st["ticks"], "lanes": st["lanes"]}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    W = headline(args)
    config = {"workload": W.name, "L": W.L, "realizations_per_gpu": W.n_real,
              "chains_per_gpu": W.n_real, "ensembles": [f"power-law(alpha={W.alpha:g}, dE={W.pole:g})"],
              "sweeps_per_step": args.sweeps_per_step,
              "weight_iteration": f"{W.iter_steps} x {W.iter_sweeps} sweeps, {W.recursion} recursion, "
                                  f"before timing; then E_g fixed, weights frozen",
              "step": "production sweeps with histogram, lowest-energy and round-trip measurement",
              "sweep_order": {"lex": "lexicographic", "colour": "checkerboard (colour class by colour "
                              "class, each in lexicographic order)"}[W.order],
              "l2": "flushed between steps (256 MB write)",
              "parallelism": f"independent realizations, {world} GPU(s)"}

    if args.impl == "reference":
        if rank != 0:
            return
        steps = []
        per = max(4.0, 60.0 / max(1, args.steps + args.warmup))
        base = None
        for k in range(args.warmup + args.steps):
            base = oracle_sample(target_s=min(per, 20.0), W=W)
            if k >= args.warmup:
                steps.append(base)
        val = statistics.mean(s["value"] for s in steps)
        wall = sum(s["wall_s"] for s in steps)
        line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * wall / max(1, len(steps)),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
                "data": "synthetic (seeded +-J disorder)", "config": config, "impl": "reference",
                "cpu_baseline": {"value": val, "unit": UNIT, "cores": base["cores"], "kind": "oracle",
                                 "sample": base["sample"]},
                "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if args.only:
        fn = {"pt": lambda: bench_pt(args.pt_sweeps), "pt_protocol": bench_pt_protocol,
              "uneven": bench_uneven, "uneven_checkerboard": lambda: bench_uneven(order=1),
              "serving": lambda: bench_serving(order=1), "serving_colour": lambda: bench_serving(order=1),
              "serving_lex": lambda: bench_serving(order=0),
              "scan": lambda: bench_profile_scan(L=args.scan_L, prod_sweeps=args.scan_prod_sweeps),
              "scan_checkerboard": lambda: bench_profile_scan(L=args.scan_L, prod_sweeps=args.scan_prod_sweeps,
                                                              order=1),
              "recursion": bench_recursion, "small": bench_small, "flat": bench_flat_same_schedule,
              "serving_saturated": bench_serving_saturated, "table_one_l8": bench_table_one_l8,
              "table_one_l8_checkerboard": lambda: bench_table_one_l8(order=1),
              "paper_samples": bench_paper_samples, "lex": lambda: bench_order("lex"),
              "l6": bench_l6_flat_pl}
        print(json.dumps({"only": args.only, **fn[args.only]()}))
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(W=W)   # spawn pool before the first CUDA call
    r = run_gpu(args, rank, world)
    extras = None
    if rank == 0 and world == 1 and not args.no_extras:
        extras = {"headline_lexicographic": bench_order("lex"),
                  "paper_samples_l8": bench_paper_samples(), "table_one_l8": bench_table_one_l8(),
                  "table_one_l8_checkerboard": bench_table_one_l8(order=1),
                  "l6_flat_pl": bench_l6_flat_pl(),
                  "small": bench_small(), "pt": bench_pt(args.pt_sweeps), "pt_protocol": bench_pt_protocol(),
                  "uneven": bench_uneven(), "serving": bench_serving(order=1),
                  "serving_lexicographic": bench_serving(order=0),
                  "serving_saturated": bench_serving_saturated(), "recursion": bench_recursion(),
                  "scan": bench_profile_scan(), "scan_checkerboard": bench_profile_scan(order=1)}
    if rank != 0:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
        return
    attempts_e2e = r["attempts_per_step"] * world
    lat_peak = world * r["n_chains"] * r["sm_max_mhz"] * 1e-3 / LATENCY_FLOOR_CYCLES
    line = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["t_ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic (seeded +-J disorder, random initial spins)", "config": config,
        "round_trips_per_s": world * r["rts"] / (r["t_ms"] / 1e3),
        # Sec. III: tau_i = (t_last - t_first) / n_rt over the production sweeps (warm-up + timed)
        "round_trip_time_sweeps": r["taus"],
        "invariant_check": r["invariants"],
        "iteration_phase": r["iteration"],
        # round trips/s against the ALU roofline: attempts/s at the roofline / (V x mean tau)
        "round_trips_roofline": rt_roofline(r, world),
        # the bound that applies to a batch of serial chains: every chain needs at least
        # LATENCY_FLOOR_CYCLES per attempt (select + shared-memory load + compare, loads issued
        # one attempt ahead), so attempts/ns <= chains x SM clock / floor
        "latency_roofline": {"achieved": r["value"], "peak": lat_peak, "unit": UNIT,
                             "frac": r["value"] / lat_peak,
                             "cycles_per_attempt_floor": LATENCY_FLOOR_CYCLES,
                             "cycles_per_attempt_achieved": world * r["n_chains"] * r["sm_max_mhz"] * 1e-3 / r["value"]},
        "plain_form": r["plain"],
        "e2e": {"value": attempts_e2e / (r["e2e_ms"] * 1e6), "unit": UNIT,
                "h2d_bytes_per_step": r["h2d"], "d2h_bytes_per_step": r["d2h"]},
        "gpu_launches": args.steps * launches_per_run(r["launch"], args.sweeps_per_step),
        "launch": r["launch"],
        "roofline": {"bound": "alu", "achieved": r["achieved_ops"] / 1e12,
                     "peak": r["alu_peak"] / 1e12, "unit": "Tops/s",
                     "frac": r["achieved_ops"] / r["alu_peak"], "traffic": SWEEP_TRAFFIC_BYTES,
                     "traffic_basis": "ncu dram read+write of one launch (one-time table and lattice "
                                      "staging, independent of the sweeps per launch)",
                     "kernel": "muca_checker_kernel<3, 0>" if W.order == "colour" else "muca_sweep_kernel<3>",
                     "ops_per_attempt": ALG_OPS_PER_ATTEMPT,
                     "peak_basis": f"{r['sm_count']} SMs x 128 lane-instructions/clk x max SM clock "
                                   f"(MEASURED_PEAKS.json sm_max_mhz)"},
        "clocks": r["clocks"],
        "cpu_baseline": cpu and {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")},
        "extras": extras,
    }
    if extras and extras.get("pt"):
        pt = extras["pt"]
        line["pt_roofline"] = {"bound": "alu", "achieved": pt["achieved_Tops"], "peak": r["alu_peak"] / 1e12,
                               "unit": "Tops/s", "frac": pt["achieved_Tops"] * 1e12 / r["alu_peak"],
                               "kernel": "pt_kernel", "ops_per_attempt": PT_ALG_OPS}
    print(json.dumps(line))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
