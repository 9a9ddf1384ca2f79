"""Benchmark: batched power-law / flat MUCA on the 3D +-J EA spin glass, one JSON line.

Workload: L=6, 1024 disorder realizations, each run as a flat-MUCA chain and as a
power-law-MUCA chain (alpha=-3.6, Delta E=96) -> 2048 chains in one context, packed 32 per
warp.  One step = one pass of the hot path over the batch: `sweeps_per_step` sweeps of
generalized Metropolis with histogram, lowest-energy and round-trip measurement
(muca_run_sweeps), then one weight-iteration update with re-quantisation
(muca_update_weights).  Metric: spin-flip attempts per ns (whole job), with round trips per
second beside it.

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

from paper_2011_08560_gb300.workloads import HEADLINE  # noqa: E402

METRIC = "spin-flip attempts/ns"
UNIT = "attempts/ns"
# algorithmic integer lane-operations per spin-flip attempt:
# 10 (quarter of a Philox4x32-10 call) + 3.5 (bit-sliced local field, 32 chains per word,
# plus extraction) + 3 (threshold fetch and compare) + 2 (flip and energy update)
# + 3 (lowest energy and round-trip check)
ALG_OPS_PER_ATTEMPT = 21.5
# per-chain latency floor of one MUCA attempt in SM cycles: with the next attempt's candidate
# thresholds loaded one attempt ahead, two attempts cost one address select, one shared-memory
# load (about 29 cycles, measured) and the compare / select of the decision, about 40 cycles
LATENCY_FLOOR_CYCLES = 20.0
# PT, per site word of 32 lattices (32 attempts): 12 word loads + 14 bit ops for the
# unsatisfied counts + 4 for the classes, about 8 compared bit planes (2 Philox4x32-10 calls of
# 40 ops, 5 ops per plane) and the flip: about 150 lane-operations per 32 attempts
PT_ALG_OPS = 4.7
# dram__bytes_read.sum + dram__bytes_write.sum of one sweep launch of the headline workload
# (ncu, profiles/muca_sweep_L6_2048chains.md)
SWEEP_TRAFFIC_BYTES = 11.59e6


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
    ap.add_argument("--only", choices=["pt", "pt_protocol", "uneven", "serving", "recursion", "scan"],
                    default=None,
                    help="run one secondary workload alone and print its record (profiling)")
    ap.add_argument("--pt-sweeps", type=int, default=200)
    ap.add_argument("--scan-L", type=int, default=6, help="lattice size of the profile scan")
    ap.add_argument("--scan-prod-sweeps", type=int, default=100_000,
                    help="production sweeps of the profile scan")
    return ap.parse_args()


# ------------------------------------------------------------------------------ oracle (CPU)
def _oracle_worker(args):
    import numpy as np

    import oracle
    dim, L, seed, rid, stream, kind, sweeps = args
    c = oracle.Chain(dim, L, seed, rid, stream)
    lnW = np.zeros(c.b_top + 1)
    t0 = time.perf_counter()
    c.sweeps(sweeps, oracle.quantize(dim, lnW), count_rt=True)
    lnW = oracle.update_weights(dim, L, c.parity, kind, HEADLINE.alpha, HEADLINE.pole,
                                c.rt.e_min, lnW, c.hist)
    dt = time.perf_counter() - t0
    return c.V * sweeps, dt, c.rt.n_rt


def oracle_sample(target_s: float = 15.0, cores: int | None = None):
    """Times the oracle on all host cores on a bounded sample of the workload."""
    import oracle
    oracle.build()
    cores = cores or os.cpu_count() or 1
    W = HEADLINE
    # calibrate one chain
    calib = _oracle_worker((W.dim, W.L, W.seed, 0, 0, 0, 200))
    per_sweep = calib[1] / 200
    chains = 2 * cores
    sweeps = max(50, int(target_s * cores / (chains * per_sweep)))
    jobs = [(W.dim, W.L, W.seed, k // 2, k % 2, k % 2, sweeps) for k in range(chains)]
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_worker, jobs)
    wall = time.perf_counter() - t0
    attempts = sum(r[0] for r in res)
    return {"value": attempts / (wall * 1e9), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{chains} chains (flat and power law alternating) x {sweeps} sweeps + one "
                      f"weight update each, L={W.L}, {wall:.1f} s wall on {cores} processes",
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


def build_context(eamc, rank: int, stream_ptr: int):
    W = HEADLINE
    ctx = eamc.Context(seed=W.seed, device=0, stream=stream_ptr)
    n = W.n_real
    rid0 = shard_rid0(rank, n)
    ctx.init_disorder(W.dim, W.L, n, rid0=rid0, stream=0)          # flat MUCA chains
    ctx.init_disorder(W.dim, W.L, n, rid0=rid0, stream=1)          # power-law MUCA chains
    ctx.set_ensemble(0, n, eamc.EA_FLAT)
    ctx.set_ensemble(n, n, eamc.EA_POWERLAW, W.alpha, W.pole)
    return ctx


def total_rt(ctx):
    return sum(r["n_rt"] for r in ctx.roundtrips())


def run_gpu(args, rank, world):
    import numpy as np
    import torch

    from paper_2011_08560_gb300 import eamc

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    W = HEADLINE
    S = args.sweeps_per_step
    stream = torch.cuda.Stream()
    ctx = build_context(eamc, rank, stream.cuda_stream)
    n_chains = ctx.num_chains()
    V = W.L ** W.dim
    attempts_per_step = n_chains * V * S
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2

    def step():
        ctx.run_sweeps(S, count_roundtrips=True)
        ctx.update_weights()

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    stream.synchronize()
    rt0 = total_rt(ctx)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    # dominant kernel alone: one sweeps launch per step, timed with its own events
    k_starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    k_ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    with ClockSampler(int(os.environ.get("LOCAL_RANK", 0))) as clk:
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(k))                       # evict L2 between steps
                starts[k].record(stream)
                k_starts[k].record(stream)
                ctx.run_sweeps(S, count_roundtrips=True)
                k_ends[k].record(stream)
                ctx.update_weights()
                ends[k].record(stream)
        stream.synchronize()
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    kern_ms = [s.elapsed_time(e) for s, e in zip(k_starts, k_ends)]
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
    # mean round-trip time in sweeps (Sec. III: tau_i = (t_last - t_first) / n_rt) of the chains
    # with a round trip so far, by ensemble; the weights iterate once per step meanwhile
    taus = {"flat": [], "power_law": []}
    for c, rec in enumerate(ctx.roundtrips()):
        if rec["n_rt"] > 0:
            taus["flat" if c < W.n_real else "power_law"].append((rec["t_last"] - rec["t_first"]) / rec["n_rt"])
    value = world * attempts_per_step * args.steps / (t_ms * 1e6)
    kern_avg_s = statistics.mean(kern_ms) / 1e3
    achieved_ops = attempts_per_step * ALG_OPS_PER_ATTEMPT / kern_avg_s
    props = torch.cuda.get_device_properties(0)
    peaks = json.loads((ROOT / "MEASURED_PEAKS.json").read_text()) if (ROOT / "MEASURED_PEAKS.json").exists() else {}
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = props.multi_processor_count * 4 * 32 * sm_max * 1e6   # lane-instr/s issue limit

    # end to end through the C ABI with host buffers in pinned memory (weights in; histograms,
    # weights and round-trip records out)
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
            ctx.update_weights()
            ctx.get_weights(rows=rows, out=lnW_host)
            ctx.roundtrips_array(out=rt)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    h2d = lnW_host.nbytes
    d2h = hist.nbytes + lnW_host.nbytes + rt.nbytes

    plain = None
    if not args.no_plain and rank == 0:
        plain = plain_form(eamc, stream, S=200)

    return {
        "value": value, "t_ms": t_ms, "step_ms": step_ms, "kern_ms": kern_ms, "wall": wall,
        "rts": rts, "attempts_per_step": attempts_per_step, "n_chains": n_chains,
        "achieved_ops": achieved_ops, "alu_peak": alu_peak, "clocks": clk.summary(),
        "e2e_ms": statistics.median(e2e_ms), "h2d": h2d, "d2h": d2h, "plain": plain,
        "sm_count": props.multi_processor_count, "taus": taus, "sm_max_mhz": sm_max,
        "invariants": invariants,
    }


def rt_roofline(r, world):
    all_taus = r["taus"]["flat"] + r["taus"]["power_law"]
    if not all_taus:
        return None
    V = HEADLINE.L ** HEADLINE.dim
    peak = world * r["alu_peak"] / ALG_OPS_PER_ATTEMPT / (V * statistics.mean(all_taus))
    achieved = world * r["rts"] / (r["t_ms"] / 1e3)
    return {"achieved": achieved, "peak": peak, "unit": "round trips/s", "frac": achieved / peak,
            "basis": "ALU peak / ops per attempt / (V x mean round-trip time in sweeps)"}


def plain_form(eamc, stream, S: int):
    """One realization per launch: the same kernel with a single chain in the context."""
    import torch
    W = HEADLINE
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
            "what": f"one realization per launch, {S} sweeps, L={W.L}"}


def bench_pt(S: int = 200):
    """PT workload: L=8, 1024 realizations x 32 temperatures (geometric beta in [0.2, 3])."""
    import torch

    from paper_2011_08560_gb300 import eamc
    from paper_2011_08560_gb300.workloads import PT, geometric_betas
    stream = torch.cuda.Stream()
    ctx = eamc.Context(seed=PT["seed"], device=0, stream=stream.cuda_stream)
    betas = geometric_betas(PT["M"], PT["beta_min"], PT["beta_max"])
    ctx.pt_init(PT["dim"], PT["L"], PT["n_real"], betas)
    ctx.pt_run(20)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.pt_run(S)
    e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1)
    attempts = PT["n_real"] * PT["M"] * PT["L"] ** 3 * S
    swaps = ctx.pt_swap_counts()
    ctx.close()
    return {"workload": "PT: 3D L=8, 1024 realizations x 32 temperatures, beta geometric in [0.2, 3]",
            "sweeps": S, "ms": ms, "attempts_per_ns": attempts / (ms * 1e6),
            "alg_ops_per_attempt": PT_ALG_OPS, "achieved_Tops": attempts * PT_ALG_OPS / (ms * 1e9),
            "swap_acceptance_mean": float(swaps.sum() / max(1, (PT["M"] - 1) * PT["n_real"] * (20 + S) / 2))}


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


def build_uneven(eamc, autotune, stream_ptr, S: int):
    """The uneven batch as the bench runs it: chains, autotuned launch, one iteration step, then
    the 1/k chains take 1/k weights built from their estimate."""
    from paper_2011_08560_gb300.workloads import UNEVEN
    ctx = eamc.Context(seed=UNEVEN["seed"], device=0, stream=stream_ptr)
    groups, one_over_k = [], []
    for kind_idx, L, rid0, n in uneven_groups():
        first = ctx.init_disorder(3, L, n, rid0=rid0, stream=kind_idx)
        ctx.set_ensemble(first, n, eamc.EA_POWERLAW if kind_idx == 0 else eamc.EA_FLAT)
        if kind_idx == 2:
            one_over_k.append((first, n))
        groups.append((3, L, n))
    best = autotune.apply(ctx, groups, sweeps=20)
    ctx.run_sweeps(S, count_roundtrips=False)
    ctx.update_weights()
    for first, n in one_over_k:
        ctx.build_ensemble(first, n, eamc.EA_ONE_OVER_K)
    return ctx, groups, best


def bench_uneven(S: int = 100, iters: int = 3):
    """Uneven batch: 4096 realizations, L uniform over {4,6,8,10,12} (round robin by id), each
    as a power-law, a flat and a 1/k chain, in one persistent launch per step; the
    weight-iteration loop is a captured CUDA graph."""
    import torch

    from paper_2011_08560_gb300 import autotune, eamc
    stream = torch.cuda.Stream()
    ctx, groups, best = build_uneven(eamc, autotune, stream.cuda_stream, S)
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
                        "(power law, flat, 1/k), graph-captured iteration loop",
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


def bench_profile_scan(L: int = 6, n_real: int = 128, dos_iters: int = 100, dos_sweeps: int = 10000,
                       prod_sweeps: int = 100000):
    """Profile-parameter scan (Sec. II): power-law alpha x Delta E grid, flat and 1/k beside
    it, n_real realizations of L^3, density of states once per realization (power-law target,
    Berg's recursion), production with round-trip counting in one batched launch.  Reports the
    mean round-trip time per ensemble and its ratio to flat (jackknife over realizations)."""
    import time

    import torch

    from paper_2011_08560_gb300 import eamc, scan
    alphas, poles = (-1.5, -2.5, -3.6, -5.0), (24.0, 48.0, 96.0, 192.0)
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    res = scan.profile_scan(3, L, n_real, alphas, poles, seed=6, dos_iters=dos_iters,
                            dos_sweeps=dos_sweeps, prod_sweeps=prod_sweeps,
                            recursion=eamc.EA_REC_BERG, stream=stream.cuda_stream)
    wall = time.perf_counter() - t0
    rows = res.summary()
    return {"workload": f"3D L={L}, {n_real} realizations (seed 6), power law alpha in {list(alphas)} x "
                        f"Delta E in {list(poles)}, flat and 1/k; density of states {dos_iters} x "
                        f"{dos_sweeps} sweeps (Berg), {prod_sweeps} production sweeps",
            "wall_s": wall, "best_power_law": res.best(),
            "ensembles": {r["ensemble"]: {k: v for k, v in r.items() if k != "ensemble"} for r in rows}}


def bench_serving(window_s: float = 4.0, drain_s: float = 20.0):
    """Serving: Poisson arrivals (200 jobs/s) of realization jobs, L in {4..12}, round-trip
    targets log-uniform in [10, 1000]; device-resident state, memory-based admission."""
    from paper_2011_08560_gb300 import serve
    from paper_2011_08560_gb300.workloads import SERVING
    jobs = serve.poisson_jobs(SERVING["rate_hz"], window_s, SERVING["Ls"], SERVING["rt_min"],
                              SERVING["rt_max"], seed=SERVING["seed"], iter_steps=4,
                              ticks_per_step=4, max_prod_ticks=200)
    server = serve.Server(seed=SERVING["seed"], Ls=SERVING["Ls"], base_sweeps=16,
                          mem_budget=4 << 30)
    stats = serve.run_poisson(server, jobs, duration_s=window_s, drain_s=drain_s)
    server.close()
    stats["workload"] = (f"Poisson {SERVING['rate_hz']:.0f} jobs/s for {window_s:.0f} s, L in 4..12, "
                         f"round-trip targets log-uniform [10, 1000], sweep caps (censored jobs counted)")
    return stats


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    W = HEADLINE
    config = {"workload": W.name, "L": W.L, "realizations_per_gpu": W.n_real,
              "chains_per_gpu": 2 * W.n_real, "ensembles": ["flat", "power-law(alpha=-3.6, dE=96)"],
              "sweeps_per_step": args.sweeps_per_step,
              "step": "sweeps with measurement + one weight-iteration update",
              "l2": "flushed between steps (256 MB write)",
              "parallelism": f"independent realizations, {world} GPU(s)"}

    if args.impl == "reference":
        if rank != 0:
            return
        steps = []
        per = max(4.0, 60.0 / max(1, args.steps + args.warmup))
        base = None
        for k in range(args.warmup + args.steps):
            base = oracle_sample(target_s=min(per, 20.0))
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
              "uneven": bench_uneven, "serving": bench_serving,
              "scan": lambda: bench_profile_scan(L=args.scan_L, prod_sweeps=args.scan_prod_sweeps),
              "recursion": bench_recursion}
        print(json.dumps({"only": args.only, **fn[args.only]()}))
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample()      # spawn pool before the first CUDA call
    r = run_gpu(args, rank, world)
    extras = None
    if rank == 0 and world == 1 and not args.no_extras:
        extras = {"pt": bench_pt(), "pt_protocol": bench_pt_protocol(), "uneven": bench_uneven(),
                  "serving": bench_serving(), "recursion": bench_recursion(), "scan": bench_profile_scan()}
    if rank != 0:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
        return
    attempts_e2e = r["attempts_per_step"] * world
    line = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["t_ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic (seeded +-J disorder, random initial spins)", "config": config,
        "round_trips_per_s": world * r["rts"] / (r["t_ms"] / 1e3),
        "invariant_check": r["invariants"],
        "round_trip_time_sweeps": {
            k: {"mean": statistics.mean(v) if v else None, "chains_with_round_trip": len(v)}
            for k, v in r["taus"].items()},
        # round trips/s against the ALU roofline: attempts/s at the roofline / (V x mean tau)
        "round_trips_roofline": rt_roofline(r, world),
        # the bound that applies to a batch of serial chains: every chain needs at least
        # LATENCY_FLOOR_CYCLES per attempt (select + shared-memory load + compare, loads issued
        # one attempt ahead), so attempts/ns <= chains x SM clock / floor
        "latency_roofline": {"achieved": r["value"],
                             "peak": world * r["n_chains"] * r["sm_max_mhz"] * 1e-3 / LATENCY_FLOOR_CYCLES,
                             "unit": UNIT,
                             "frac": r["value"] / (world * r["n_chains"] * r["sm_max_mhz"] * 1e-3 / LATENCY_FLOOR_CYCLES),
                             "cycles_per_attempt_floor": LATENCY_FLOOR_CYCLES,
                             "cycles_per_attempt_achieved": world * r["n_chains"] * r["sm_max_mhz"] * 1e-3 / r["value"]},
        "plain_form": r["plain"],
        "e2e": {"value": attempts_e2e / (r["e2e_ms"] * 1e6), "unit": UNIT,
                "h2d_bytes_per_step": r["h2d"], "d2h_bytes_per_step": r["d2h"]},
        "gpu_launches": 3 * args.steps,
        "roofline": {"bound": "alu", "achieved": r["achieved_ops"] / 1e12,
                     "peak": r["alu_peak"] / 1e12, "unit": "Tops/s",
                     "frac": r["achieved_ops"] / r["alu_peak"], "traffic": SWEEP_TRAFFIC_BYTES,
                     "traffic_source": "profiles/muca_sweep_L6_2048chains.md (dram read+write of one "
                                       "launch; one-time staging of the tables, independent of sweeps)",
                     "kernel": "muca_sweep_kernel<3>",
                     "ops_per_attempt": ALG_OPS_PER_ATTEMPT,
                     "peak_basis": f"{r['sm_count']} SMs x 128 lane-instructions/clk x max SM clock"},
        "clocks": r["clocks"],
        "cpu_baseline": cpu and {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")},
        "extras": extras,
    }
    print(json.dumps(line))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
