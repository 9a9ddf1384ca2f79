"""Profile-parameter scan of the power-law ensemble (Sec. II, Eq. "power_law"), batched.

The paper tunes the two profile parameters (exponent alpha, pole offset Delta E) by comparing
mean round-trip times (Sec. III) over its disorder realizations, with the density of states of
each realization determined once and shared by the ensembles compared.  Here every step runs
on the device in one context:

1. density of states: one chain per realization iterates its weights with a power-law target
   (as the paper determined its densities of states; Sec. II recursion, plain or Berg's
   accumulated form); ln Omega = ln P_SH - ln W afterwards, E_g = its lowest energy;
2. for the flat ensemble, each parameter pair (alpha, Delta E) and the 1/k ensemble
   (Eq. "1/k"), one chain per realization (a separate random stream) receives that estimate
   (muca_copy_weights) and builds its weights (muca_build_ensemble);
3. production: all chains sweep in one batched launch with round-trip counting;
   tau_i = (t_last - t_first) / n_rt per chain (the estimation chains sweep along, unused).

The result holds, per ensemble, the per-realization round-trip times, their mean, the number
of realizations without a round trip, and (Sec. III) the ratio of mean round-trip times to the
flat ensemble with a jackknife error over realizations that have a round trip in both.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import analysis, eamc


@dataclass
class ScanResult:
    labels: list            # ensemble names, "flat", "1/k", "pl(alpha,dE)"
    params: list            # (kind, alpha, pole) per label
    tau: np.ndarray         # [ensembles, realizations] round-trip time in sweeps (inf: none)
    n_rt: np.ndarray        # [ensembles, realizations]
    requeue: np.ndarray     # [ensembles, realizations] a lower energy than E_g was found
    e_g: np.ndarray         # [realizations] E_g from the density-of-states stage

    def summary(self) -> list[dict]:
        out = []
        flat = self.tau[0]
        for k, lab in enumerate(self.labels):
            t = self.tau[k]
            ok = np.isfinite(t)
            rec = {"ensemble": lab, "mean_tau": float(np.mean(t[ok])) if ok.any() else math.inf,
                   "median_tau": float(np.median(t[ok])) if ok.any() else math.inf,
                   "without_rt": int((~ok).sum()), "requeued": int(self.requeue[k].sum())}
            both = ok & np.isfinite(flat)
            if k > 0 and both.sum() >= 3:
                r, err = analysis.jackknife(t[both], flat[both], np.mean)
                rec["tau_over_flat"], rec["tau_over_flat_err"] = float(r), float(err)
            out.append(rec)
        return out

    def best(self) -> dict:
        rows = [r for r in self.summary() if r["ensemble"].startswith("pl")]
        return min(rows, key=lambda r: r.get("tau_over_flat", math.inf))

    def table_one(self, pt_tau=None, pt_below_eg=None, pl_label: str = "pl(-3.6,96)", eps: float = 1e-4,
                  n_blocks: int = 16) -> dict:
        """Table I of the paper on these realizations: for flat MUCA, the 1/k ensemble and (when
        given) PT, r_pop and r_eps = ratio of the method's population / quantile mean round-trip
        time to the power-law ensemble's, with jackknife errors.  Realizations where any method
        found an energy below E_g are left out (the paper requeues them until none does), as are
        realizations without a round trip in the method or in the power-law ensemble."""
        k_pl = self.labels.index(pl_label)
        bad = self.requeue.any(axis=0)
        if pt_below_eg is not None:
            bad = bad | np.asarray(pt_below_eg, dtype=bool)
        out = {"excluded_below_eg": int(bad.sum()), "reference": pl_label, "eps": eps}
        methods = [(lab, self.tau[self.labels.index(lab)]) for lab in ("flat", "1/k") if lab in self.labels]
        if pt_tau is not None:
            methods.append(("PT", np.asarray(pt_tau, dtype=float)))
        for lab, tau in methods:
            a, b = tau[~bad], self.tau[k_pl][~bad]
            ok = np.isfinite(a) & np.isfinite(b)
            if ok.sum() < 8:
                out[lab] = {"pairs": int(ok.sum())}
                continue
            out[lab] = analysis.relative_performance(a, b, eps=eps, n_blocks=n_blocks)
        return out


def pt_round_trips(dim: int, L: int, n_real: int, M: int, e_g, seed: int = 0, rid0: int = 0,
                   beta_min: float = 0.3, beta_max: float = 2.15, windows: int = 8, window: int = 1000,
                   prod_sweeps: int = 20000, stream=None):
    """PT on the same realizations (Sec. II, PT: M replicas, constant exchange rates imposed on each
    realization during equilibration by moving its temperatures; T_max = 1 / beta_min > 3).  The
    round trip runs between E_g (bottom, given per realization: the MUCA stage's lowest energy)
    and E_hot, the mean energy at the hottest temperature over the equilibration (an energy
    typical of a temperature well above freezing, Sec. III), per replica.  A realization's time
    pools its replicas: tau_i = sum over replicas of (t_last - t_first) / sum of round trips.
    Returns (tau [n_real] (inf: no round trip), below_eg [n_real]: a replica went below E_g)."""
    from .workloads import geometric_betas
    ctx = eamc.Context(seed=seed, stream=stream)
    try:
        ctx.pt_init(dim, L, n_real, geometric_betas(M, beta_min, beta_max), rid0=rid0)
        hot = []
        for w in range(windows):
            for _ in range(10):
                ctx.pt_run(window // 10)
                _, E, _, _ = ctx.pt_state(spins=False)
                hot.append(E[:, 0].astype(np.int64))
            ctx.pt_adapt(0.5)
        e_hot = np.floor(np.mean(hot, axis=0)).astype(np.int32)
        e_g = np.ascontiguousarray(e_g, dtype=np.int32)
        ctx.pt_roundtrips(reset=True)
        ctx.pt_set_rt_bounds(e_g, e_hot)
        ctx.pt_run(prod_sweeps, count_roundtrips=True)
        recs = ctx.pt_roundtrips()
    finally:
        ctx.close()
    tau = np.full(n_real, math.inf)
    below = np.zeros(n_real, dtype=bool)
    for r, reps in enumerate(recs):
        n = sum(x["n_rt"] for x in reps)
        span = sum(x["t_last"] - x["t_first"] for x in reps if x["n_rt"] > 0)
        if n > 0:
            tau[r] = span / n
        below[r] = min(x["e_min"] for x in reps) < e_g[r]
    return tau, below


def profile_scan(dim: int, L: int, n_real: int, alphas, poles, seed: int = 0, rid0: int = 0,
                 dos_iters: int = 30, dos_sweeps: int = 2000, recursion: int = eamc.EA_REC_BERG,
                 dos_alpha: float = -3.6, dos_pole: float = 96.0, prod_sweeps: int = 20000,
                 with_one_over_k: bool = True, stream=None, tile_width: int = 32,
                 order: int = 0) -> ScanResult:
    """Runs the three stages above for every (alpha, Delta E) in alphas x poles (tile_width:
    chains per tile, see muca_set_tile_width; order: the sites' order within a sweep,
    muca_set_sweep_order, for every stage)."""
    ctx = eamc.Context(seed=seed, stream=stream)
    try:
        ctx.set_sweep_order(order)
        if tile_width != 32:
            ctx.set_tile_width(L, tile_width)
        # 1. density of states (power-law target, stream 0)
        dos = ctx.init_disorder(dim, L, n_real, rid0=rid0, stream=0)
        ctx.set_ensemble(dos, n_real, eamc.EA_POWERLAW, dos_alpha, dos_pole)
        ctx.set_recursion(dos, n_real, recursion)
        for _ in range(dos_iters):
            ctx.run_sweeps(dos_sweeps)
            ctx.update_weights()
        ctx.set_eg(dos, n_real, None)
        # 2. one chain per realization and ensemble, each on its own random stream
        params = [(eamc.EA_FLAT, 0.0, 0.0)] + [(eamc.EA_POWERLAW, a, p) for a in alphas for p in poles]
        labels = ["flat"] + [f"pl({a:g},{p:g})" for _, a, p in params[1:]]
        if with_one_over_k:
            params.append((eamc.EA_ONE_OVER_K, 0.0, 0.0))
            labels.append("1/k")
        firsts = [ctx.init_disorder(dim, L, n_real, rid0=rid0, stream=1 + j) for j in range(len(params))]
        src = np.concatenate([np.arange(dos, dos + n_real)] * len(firsts)).astype(np.int32)
        dst = np.concatenate([np.arange(f, f + n_real) for f in firsts]).astype(np.int32)
        ctx.copy_weights(src, dst)
        for (kind, a, p), f in zip(params, firsts):
            ctx.build_ensemble(f, n_real, kind, alpha=a if kind == eamc.EA_POWERLAW else dos_alpha,
                               pole=p if kind == eamc.EA_POWERLAW else dos_pole)
        # the production chains start their clocks now
        ctx.roundtrips(reset=True)
        # 3. production
        ctx.run_sweeps(prod_sweeps, count_roundtrips=True)
        R = ctx.roundtrips()
        E = len(firsts)
        tau = np.full((E, n_real), math.inf)
        nrt = np.zeros((E, n_real), dtype=np.int64)
        req = np.zeros((E, n_real), dtype=bool)
        for k, f in enumerate(firsts):
            for r in range(n_real):
                rec = R[f + r]
                nrt[k, r] = rec["n_rt"]
                req[k, r] = bool(rec["requeue"])
                if rec["n_rt"] > 0:
                    tau[k, r] = (rec["t_last"] - rec["t_first"]) / rec["n_rt"]
        e_g = np.array([R[dos + r]["e_g"] for r in range(n_real)])
        return ScanResult(labels, params, tau, nrt, req, e_g)
    finally:
        ctx.close()
