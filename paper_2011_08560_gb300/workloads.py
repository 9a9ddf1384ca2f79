"""Seeded synthetic workloads (sizes, seeds, realization ids) shared by tests and bench.

Holds none of the Monte Carlo arithmetic: every random number of the method is drawn by
the CUDA library and, independently, by the oracle from the same counter-based Philox
definition, keyed by the seeds below.  The paper's own disorder sets are not available;
seeded +-J disorder (couplings +-1 with p = 1/2, Sec. II) is an exact distributional
stand-in for them.
"""
from dataclasses import dataclass, field


@dataclass(frozen=True)
class MucaWorkload:
    name: str
    dim: int
    L: int
    n_real: int
    seed: int
    ensembles: tuple = ("flat",)
    alpha: float = -3.6          # paper's best power-law exponent (Sec. II)
    pole: float = 96.0           # paper's best pole offset Delta E (Sec. II)
    sweeps: int = 10_000         # sweeps per timed step
    # weight iteration before production: iter_steps updates after iter_sweeps sweeps each,
    # with Berg's accumulated recursion ("berg") or the plain step ("plain")
    iter_steps: int = 0
    iter_sweeps: int = 0
    recursion: str = "berg"
    prod_sweeps: int = 0
    # order of the attempts within a sweep: "lex" (lexicographic) or "colour" (colour class by
    # colour class, the checkerboard for even L); the paper fixes none
    order: str = "lex"


# L=4, one realization, flat MUCA: 20 x 10^4 iteration sweeps, then 10^5 production sweeps;
# the small case the oracle finishes in seconds
SMALL = MucaWorkload("3D +-J EA L=4, 1 realization (seed 1), flat MUCA, 20 x 10^4 iteration + "
                     "10^5 production sweeps", 3, 4, 1, seed=1, iter_steps=20, iter_sweeps=10_000,
                     recursion="plain", prod_sweeps=100_000)

# the headline: L=8, 1024 realizations, power-law MUCA (alpha = -3.6, Delta E = 96); weights
# from Berg's recursion, then E_g fixed and round trips counted in production sweeps; sites in
# the checkerboard order
HEADLINE = MucaWorkload("3D +-J EA L=8, 1024 realizations, power-law MUCA (alpha=-3.6, "
                        "Delta E=96), production with frozen weights, checkerboard sweeps", 3, 8,
                        1024, seed=2, ensembles=("powerlaw",), sweeps=10_000, iter_steps=60,
                        iter_sweeps=10_000, recursion="berg", order="colour")

# L=6, 1024 realizations, flat MUCA beside the power-law ensemble (2048 chains)
L6_FLAT_PL = MucaWorkload("3D +-J EA L=6, 1024 realizations, flat MUCA + power-law MUCA", 3, 6,
                          1024, seed=2, ensembles=("flat", "powerlaw"))

# PT baseline: L=8, 1024 realizations x 32 temperatures, geometric beta in [0.2, 3.0]
PT = dict(dim=3, L=8, n_real=1024, M=32, beta_min=0.2, beta_max=3.0, seed=3)

# batched uneven: 4096 realizations, L uniform over {4,6,8,10,12} by id (round robin)
UNEVEN = dict(dim=3, Ls=(4, 6, 8, 10, 12), n_real=4096, seed=4)

# serving: Poisson arrivals, L in {4..12}, round-trip targets log-uniform in [10, 1000]
SERVING = dict(rate_hz=200.0, Ls=(4, 5, 6, 7, 8, 9, 10, 11, 12), rt_min=10, rt_max=1000, seed=5)


def order_code(order: str) -> int:
    """The library's sweep-order constant (EA_ORDER_LEX 0, EA_ORDER_COLOUR 1) of a workload."""
    return {"lex": 0, "colour": 1}[order]


def geometric_betas(M: int, beta_min: float, beta_max: float):
    """beta_k = beta_min (beta_max/beta_min)^(k/(M-1)), slot 0 hottest."""
    return [beta_min * (beta_max / beta_min) ** (k / (M - 1)) for k in range(M)]
