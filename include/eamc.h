/*
 * eamc.h -- C ABI of the GB300 library for generalized-ensemble Monte Carlo on the
 * bimodal (+-J) Edwards-Anderson spin glass (Mueller, Schnabel, Janke,
 * "Nonflat Histogram Techniques for Spin Glasses", arXiv:2011.08560).
 *
 * Model (Sec. II, Eq. "hamiltonian"): H = -sum_<ij> J_ij S_i S_j on an L^dim periodic
 * simple-cubic lattice (dim = 3; dim = 2 is accepted for small test lattices), with 3V
 * quenched couplings J = +-1 drawn with probability 1/2.
 *
 * Conventions shared by every entry point
 *   - A context owns a batch of independent MUCA chains.  A chain is one disorder
 *     realization (id `rid`) with one random stream (`stream`); two chains with the same
 *     rid share their couplings.  Chains are numbered 0..ea_num_chains()-1 in the order
 *     they were added.
 *   - Site i = x + L*y (+ L*L*z); bond (i,d) joins i and i+e_d; per-bond arrays use
 *     index i*dim + d.  Spins and couplings cross the ABI as int8 +1/-1.
 *   - Energies are integers: E = 2u - dim*V with u the number of unsatisfied bonds.  The
 *     bin of E is b = u >> 1 (u's parity is fixed per realization).  E_top is the largest
 *     attainable E <= 0 ("E approx 0", Sec. III) and b_top its bin; MUCA chains stay at
 *     E <= E_top (hard wall).
 *   - Weights are ln W(b) in FP64, b = 0..b_top.  Acceptance thresholds are uint32:
 *     thr[b*8 + n] is used for a move from bin b at a site with n unsatisfied bonds
 *     (the move changes E by 2*(2*dim) - 4n); EA_ALWAYS accepts unconditionally, any
 *     other value accepts iff the move's 32-bit random word r < thr.
 *   - Random words come from Philox4x32-10 keyed by the context seed.  The MUCA update of
 *     site (x, row) in sweep t uses word x&3 of counter (4*row + x/4, t, rid, stream<<8),
 *     row = y (+ L*z), so a chain's trajectory does not depend on which other chains share
 *     the batch.
 *   - All pointers in this header are HOST pointers to caller-owned buffers unless stated
 *     otherwise; inputs are copied before the call returns, outputs are written before it
 *     returns.  Device state lives in the context until ea_destroy.
 *   - Every int-returning function returns EA_OK (0) or a negative EA_E* code and never
 *     aborts; ea_last_error() gives the calling thread's last message.  A context is not
 *     thread-safe: use one context per host thread / stream.
 */
#ifndef EAMC_H
#define EAMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EA_OK 0
#define EA_EINVAL (-1)   /* bad argument (size, range, null pointer) */
#define EA_ENOMEM (-2)   /* device or host allocation failed */
#define EA_ECUDA (-3)    /* a CUDA call failed; message in ea_last_error() */
#define EA_ETIMEOUT (-4) /* a bounded device wait gave up */
#define EA_ESTATE (-5)   /* call not valid in the context's current state */

#define EA_ALWAYS 0xFFFFFFFFu

/* ensemble kinds */
#define EA_FLAT 0       /* W ~ 1/Omega (Eq. "muca-weights") */
#define EA_POWERLAW 1   /* W ~ P_SH/Omega, P_SH of Eq. "power_law" */
#define EA_ONE_OVER_K 2 /* W ~ 1/k, k(E) = sum_{E_g<=E'<=E} Omega(E') (Eq. "1/k") */
#define EA_CANON 3      /* W = exp(-beta E) (textbook Metropolis) */

/* weight recursions (muca_set_recursion) */
#define EA_REC_PLAIN 0  /* the plain step of muca_update_weights */
#define EA_REC_BERG 1   /* Berg's accumulated error-weighted recursion */

typedef struct ea_ctx ea_ctx;

/* Round-trip record of one chain (Sec. III).  phase: 0 = waiting for the first visit of
 * E_top, 1 = heading down to E_g, 2 = heading up to E_top.  A round trip completes at each
 * top visit after a bottom visit.  t_first / t_last are sweep indices of the first top
 * visit and of the last completed round trip (-1 if none); tau = (t_last-t_first)/n_rt.
 * e_min is the lowest energy seen; requeue is set when e_min < e_g while counting
 * (the paper's requeue on a lower energy, Sec. III). */
typedef struct {
    int32_t phase, n_rt;
    int64_t t_first, t_last;
    int32_t e_min, e_g;
    int32_t requeue, pad;
} ea_rt_stats;

/* Static description of one chain. */
typedef struct {
    int32_t dim, L, b_top, parity; /* parity of u */
    uint32_t rid, stream;
    int32_t E, kind;                /* current energy, ensemble kind */
    uint64_t t;                     /* sweeps done */
} ea_chain_desc;

const char *ea_last_error(void);

/* Creates a context on CUDA device `device`; all work is queued on `cuda_stream` (a
 * cudaStream_t, may be NULL for the legacy default stream; e.g. torch's current stream).
 * `seed` keys every random word of the context.  *out receives the context. */
int ea_create(ea_ctx **out, int device, void *cuda_stream, uint64_t seed);
void ea_destroy(ea_ctx *ctx);

/* a1 -- disorder and initial state (Sec. II: 3V couplings J = +-1 with p = 1/2, quenched).
 * Appends n chains of linear size L (dim 2 or 3, 3 <= L <= 12) for realizations
 * rid0, rid0+1, ... with random stream `stream`.  couplings_or_null: NULL to draw the
 * couplings from the seed, else int8[n][dim*V] of +-1.  spins_or_null: NULL for random
 * initial spins, else int8[n][V] of +-1.  Each chain then descends deterministically
 * (lexicographic sweeps flipping spins that lower E) until E <= E_top.  Weights start at
 * ln W = 0 (flat), ensemble EA_FLAT.  *first_chain (may be NULL) receives the index of the
 * first new chain.  Returns EA_ESTATE if a descent gets stuck above E_top. */
int ea_init_disorder(ea_ctx *ctx, int dim, int L, int n, uint32_t rid0, uint32_t stream,
                     const int8_t *couplings_or_null, const int8_t *spins_or_null,
                     int *first_chain);

int ea_num_chains(const ea_ctx *ctx);
int ea_describe(ea_ctx *ctx, int chain0, int n, ea_chain_desc *out);

/* a5 -- ensemble parameters of chains chain0..chain0+n-1: kind (EA_FLAT, EA_POWERLAW,
 * EA_ONE_OVER_K, EA_CANON), power-law exponent alpha and pole offset pole_dE (Eq.
 * "power_law", the paper's best values are -3.6 and 96), inverse temperature beta (canon).
 * Only records the parameters used by muca_update_weights / muca_build_ensemble. */
int muca_set_ensemble(ea_ctx *ctx, int chain0, int n, int kind, double alpha,
                      double pole_dE, double beta);

/* ln W input/output: lnW[c*stride + b] for chain c of the range, b = 0..b_top(c); stride
 * >= the largest b_top+1 of the range.  set re-quantises the thresholds on the device. */
int muca_set_weights(ea_ctx *ctx, int chain0, int n, const double *lnW, int stride);
int muca_get_weights(ea_ctx *ctx, int chain0, int n, double *lnW, int stride);

/* Thresholds input/output: thr[c*stride + b*8 + k], stride >= 8*(b_top+1).  set injects a
 * table verbatim (parity testing); the next muca_set_weights / muca_update_weights /
 * muca_build_ensemble overwrites it. */
int muca_set_thresholds(ea_ctx *ctx, int chain0, int n, const uint32_t *thr, int stride);
int muca_get_thresholds(ea_ctx *ctx, int chain0, int n, uint32_t *thr, int stride);

/* Lowest-energy reference E_g per chain (bottom of a round trip, pole of the profile).
 * e_g NULL takes each chain's lowest energy seen so far. */
int muca_set_eg(ea_ctx *ctx, int chain0, int n, const int32_t *e_g);

/* a2 + a3 -- n_sweeps sweeps of single-spin-flip generalized Metropolis (Eq. "muca",
 * P_acc = min(1, W(E_new)/W(E_old))), sites in lexicographic order, for every chain of
 * the context.  After every attempt: lowest-energy update and, if count_roundtrips, one
 * round-trip check against E_top and E_g.  After every sweep: H(bin(E)) += 1.  Requires
 * t + n_sweeps <= 2^32 for every chain.  Asynchronous on the context stream. */
int muca_run_sweeps(ea_ctx *ctx, uint64_t n_sweeps, int count_roundtrips);

/* a8 -- launch configuration of muca_run_sweeps.  persistent = 0: one thread block per tile;
 * persistent = 1: a grid of blocks_per_sm blocks per SM (0 = as
 * many as fit) whose blocks pull tiles from a work queue, longest lattices first (for batches
 * of uneven L).  sweeps_per_launch > 0 splits a run into launches of at most that many
 * sweeps (0 = one launch).  Results do not depend on any of these settings. */
int muca_set_launch(ea_ctx *ctx, int persistent, uint64_t sweeps_per_launch, int blocks_per_sm);

/* sweep orders (muca_set_sweep_order) */
#define EA_ORDER_LEX 0     /* sites in lexicographic order */
#define EA_ORDER_COLOUR 1  /* colour class by colour class, each class in lexicographic order */

/* a2 -- the order of the attempts within a sweep for every chain of the context (the paper fixes
 * none; any fixed order samples the same ensemble, but trajectories differ):
 *   EA_ORDER_LEX (default): i = 0 .. V-1; random word of site (x, row): word x&3 of Philox call
 *   (4 row + x/4, t, rid, stream << 8);
 *   EA_ORDER_COLOUR: the colour classes of the PT sweep one after the other (the checkerboard,
 *   even coordinate sum first, for even L; for odd L colour (c(x)+c(y)+c(z)) mod 3 with
 *   c(x) = x mod 3 except c(L-1) = 1 when L = 1 (mod 3)), each in lexicographic order; the
 *   j-th colour-c site of a row takes word j&3 of call (4 row + j/4, t, rid, (5 + c) | stream << 8).
 *   No two sites of a class are neighbours, so each attempt's class is fixed when its class
 *   begins.  One kernel runs it for every L, one lane per chain in the tiles of the lexicographic
 *   kernel (the tile widths of muca_set_tile_width apply; odd L has three colour passes and
 *   rows with different numbers of colour sites, padded with attempts that move nothing): one
 *   candidate-threshold pair per attempt instead of two classes' worth, the faster order for
 *   L <= 8.
 * chains_per_cta: 0 or one of 1, 2, 4, 8 (kept for callers of an earlier form of this call; it
 * has no effect).  Applies from the next muca_run_sweeps or graph capture; the order is not part
 * of a snapshot.  EA_EINVAL for an unknown order or count. */
int muca_set_sweep_order(ea_ctx *ctx, int order, int chains_per_cta);

/* a8 -- chains per tile for chains of linear size L added afterwards (ea_init_disorder):
 * width 32 (the default, every L), 16 (3D, L = 7, 8), or, for chains swept in the colour order
 * only, 16 (3D, L = 4, 5, 6), 8 (3D, L = 4..10) and 4 (3D, L = 11, 12); muca_run_sweeps in the
 * lexicographic order refuses tiles of a width that kernel lacks (EA_EINVAL).  A tile is one
 * warp; with width W < 32 each of its W chains runs on 32/W lanes side by side, so the tile needs
 * W/32 of the shared memory of a full one: at L >= 7 the acceptance thresholds then fit in shared
 * memory instead of being read through L1, and at every L a batch spreads over more SMs with less
 * producer work on each; each chain runs faster, the SM holds fewer chains.  Narrow tiles suit
 * batches with fewer chains than the GPU can hold; results do not depend on the width.
 * EA_EINVAL for a width not available at this L. */
int muca_set_tile_width(ea_ctx *ctx, int L, int width);

/* Properties of the sweep kernel for tiles of (dim, L, width): dynamic shared memory per block
 * (*smem_bytes, may be NULL) and whether the thresholds live in shared memory
 * (*thresholds_in_smem, may be NULL).  EA_EINVAL for a width not available at this L. */
int muca_get_tile_width(int dim, int L, int width, size_t *smem_bytes, int *thresholds_in_smem);
/* The same for the colour-order kernel (muca_set_sweep_order). */
int muca_get_tile_width_colour(int dim, int L, int width, size_t *smem_bytes, int *thresholds_in_smem);

/* a8 / a9 -- every tile of linear size L runs multiplier x the requested sweeps in each
 * muca_run_sweeps call (default 1), so a launch over tiles of uneven L can give small lattices
 * proportionally more sweeps.  A chain's trajectory depends only on its own sweep count. */
int muca_set_sweep_multiplier(ea_ctx *ctx, int L, int multiplier);

/* a8 -- captures n_iter iterations of [muca_run_sweeps(sweeps_per_iter, count_roundtrips),
 * then muca_update_weights if update_weights] into a CUDA graph on the context stream (which
 * must not be the legacy default stream).  ea_graph_launch replays it; ea_graph_release
 * frees it.  Replays see the launch configuration at capture time.  Adding chains
 * (ea_init_disorder), loading a snapshot and the first EA_REC_BERG recursion release the graph
 * (the arenas it points into may move); ea_graph_launch then returns EA_ESTATE. */
int ea_graph_capture(ea_ctx *ctx, int n_iter, uint64_t sweeps_per_iter, int count_roundtrips,
                     int update_weights);
int ea_graph_launch(ea_ctx *ctx, int replays);
int ea_graph_release(ea_ctx *ctx);

/* a4 -- one step of the weight iteration (Sec. II, iterative procedure after Janke 2003,
 * with shaped histograms): ln W <- ln W + ln P_SH(E) - ln max(H(E), 1), shifted to 0 at
 * b_top, with P_SH from the chain's kind (flat: 1, power law: Eq. "power_law" with E_g =
 * lowest energy seen).  E_g is updated to that energy, the histogram is cleared and the
 * thresholds are re-quantised.  Chains of kind EA_ONE_OVER_K / EA_CANON are untouched. */
int muca_update_weights(ea_ctx *ctx);

/* f1 -- chooses the weight recursion of chains chain0..chain0+n-1 (mode EA_REC_PLAIN or
 * EA_REC_BERG) and empties their accumulators.  EA_REC_BERG is Berg's accumulated form
 * (B. A. Berg, J. Stat. Phys. 82, 323 (1996); one of the iterative procedures collected in
 * Janke 2003, which Sec. II refers to): for each pair of neighbouring bins (b, b+1) visited in
 * an iteration, s = [ln H(b+1) - ln W(b+1)] - [ln H(b) - ln W(b)] estimates
 * ln Omega(b+1) - ln Omega(b) with inverse Poisson variance g = H(b)H(b+1)/(H(b)+H(b+1)); the
 * chain keeps D(b) (the g-weighted mean of all its estimates) and G(b) (the sum of the g), and
 * muca_update_weights then sets ln W(b) - ln W(b+1) = ln P_SH(b) - ln P_SH(b+1) + D(b) where
 * G(b) > 0 and the plain step's difference elsewhere, ln W(b_top) = 0.  A pair of which an
 * iteration visited exactly one bin, although D predicted at least 10 counts on the other
 * (H(visited) Omega W ratio >= 10), starts over (D = G = 0): weights that confine the chain to
 * one side of a pair would otherwise never be corrected.  An iteration run with
 * weights that are constant over the range adds no estimates (every move inside the range is
 * then accepted, so the sequential sweep is deterministic).  The first EA_REC_BERG call of a
 * context allocates 16 bytes per bin of every chain and releases a captured graph.
 * EA_EINVAL: bad range or mode; EA_ENOMEM: allocation failed. */
int muca_set_recursion(ea_ctx *ctx, int chain0, int n, int mode);

/* Berg accumulators of chains chain0..: out[c*stride + 2b] = D(b), out[c*stride + 2b + 1] = G(b)
 * for b = 0..b_top(c) (host buffer; stride in doubles, >= 2 (b_top+1); the entry at b_top is
 * unused and 0).  EA_ESTATE if no chain of the context ever used EA_REC_BERG. */
int muca_get_recursion_state(ea_ctx *ctx, int chain0, int n, double *out, int stride);

/* a5 -- rebuilds ln W of chains chain0..chain0+n-1 for a new ensemble from the density of
 * states implied by the current weights (ln Omega = ln P_SH(current kind) - ln W), see
 * EA_FLAT..EA_CANON, then re-quantises.  The new kind and parameters are recorded. */
int muca_build_ensemble(ea_ctx *ctx, int chain0, int n, int kind, double alpha,
                        double pole_dE, double beta);

/* a9 -- serving support.  Re-initialises the listed chains (host int32 chain indices)
 * in place as new jobs: realization rids[k] with stream streams[k] (host uint32 arrays),
 * couplings and spins drawn from the seed, deterministic descent to E <= E_top, flat weights,
 * kind EA_FLAT, recursion EA_REC_PLAIN, sweep counter 0, cleared histogram and round trips.  The chain keeps its L.
 * Other chains of the context are untouched, so their trajectories do not change. */
int ea_reset_chains(ea_ctx *ctx, const int32_t *chains, int n, const uint32_t *rids,
                    const uint32_t *streams);

/* f4 -- for k < n, chain dst[k] takes chain src[k]'s ln W row, ensemble (kind, alpha, pole,
 * beta) and E_g, then thresholds are re-quantised; the chains' lattices, histograms and
 * round-trip records stay.  Serves the profile scan: a density of states estimated once per
 * realization (Sec. II: determined once, then shared by the ensembles compared) is copied to
 * chains of the same realization that then build other ensembles (muca_build_ensemble).
 * Host int32 lists; pairs must share L and b_top; a chain may not be a destination twice nor
 * both a source and a destination (EA_EINVAL). */
int muca_copy_weights(ea_ctx *ctx, const int32_t *src, const int32_t *dst, int n);

/* a4 for the listed chains only (host int32 chain indices); see muca_update_weights. */
int muca_update_weights_subset(ea_ctx *ctx, const int32_t *chains, int n);

/* Histograms H[c*stride + b], b = 0..b_top(c); reset != 0 clears them afterwards. */
int get_histograms(ea_ctx *ctx, int chain0, int n, uint32_t *out, int stride, int reset);

/* Round-trip records; reset != 0 restarts counting (phase 0, n_rt 0, e_min = E). */
int get_roundtrips(ea_ctx *ctx, int chain0, int n, ea_rt_stats *out, int reset);

/* Spins spins[c*stride + i] (+-1, may be NULL), energies E[c] (may be NULL), sweeps t[c]
 * (may be NULL). */
int get_state(ea_ctx *ctx, int chain0, int n, int8_t *spins, int stride, int32_t *E,
              uint64_t *t);

/* Checkpoint / resume (not in the paper; random words are keyed by each chain's sweep
 * counter, so a run resumed from a snapshot continues the identical trajectory).  size gives
 * the snapshot's byte count; save writes the MUCA state of every chain (lattices, chain
 * states, weights, histograms, thresholds, Berg accumulators, launch layout, seed) into a host
 * buffer of at least
 * that size; load restores it into a context that has no chains yet (PT state and the launch
 * configuration are not part of a snapshot). */
int ea_snapshot_size(ea_ctx *ctx, size_t *bytes);
int ea_snapshot_save(ea_ctx *ctx, void *buf, size_t cap);
int ea_snapshot_load(ea_ctx *ctx, const void *buf, size_t size);

/* Invariant check (the role a sanitizer would have; not in the paper): while sweeping, the
 * kernel checks off the critical path that every chain's energy stays inside its range
 * [E_min of the table, E_top], i.e. its bin inside [0, b_top].  Waits for the context's work,
 * returns EA_ESTATE (message in ea_last_error) if a check failed since the last call, EA_OK
 * otherwise, and clears the record. */
int ea_check(ea_ctx *ctx);

/* Waits for all queued work of the context. */
int ea_synchronize(ea_ctx *ctx);

/* ------------------------------------------------------------------ parallel tempering
 * a6 + a7 -- the paper's PT baseline (Sec. II, PT; Eq. "temperatureexchange"): M replicas of
 * each realization, Metropolis at inverse temperatures beta_0 < ... < beta_{M-1} (slot 0
 * hottest), exchanges between neighbouring slots.  A context holds one PT batch beside its
 * MUCA chains. */

/* Round-trip record of one PT replica (Sec. III, PT variant: between E_g and E_hot). */
typedef struct {
    int32_t n_rt, phase;
    int64_t t_first, t_last;
    int32_t e_min, pad;
} ea_pt_stats;

/* Sets up n_real realizations rid0 .. rid0+n_real-1 (rid0 a multiple of 32; realizations
 * are packed 32 to a word) of lattices of linear size L (3 <= L <= 12) with M replicas
 * (2 <= M <= 64), every realization at host betas[M] (strictly increasing; pt_set_betas gives
 * each realization its own set).  Couplings from the seed (as ea_init_disorder) or from
 * couplings_or_null (int8[n_real][dim*V]); replica k of realization r starts from the random
 * spins of stream k.  Metropolis thresholds floor(exp(-beta_k dE) 2^32) are built on the
 * device; exchange thresholds floor(exp(-(beta_{k+1}-beta_k) 4d) 2^32) are evaluated there at
 * each exchange.  Replaces any previous PT batch of the context. */
int pt_init(ea_ctx *ctx, int dim, int L, int n_real, uint32_t rid0, int M, const double *betas,
            const int8_t *couplings_or_null);

/* Round-trip bounds per realization (host int32[n_real] each): bottom E_g, top E_hot. */
int pt_set_rt_bounds(ea_ctx *ctx, const int32_t *e_g, const int32_t *e_hot);

/* n_sweeps PT sweeps: per sweep, a Metropolis sweep of every replica colour class by colour
 * class, each class in lexicographic order -- even L: the checkerboard (even coordinate sum
 * first); odd L, where the checkerboard is not a proper colouring under periodic boundaries:
 * colour (c(x) + c(y) + c(z)) mod 3 with c(x) = x mod 3, except c(L-1) = 1 when L = 1 (mod 3)
 * -- then exchanges between slots
 * (k, k+1) for k = t mod 2, t mod 2 + 2, ... (accepted if E_{k+1} >= E_k, else with
 * probability exp((beta_{k+1}-beta_k)(E_{k+1}-E_k))), then, if count_roundtrips, one
 * round-trip check per replica.  The random word of an uphill update of realization r at
 * slot k, site i, sweep t has bit 31-m equal to bit r&31 of word m&3 of Philox counter
 * (8i + m/4, t, r>>5, 4 | k<<8); the exchange (k, k+1) uses word 0 of (k, t, r, 1). */
int pt_run(ea_ctx *ctx, uint64_t n_sweeps, int count_roundtrips);

/* State by slot: spins int8[n_real][M][V] (may be NULL), energies int32[n_real][M] (may be
 * NULL), replica labels int32[n_real][M] (may be NULL; label = the slot a configuration
 * started at), sweeps done (may be NULL). */
int pt_get_state(ea_ctx *ctx, int8_t *spins, int32_t *E, int32_t *labels, uint64_t *t);

/* Round-trip records by replica label, out[n_real][M]; reset restarts counting. */
int pt_get_roundtrips(ea_ctx *ctx, ea_pt_stats *out, int reset);

/* Accepted exchanges per slot pair (k, k+1), summed over realizations: uint64[M-1]. */
int pt_get_swap_counts(ea_ctx *ctx, uint64_t *out);

/* f2 -- the paper's PT protocol (Sec. II, PT): constant exchange rates imposed on every
 * realization during equilibration by moving its temperatures.
 * pt_set_betas / pt_get_betas: per-realization inverse temperatures, host double[n_real][M],
 * each row strictly increasing (EA_EINVAL otherwise); setting rebuilds the thresholds.
 * pt_get_exchange_counts: since pt_init or the last pt_adapt, accepted exchanges of pair
 * (k, k+1) per realization (uint32[n_real][M-1], may be NULL) and the attempts per pair, the
 * same for every realization (uint64[M-1], may be NULL: pair k is tried at sweeps t = k mod 2).
 * pt_adapt: one adaptation step per realization from those counts, then a new count window.
 * Rate A_k = accepted / attempts clamped to [0.005, 0.995], gap D_k = beta_{k+1} - beta_k,
 * stiffness s_k = -ln(A_k) / D_k; the gaps that give every pair the same rate are
 * D*_k = (beta_{M-1} - beta_0) (1/s_k) / sum_j (1/s_j); the new gaps are
 * (1 - eta) D_k + eta D*_k (0 <= eta <= 1) with beta_0 and beta_{M-1} fixed.  A realization
 * whose window holds a pair without attempts keeps its temperatures. */
int pt_set_betas(ea_ctx *ctx, const double *betas);
int pt_get_betas(ea_ctx *ctx, double *betas);
int pt_get_exchange_counts(ea_ctx *ctx, uint32_t *accepted, uint64_t *attempted);
int pt_adapt(ea_ctx *ctx, double eta);

/* ------------------------------------------------------------------ serving
 * a9 -- continuous batching of realization jobs (Sec. II ensembles, Sec. III round trips and
 * requeue).  A server owns one context whose tiles form a pool of lanes per lattice size; jobs
 * are admitted into free lanes (the pool of an L grows while the memory budget allows: admission
 * by memory), and all jobs advance together, one tick after another: a sweep launch over every
 * tile, then per-slot job control on the device (weight steps at each job's step boundaries,
 * the switch to production, requeue, completion).  The host never waits for a tick: finished
 * jobs are read back asynchronously every poll_ticks ticks.  A job's schedule is counted in its
 * own ticks and its random numbers are keyed by its own sweep counter, so its result is the same
 * alone and among other jobs.  Served chains sweep in the configured order (sweep_order).  A
 * server is not thread-safe. */
typedef struct ea_srv ea_srv;

typedef struct {
    int32_t dim;             /* 3 (2 for small test lattices) */
    int32_t n_L, Ls[16];     /* lattice sizes served, 3 <= L <= 12 */
    size_t mem_budget;       /* device bytes the lane pool may take */
    int32_t base_sweeps;     /* sweeps per tick at the largest L; a lattice of size L gets
                              * base_sweeps * round((L_max / L)^3), about equal work per tick */
    int32_t poll_ticks;      /* ticks between completion read-backs */
    int32_t max_ahead;       /* ticks queued at most beyond the last completed read-back */
    int32_t sweep_order;     /* EA_ORDER_LEX (0) or EA_ORDER_COLOUR (1), see muca_set_sweep_order */
} ea_srv_config;

/* One job: realization rid (couplings and initial spins drawn from the server's seed, as
 * ea_init_disorder), random stream, ensemble kind EA_FLAT or EA_POWERLAW (alpha, pole), weight
 * recursion EA_REC_PLAIN or EA_REC_BERG.  Schedule in the job's own ticks: iter_steps weight
 * steps, one every ticks_per_step ticks; then E_g = the lowest energy seen and production until
 * rt_target round trips (status EA_JOB_DONE) or max_prod_ticks production ticks (EA_JOB_CENSORED);
 * a chain that goes below E_g in production is requeued (new E_g, one more weight step,
 * counting restarts) at most max_requeues times. */
typedef struct {
    int32_t L;
    uint32_t rid, stream;
    int32_t kind, recursion;
    double alpha, pole;
    int32_t rt_target, iter_steps, ticks_per_step, max_prod_ticks, max_requeues, pad;
} ea_job;

#define EA_JOB_DONE 1
#define EA_JOB_CENSORED 2
#define EA_JOB_FAILED 3  /* the chain's descent to E <= E_top got stuck at admission */

/* A finished job: round-trip record of its production (t_first / t_last are sweep indices of
 * the job's own chain, tau = (t_last - t_first) / n_rt), requeues taken, E_g and the lowest
 * energy, sweeps done, and host times in seconds since the server was created: submission,
 * admission into a lane, and the read-back that reported it. */
typedef struct {
    uint64_t job_id;
    int32_t status, L;
    uint32_t rid;
    int32_t rt_target, n_rt, requeues;
    int64_t t_first, t_last;
    int32_t e_g, e_min;
    uint64_t sweeps;
    double t_submit, t_admit, t_done;
} ea_srv_result;

typedef struct {
    uint64_t ticks, ticks_read;       /* ticks queued / covered by the last read-back */
    uint64_t attempts;                /* spin-flip attempts of job lanes (at the last read-back) */
    int32_t queued, running, lanes, pad;
    uint64_t done, censored, failed, cancelled, round_trips;
    size_t mem_used;
    double seconds;                   /* since the server was created */
} ea_srv_counters;

/* Creates a server on CUDA device `device`, queuing all work on cuda_stream (not the legacy
 * default stream if other work shares the device).  EA_EINVAL for a bad configuration. */
int ea_srv_create(ea_srv **out, int device, void *cuda_stream, uint64_t seed, const ea_srv_config *cfg);
void ea_srv_destroy(ea_srv *srv);

/* Queues a job (admitted at the next ea_srv_step); *job_id (may be NULL) receives its id.
 * EA_EINVAL for an L not served, a bad kind / recursion / schedule, or a schedule whose sweeps
 * would exceed 2^32. */
int ea_srv_submit(ea_srv *srv, const ea_job *job, uint64_t *job_id);

/* Withdraws a waiting or running job (a running job's lane stops before the next tick and is
 * reused); EA_ESTATE if the job is neither (unknown or already finished). */
int ea_srv_cancel(ea_srv *srv, uint64_t job_id);

/* Admits waiting jobs into free lanes (growing the pool within the budget), then queues `ticks`
 * ticks (none while no job runs).  Returns without waiting for the GPU, except to keep at most
 * max_ahead ticks in flight. */
int ea_srv_step(ea_srv *srv, int ticks);

/* Copies up to cap finished jobs into out (host buffer) and their count into *n_out.  wait = 0
 * only looks at read-backs that have completed; wait != 0 first reads back everything queued. */
int ea_srv_poll(ea_srv *srv, ea_srv_result *out, int cap, int *n_out, int wait);

int ea_srv_stats(ea_srv *srv, ea_srv_counters *out);

/* Device bytes one tile of 32 lanes of size L takes from a server's memory budget (0 for a bad
 * dim / L). */
size_t ea_srv_tile_bytes(int dim, int L);

/* The server's context (its chains by lane), for inspection; owned by the server. */
int ea_srv_context(ea_srv *srv, ea_ctx **ctx);

/* ------------------------------------------------------------------ no allocation
 * The paper has no counterpart to this entry point: it serves callers that cannot allocate
 * device memory (code inside another framework's memory pool or under a fixed device-memory
 * budget, plugins that may only touch the buffers they are given).  It runs n_sweeps MUCA
 * sweeps (the muca_run_sweeps kernel in the lexicographic order, without round-trip counting) on n chains of linear size
 * L without a context and without allocating anything: no cudaMalloc, no cudaFree, no
 * allocating library call.  Its working memory is one static device array of 4 MiB in the
 * library, which every GPU that loads the library holds until the process exits; at most
 * 256 chains, and fewer at large L (L=8: 256, L=12: about 90) -- larger requests return
 * EA_EINVAL.  The first call on a device looks up the array's device address and should come
 * before any stream capture.  Calls share the array: calls that overlap on the GPU race.
 *
 * All buffers are DEVICE pointers owned by the caller, for chains c = 0..n-1:
 *   rid[c], stream_id[c]       uint32 realization id and random stream (as ea_init_disorder)
 *   couplings[c][dim*V]        int8 +-1 (in)
 *   spins[c][V]                int8 +-1 (in / out); every chain must start with E <= E_top
 *   energies[c]                int32 (out)
 *   thr[c][B][8]               uint32 acceptance thresholds (in), B = (dim*V/2 >> 1) + 1
 *   hist[c][B]                 uint32 histogram (in / out, accumulated)
 * t0 is the sweep index of the first sweep (random words are keyed by it, so two calls with
 * t0 and t0 + n_sweeps continue one trajectory); t0 + n_sweeps <= 2^32.  As in a context, moves
 * out of a chain's range [0, b_top] are rejected whatever thr holds there.  Work is queued on
 * cuda_stream (may be NULL) and the call returns after it completes.  EA_EINVAL if a chain
 * starts above E_top: the call then runs nothing and writes no output buffer, so it may be
 * repeated with the same t0 once the input is fixed. */
int muca_run_sweeps_noalloc(int dim, int L, int n, uint64_t seed, const uint32_t *rid,
                            const uint32_t *stream_id, const int8_t *couplings, int8_t *spins,
                            int32_t *energies, const uint32_t *thr, uint32_t *hist, uint64_t t0,
                            uint64_t n_sweeps, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* EAMC_H */
