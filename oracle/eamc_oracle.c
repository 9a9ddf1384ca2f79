/*
 * eamc_oracle.c -- plain, slow, obviously-correct CPU oracle for generalized-ensemble
 * Monte Carlo on the bimodal (+-J) Edwards-Anderson spin glass.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference legs may load this library.  It shares no code, header,
 * table or constant generator with the CUDA library: it is written from the paper
 * (Mueller, Schnabel, Janke, "Nonflat Histogram Techniques for Spin Glasses") and
 * from the published Philox definition (Salmon, Moraes, Dror, Shaw, SC'11).
 *
 * Spins and couplings are stored as int8 values +1/-1 and every energy change is
 * obtained from the Hamiltonian's definition (Sec. II, Eq. "hamiltonian"):
 *     H = - sum_<ij> J_ij S_i S_j ,
 * on an L^dim simple (hyper)cubic lattice with periodic boundaries.
 *
 * Conventions fixed where the paper is silent (the same readings are implemented,
 * independently, by the CUDA path):
 *   site index   i = x + L*y (+ L*L*z); bond (i,d) joins i and i + e_d (periodic);
 *                J is stored as J[i*dim + d].
 *   energy bins  u = number of unsatisfied bonds, E = 2u - dim*V; u's parity never
 *                changes under single flips, so the bin is b = u >> 1.  E_top is the
 *                largest attainable E <= 0, b_top its bin (hard wall above it).
 *   RNG          Philox4x32-10, key = (seed lo, seed hi).  Counter words:
 *                  disorder      (j>>2, 0, rid, 3)            word j&3, j = bond index
 *                  initial spins (i>>2, 0, rid, 2 | stream<<8) word i&3
 *                  MUCA update   (4*row + x/4, t, rid, 0 | stream<<8) word x&3, where
 *                                row = y (+ L z) is the site's lattice row along x
 *                  MUCA update in the colour order
 *                                (4*row + j/4, t, rid, (5 + c) | stream<<8) word j&3, where
 *                                c is the site's colour and j its rank among the colour-c
 *                                sites of its row (in x order)
 *                  PT update     (8*i + m/4, t, rid>>5, 4 | slot<<8) word m&3,
 *                                32 words whose bit (rid&31) gives bit 31-m of r
 *                  PT swap       (k, t, rid, 1) word 0
 *                A value is "negative" (J=-1, S=-1) iff the word's top bit is set.
 *   acceptance   thr = 0xFFFFFFFF means "always"; otherwise accept iff r < thr
 *                (Eq. "muca": P_acc = min(1, W(E_new)/W(E_old)), quantised to 2^-32).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_ALWAYS 0xFFFFFFFFu

/* ---------------------------------------------------------------- Philox4x32-10 */
/* Salmon et al. (SC'11), Sec. 4.2: the Philox-4x32 S-box multiplies counter words 0
 * and 2 by two odd constants; the high halves are xored with the other counter words
 * and the round key, and the key is bumped by the Weyl constants between rounds. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static uint32_t rand_word(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                          uint32_t c3, int which) {
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    or_philox4x32_10(ctr, key, out);
    return out[which];
}

/* ---------------------------------------------------------------- lattice basics */
int or_volume(int dim, int L) { return dim == 2 ? L * L : L * L * L; }
int or_nbonds(int dim, int L) { return dim * or_volume(dim, L); }

/* neighbour of site i one step along direction d (0=x,1=y,2=z), sign +1 or -1 */
static int neighbour(int dim, int L, int i, int d, int sign) {
    int x = i % L, y = (i / L) % L, z = (dim == 3) ? i / (L * L) : 0;
    int c[3] = {x, y, z};
    c[d] = (c[d] + sign + L) % L;
    return c[0] + L * c[1] + L * L * c[2];
}

/* Quenched disorder (Sec. II): 3V couplings, +1 or -1 with probability 1/2 each. */
void or_make_disorder(int dim, int L, uint64_t seed, uint32_t rid, int8_t *J) {
    int nb = or_nbonds(dim, L);
    for (int j = 0; j < nb; ++j) {
        uint32_t w = rand_word(seed, (uint32_t)(j >> 2), 0u, rid, 3u, j & 3);
        J[j] = (w >> 31) ? -1 : +1;
    }
}

void or_make_spins(int dim, int L, uint64_t seed, uint32_t rid, uint32_t stream, int8_t *S) {
    int V = or_volume(dim, L);
    for (int i = 0; i < V; ++i) {
        uint32_t w = rand_word(seed, (uint32_t)(i >> 2), 0u, rid, 2u | (stream << 8), i & 3);
        S[i] = (w >> 31) ? -1 : +1;
    }
}

/* Eq. "hamiltonian": H = -sum over nearest-neighbour pairs of J_ij S_i S_j. */
int or_energy(int dim, int L, const int8_t *J, const int8_t *S) {
    int V = or_volume(dim, L), E = 0;
    for (int i = 0; i < V; ++i)
        for (int d = 0; d < dim; ++d)
            E -= J[i * dim + d] * S[i] * S[neighbour(dim, L, i, d, +1)];
    return E;
}

/* local field h_i = sum_j J_ij S_j over the 2*dim neighbours of i */
static int local_field(int dim, int L, const int8_t *J, const int8_t *S, int i) {
    int h = 0;
    for (int d = 0; d < dim; ++d) {
        int jp = neighbour(dim, L, i, d, +1);
        int jm = neighbour(dim, L, i, d, -1);
        h += J[i * dim + d] * S[jp];
        h += J[jm * dim + d] * S[jm];
    }
    return h;
}

/* ---------------------------------------------------------------- energy bins */
/* parity of the number of unsatisfied bonds (= parity of #negative couplings) */
int or_parity(int dim, int L, const int8_t *J) {
    int nb = or_nbonds(dim, L), neg = 0;
    for (int j = 0; j < nb; ++j) neg += (J[j] < 0);
    return neg & 1;
}

/* E = 2u - nb  =>  u = (E + nb)/2, bin = u >> 1 */
int or_bin_of_energy(int dim, int L, int E) { return ((E + or_nbonds(dim, L)) / 2) >> 1; }
int or_energy_of_bin(int dim, int L, int parity, int b) {
    return 2 * (2 * b + parity) - or_nbonds(dim, L);
}
/* the largest attainable energy <= 0 ("E approx 0" of Sec. III) and its bin */
int or_btop(int dim, int L, int parity) {
    int uhalf = or_nbonds(dim, L) / 2;
    int utop = ((uhalf & 1) == parity) ? uhalf : uhalf - 1;
    return utop >> 1;
}

/* Deterministic start inside the MUCA range: from the random start, sweep the sites in
 * lexicographic order flipping every spin whose flip lowers E, until E <= e_top. */
int or_descend(int dim, int L, const int8_t *J, int8_t *S, int e_top, int32_t *E_io) {
    int V = or_volume(dim, L), E = *E_io;
    while (E > e_top) {
        int flipped = 0;
        for (int i = 0; i < V && E > e_top; ++i) {
            int dE = 2 * S[i] * local_field(dim, L, J, S, i);
            if (dE < 0) { S[i] = (int8_t)-S[i]; E += dE; flipped = 1; }
        }
        if (!flipped) return -1;
    }
    *E_io = E;
    return 0;
}

/* ---------------------------------------------------------------- round trips */
/* Sec. III: a round trip runs from the top of the energy range to the lowest energy
 * E_g and back.  Phases: 0 = waiting for the first top visit, 1 = heading down,
 * 2 = heading up.  Times are sweep indices.  One transition at most per check. */
typedef struct {
    int32_t phase, n_rt;
    int64_t t_first, t_last;
    int32_t e_min, e_g;
    int32_t requeue, pad;
} or_rt;

static void rt_check(or_rt *rt, int E, int e_top, int e_bottom, uint64_t t) {
    if (rt->phase == 0) {
        if (E >= e_top) { rt->t_first = (int64_t)t; rt->phase = 1; }
    } else if (rt->phase == 1) {
        if (E <= e_bottom) rt->phase = 2;
    } else {
        if (E >= e_top) { rt->n_rt += 1; rt->t_last = (int64_t)t; rt->phase = 1; }
    }
}

/* The same check applied to a given sequence of energies E[k] observed at sweep indices t[k]
 * (one check per element, in order): exposes the counter on its own so that it can be pinned
 * with hand-made sequences. */
void or_rt_replay(const int32_t *E, const int64_t *t, int n, int e_top, int e_bottom, or_rt *rt) {
    for (int k = 0; k < n; ++k) rt_check(rt, E[k], e_top, e_bottom, (uint64_t)t[k]);
}

/* ---------------------------------------------------------------- MUCA chain */
int or_pt_colours(int L);
int or_pt_colour(int dim, int L, int i);

/* n_sweeps sweeps of single-spin-flip generalized Metropolis (Eq. "muca").  The paper fixes
 * no order of the sites within a sweep; two orders are provided:
 *   order 0: lexicographic (i = 0 .. V-1);
 *   order 1: colour class by colour class (the colouring of the PT sweep, or_pt_colour: the
 *            checkerboard for even L, three classes for odd L), each class in lexicographic
 *            order.
 * The random word of an attempt is keyed by its site and sweep; the colour order draws from
 * its own streams (tags 5 + colour), numbered by the site's rank within the colour-c sites of
 * its row, so that a row's colour-c attempts take consecutive words.  thr is the chain's table, thr[b*8 + n] = threshold for a move from bin b at a
 * site with n unsatisfied bonds (the move changes E by 2*(2*dim) - 4n).  After every
 * attempt: e_min update, (if count_rt) one round-trip check against rt->e_g, and
 * a_trace[s*V + k] = E after the k-th attempt of the sweep (if non-null).  After every sweep:
 * hist[bin(E)] += 1 and e_trace[s] = E (if non-null). */
int or_muca_sweeps_order(int dim, int L, uint64_t seed, uint32_t rid, uint32_t stream,
                         const int8_t *J, int8_t *S, int32_t *E_io, uint64_t t0, uint64_t n_sweeps,
                         const uint32_t *thr, int b_top, uint32_t *hist, or_rt *rt, int count_rt,
                         int32_t *e_trace, int32_t *a_trace, int order) {
    int V = or_volume(dim, L), z = 2 * dim;
    int E = *E_io;
    int parity = ((E + or_nbonds(dim, L)) / 2) & 1;
    int e_top = or_energy_of_bin(dim, L, parity, b_top);
    int ncol = order ? or_pt_colours(L) : 1;
    for (uint64_t s = 0; s < n_sweeps; ++s) {
        uint64_t t = t0 + s;
        int k_att = 0;
        for (int colour = 0; colour < ncol; ++colour)
        for (int i = 0; i < V; ++i) {
            if (order && or_pt_colour(dim, L, i) != colour) continue;
            int x = i % L, row = i / L;            /* row = y (+ L z) */
            uint32_t r;
            if (order) {
                int j = 0;                             /* rank among the row's colour-c sites */
                for (int x2 = 0; x2 < x; ++x2) j += or_pt_colour(dim, L, row * L + x2) == colour;
                r = rand_word(seed, (uint32_t)(4 * row + (j >> 2)), (uint32_t)t, rid,
                              (uint32_t)(5 + colour) | (stream << 8), j & 3);
            } else {
                r = rand_word(seed, (uint32_t)(4 * row + (x >> 2)), (uint32_t)t, rid,
                              0u | (stream << 8), x & 3);
            }
            int h = local_field(dim, L, J, S, i);
            int n_unsat = (z - S[i] * h) / 2;        /* S_i h_i = #sat - #unsat */
            int dE = 2 * S[i] * h;                    /* = 2z - 4 n_unsat */
            int b = or_bin_of_energy(dim, L, E);
            uint32_t th = thr[(size_t)b * 8 + n_unsat];
            int accept = (th == OR_ALWAYS) || (r < th);
            if (accept) { S[i] = (int8_t)-S[i]; E += dE; }
            if (E < rt->e_min) rt->e_min = E;
            if (count_rt) rt_check(rt, E, e_top, rt->e_g, t);
            if (a_trace) a_trace[(size_t)s * V + k_att] = E;
            ++k_att;
        }
        hist[or_bin_of_energy(dim, L, E)] += 1;
        if (e_trace) e_trace[s] = E;
    }
    if (count_rt && rt->e_min < rt->e_g) rt->requeue = 1;
    *E_io = E;
    return 0;
}

/* the lexicographic order (order 0) */
int or_muca_sweeps(int dim, int L, uint64_t seed, uint32_t rid, uint32_t stream,
                   const int8_t *J, int8_t *S, int32_t *E_io, uint64_t t0, uint64_t n_sweeps,
                   const uint32_t *thr, int b_top, uint32_t *hist, or_rt *rt, int count_rt,
                   int32_t *e_trace, int32_t *a_trace) {
    return or_muca_sweeps_order(dim, L, seed, rid, stream, J, S, E_io, t0, n_sweeps, thr, b_top,
                                hist, rt, count_rt, e_trace, a_trace, 0);
}

/* ---------------------------------------------------------------- weights */
/* Quantised acceptance table from ln W (Eq. "muca"): p = W(E')/W(E) = exp(lnW(b')-lnW(b)).
 * "always" when p >= 1, else min(floor(p*2^32), 2^32-2).  Moves out of [0, b_top] get 0. */
void or_quantize(int dim, int b_top, const double *lnW, uint32_t *thr) {
    for (int b = 0; b <= b_top; ++b) {
        for (int n = 0; n < 8; ++n) {
            uint32_t v = 0u;
            int bn = b + dim - n;
            if (n <= 2 * dim && bn >= 0 && bn <= b_top) {
                double x = lnW[bn] - lnW[b];
                if (x >= 0.0) {
                    v = OR_ALWAYS;
                } else {
                    double q = floor(exp(x) * 4294967296.0);
                    v = (q >= 4294967294.0) ? 0xFFFFFFFEu : (uint32_t)q;
                }
            }
            thr[(size_t)b * 8 + n] = v;
        }
    }
}

/* Eq. "power_law": P_SH(E) = (E/(dE - E_g) + 1)^alpha, normalised to 1 at E = 0.
 * Below E_g the profile is held at its value at E_g. */
double or_ln_profile(int kind, double alpha, double pole_dE, int e_g, int E) {
    if (kind != 1) return 0.0;
    double Ec = (E < e_g) ? (double)e_g : (double)E;
    return alpha * log(Ec / (pole_dE - (double)e_g) + 1.0);
}

/* One step of the weight iteration (Sec. II, the iterative procedure the paper takes
 * from Janke 2003, with a shaped target histogram): W_{n+1}(E) = W_n(E) P_SH(E)/H_n(E),
 * H_n taken as 1 in unvisited bins; then ln W is shifted to 0 at the top bin.  kind:
 * 0 flat (P_SH = 1), 1 power law.  e_g is the lowest energy found so far. */
void or_update_weights(int dim, int L, int parity, int b_top, int kind, double alpha,
                       double pole_dE, int e_g, double *lnW, const uint32_t *hist) {
    for (int b = 0; b <= b_top; ++b) {
        int E = or_energy_of_bin(dim, L, parity, b);
        double h = hist[b] > 0 ? (double)hist[b] : 1.0;
        lnW[b] = lnW[b] + or_ln_profile(kind, alpha, pole_dE, e_g, E) - log(h);
    }
    double top = lnW[b_top];
    for (int b = 0; b <= b_top; ++b) lnW[b] -= top;
}

/* Accumulated, error-weighted form of the weight iteration: Berg's multicanonical recursion
 * (B. A. Berg, J. Stat. Phys. 82, 323 (1996); one of the iterative procedures of Janke 2003
 * that Sec. II refers to), written for bins b of a shaped target P_SH.
 *
 * An iteration run with weights W_n and histogram H_n estimates, for a pair of neighbouring
 * bins that were both visited,
 *     s(b) = ln Omega(b+1) - ln Omega(b) = [ln H(b+1) - ln W_n(b+1)] - [ln H(b) - ln W_n(b)],
 * with a Poisson variance of about 1/H(b) + 1/H(b+1).  D(b) is the mean of all iterations'
 * estimates weighted by the inverse variances g = H(b) H(b+1) / (H(b) + H(b+1)), G(b) the sum
 * of those weights (both start at 0).  The new weights follow from
 *     ln W(b) - ln W(b+1) = ln P_SH(b) - ln P_SH(b+1) + D(b)       (target with the current E_g)
 * for every pair with G(b) > 0; a pair never visited together takes the difference that the
 * plain step (or_update_weights) gives it.  ln W is 0 at the top bin.  From D = G = 0 the
 * first step equals the plain step.  A pair of which the iteration visited exactly one bin,
 * although the accumulated estimate expected at least 10 counts on the other side, restarts
 * (D = G = 0) and takes the plain step: accumulated weights that confine the chain to one side
 * of a pair would otherwise never be corrected (found on ground-state bins, which the chain
 * could not leave once their accumulated weight was too large).
 *
 * Weights that are constant over the range add no estimates: every move inside the range is
 * then accepted with probability 1, so the sequential sweep is deterministic (it only flips
 * back and forth) and its histogram is not the equilibrium one that the estimates assume. */
void or_update_weights_berg(int dim, int L, int parity, int b_top, int kind, double alpha,
                            double pole_dE, int e_g, double *lnW, const uint32_t *hist,
                            double *D, double *G) {
    double *diff = (double *)malloc(sizeof(double) * (size_t)(b_top > 0 ? b_top : 1));
    int informative = 0;
    for (int b = 0; b < b_top; ++b)
        if (lnW[b] != lnW[b_top]) informative = 1;
    for (int b = 0; b < b_top; ++b) {
        double lp0 = or_ln_profile(kind, alpha, pole_dE, e_g, or_energy_of_bin(dim, L, parity, b));
        double lp1 = or_ln_profile(kind, alpha, pole_dE, e_g, or_energy_of_bin(dim, L, parity, b + 1));
        double h0 = (double)hist[b], h1 = (double)hist[b + 1];
        if (informative && hist[b] > 0 && hist[b + 1] > 0) {
            double s = (log(h1) - lnW[b + 1]) - (log(h0) - lnW[b]);
            double g = h0 * h1 / (h0 + h1);
            D[b] = (G[b] * D[b] + g * s) / (G[b] + g);
            G[b] = G[b] + g;
        } else if (informative && G[b] > 0.0 && (hist[b] > 0) != (hist[b + 1] > 0)) {
            /* the chain stayed on one side of the pair.  Under the accumulated estimate the
             * other side should have collected H(visited) * Omega W ratio counts; if that is at
             * least 10 (zero of them has probability below 5e-5), the estimate is contradicted
             * and the weights built from it confine the chain, which no later estimate could
             * correct: the pair starts over (plain step now, accumulation from the next joint
             * visit) */
            double lnexp = (hist[b] > 0) ? (log(h0) + D[b]) + (lnW[b + 1] - lnW[b])
                                         : (log(h1) - D[b]) + (lnW[b] - lnW[b + 1]);
            if (lnexp >= 2.302585092994046) {          /* ln 10 */
                D[b] = 0.0;
                G[b] = 0.0;
            }
        }
        if (G[b] > 0.0) {
            diff[b] = lp0 - lp1 + D[b];
        } else {
            double a0 = lnW[b] + lp0 - log(h0 > 0.0 ? h0 : 1.0);
            double a1 = lnW[b + 1] + lp1 - log(h1 > 0.0 ? h1 : 1.0);
            diff[b] = a0 - a1;
        }
    }
    lnW[b_top] = 0.0;
    for (int b = b_top - 1; b >= 0; --b) lnW[b] = lnW[b + 1] + diff[b];
    free(diff);
}

/* Weights of a target ensemble from a density-of-states estimate ln Omega(b):
 *   kind 0 flat       ln W = -ln Omega                           (Eq. "muca-weights")
 *   kind 1 power law  ln W = ln P_SH - ln Omega                  (nonflat weight)
 *   kind 2 1/k        ln W = -ln sum_{E_g <= E' <= E} Omega(E')  (Eq. "1/k"), E >= E_g;
 *                     below E_g the flat form, matched at E_g
 *   kind 3 canonical  ln W = -beta E
 * then shifted to 0 at b_top. */
void or_build_weights(int dim, int L, int parity, int b_top, int kind, double alpha,
                      double pole_dE, double beta, int e_g, const double *lnOmega,
                      double *lnW) {
    int bg = or_bin_of_energy(dim, L, e_g);
    if (bg < 0) bg = 0;
    if (bg > b_top) bg = b_top;   /* an E_g above the range is read as E_top */
    for (int b = 0; b <= b_top; ++b) {
        int E = or_energy_of_bin(dim, L, parity, b);
        if (kind == 0) {
            lnW[b] = -lnOmega[b];
        } else if (kind == 1) {
            lnW[b] = or_ln_profile(1, alpha, pole_dE, e_g, E) - lnOmega[b];
        } else if (kind == 2) {
            if (b >= bg) {
                double m = lnOmega[bg];
                for (int c = bg; c <= b; ++c) if (lnOmega[c] > m) m = lnOmega[c];
                double sum = 0.0;
                for (int c = bg; c <= b; ++c) sum += exp(lnOmega[c] - m);
                lnW[b] = -(m + log(sum));
            }
        } else {
            lnW[b] = -beta * (double)E;
        }
    }
    if (kind == 2) {
        for (int b = 0; b < bg && b <= b_top; ++b)
            lnW[b] = lnW[bg] + lnOmega[bg] - lnOmega[b];
    }
    double top = lnW[b_top];
    for (int b = 0; b <= b_top; ++b) lnW[b] -= top;
}

/* ---------------------------------------------------------------- parallel tempering */
/* Metropolis thresholds per slot (Sec. II, PT): a move raising E by dE = 2z - 4n
 * (n < dim unsatisfied bonds) is accepted with p = exp(-beta_k dE).  Replica exchange
 * (Eq. "temperatureexchange") between slots k, k+1 with E_k - E_{k+1} = 4d > 0 is
 * accepted with p = exp(-(beta_{k+1} - beta_k) 4d).  Tables hold floor(p 2^32). */
static uint32_t quantize_p(double p) {
    if (p >= 1.0) return OR_ALWAYS;
    double q = floor(p * 4294967296.0);
    return (q >= 4294967294.0) ? 0xFFFFFFFEu : (uint32_t)q;
}

void or_pt_tables(int dim, int M, const double *beta, int dmax, uint32_t *thr_k,
                  uint32_t *thr_pair) {
    int z = 2 * dim;
    for (int k = 0; k < M; ++k)
        for (int n = 0; n < 8; ++n) {
            uint32_t v = 0u;
            if (n <= z) {
                int dE = 2 * z - 4 * n;
                v = (dE <= 0) ? OR_ALWAYS : quantize_p(exp(-beta[k] * (double)dE));
            }
            thr_k[k * 8 + n] = v;
        }
    for (int k = 0; k + 1 < M; ++k)
        for (int d = 0; d <= dmax; ++d)
            thr_pair[(size_t)k * (dmax + 1) + d] =
                (d == 0) ? OR_ALWAYS
                         : quantize_p(exp(-(beta[k + 1] - beta[k]) * 4.0 * (double)d));
}

/* the PT random word for one attempt: bit 31-m of r is bit (rid & 31) of word m */
static uint32_t pt_rand(uint64_t seed, uint32_t rid, int slot, int i, uint64_t t) {
    uint32_t r = 0u;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int g = 0; g < 8; ++g) {
        uint32_t ctr[4] = {(uint32_t)(8 * i + g), (uint32_t)t, rid >> 5,
                           4u | ((uint32_t)slot << 8)};
        uint32_t w[4];
        or_philox4x32_10(ctr, key, w);
        for (int j = 0; j < 4; ++j) {
            int m = 4 * g + j;
            r |= ((w[j] >> (rid & 31)) & 1u) << (31 - m);
        }
    }
    return r;
}

/* Colour of a coordinate along one axis for odd L: x mod 3, except that the last position
 * takes colour 1 when x mod 3 would give it colour 0 (L = 1 mod 3), the colour of its
 * periodic neighbour x = 0.  Neighbouring positions (periodically) never share a colour. */
static int odd_axis_colour(int L, int x) {
    if (x == L - 1 && (L - 1) % 3 == 0) return 1;
    return x % 3;
}

/* Colour classes of the PT sweep.  Even L: the checkerboard, colour (x + y + z) mod 2.
 * Odd L (the checkerboard is not a proper colouring under periodic boundaries): colour
 * (c(x) + c(y) + c(z)) mod 3 with c from odd_axis_colour; a step to a neighbour changes one
 * of c(x), c(y), c(z) by 1 or 2 (mod 3), so neighbours always differ in colour. */
int or_pt_colours(int L) { return (L % 2 == 0) ? 2 : 3; }

int or_pt_colour(int dim, int L, int i) {
    int x = i % L, y = (i / L) % L, zz = (dim == 3) ? i / (L * L) : 0;
    if (L % 2 == 0) return (x + y + zz) & 1;
    int c = odd_axis_colour(L, x) + odd_axis_colour(L, y) + (dim == 3 ? odd_axis_colour(L, zz) : 0);
    return c % 3;
}

/* One realization, M replicas.  S holds the configuration currently at slot k in
 * S[k*V ...]; E[k] its energy; label[k] the replica (configuration) number at slot k.
 * Per sweep t: every slot gets a Metropolis sweep colour class by colour class (or_pt_colour;
 * each class in lexicographic order); then exchanges between slots (k, k+1) for
 * k = t mod 2, t mod 2 + 2, ...; then, if count_rt, one round-trip check per replica with
 * bottom e_g and top e_hot (Sec. III). rt is indexed by label.  label_trace (if non-null)
 * receives, per sweep s, the energy of replica label m at [s*M + m] after the exchanges. */
int or_pt_sweeps(int dim, int L, uint64_t seed, uint32_t rid, int M, const int8_t *J,
                 int8_t *S, int32_t *E, int32_t *label, uint64_t t0, uint64_t n_sweeps,
                 const uint32_t *thr_k, const uint32_t *thr_pair, int dmax, or_rt *rt,
                 int count_rt, int e_g, int e_hot, uint64_t *swap_acc, int32_t *label_trace) {
    int V = or_volume(dim, L), z = 2 * dim;
    int ncol = or_pt_colours(L);
    int8_t *tmp = (int8_t *)malloc((size_t)V);
    for (uint64_t s = 0; s < n_sweeps; ++s) {
        uint64_t t = t0 + s;
        for (int k = 0; k < M; ++k) {
            int8_t *Sk = S + (size_t)k * V;
            for (int colour = 0; colour < ncol; ++colour) {
                for (int i = 0; i < V; ++i) {
                    if (or_pt_colour(dim, L, i) != colour) continue;
                    int h = local_field(dim, L, J, Sk, i);
                    int n_unsat = (z - Sk[i] * h) / 2;
                    int dE = 2 * Sk[i] * h;
                    int accept;
                    if (dE <= 0) {
                        accept = 1;
                    } else {
                        uint32_t r = pt_rand(seed, rid, k, i, t);
                        accept = r < thr_k[k * 8 + n_unsat];
                    }
                    if (accept) { Sk[i] = (int8_t)-Sk[i]; E[k] += dE; }
                }
            }
        }
        for (int k = (int)(t & 1); k + 1 < M; k += 2) {
            int accept;
            if (E[k + 1] >= E[k]) {
                accept = 1;
            } else {
                int d = (E[k] - E[k + 1]) / 4;
                uint32_t th = (d <= dmax) ? thr_pair[(size_t)k * (dmax + 1) + d] : 0u;
                uint32_t r = rand_word(seed, (uint32_t)k, (uint32_t)t, rid, 1u, 0);
                accept = (th == OR_ALWAYS) || (r < th);
            }
            if (accept) {
                memcpy(tmp, S + (size_t)k * V, (size_t)V);
                memcpy(S + (size_t)k * V, S + (size_t)(k + 1) * V, (size_t)V);
                memcpy(S + (size_t)(k + 1) * V, tmp, (size_t)V);
                int32_t te = E[k]; E[k] = E[k + 1]; E[k + 1] = te;
                int32_t tl = label[k]; label[k] = label[k + 1]; label[k + 1] = tl;
                if (swap_acc) swap_acc[k] += 1;
            }
        }
        for (int k = 0; k < M; ++k) {
            or_rt *r = &rt[label[k]];
            if (E[k] < r->e_min) r->e_min = E[k];
            if (count_rt) rt_check(r, E[k], e_hot, e_g, t);
            if (label_trace) label_trace[(size_t)s * M + label[k]] = E[k];
        }
    }
    free(tmp);
    return 0;
}

/* One step of the constant-exchange-rate temperature adaptation (Sec. II, PT: the
 * exchange rates are imposed on each realization during equilibration by moving its
 * temperatures; the rule below is this implementation's own).  beta[0..M-1] ascending; the
 * end points stay.  Pair k (slots k, k+1, gap D_k = beta[k+1] - beta[k]) accepted n_acc[k] of
 * n_att[k] exchange attempts, rate A_k, clamped to [0.005, 0.995].  Reading the cost
 * w_k = -ln A_k as proportional to the gap, s_k = w_k / D_k is the pair's stiffness and the
 * gaps that give every pair the same rate are D*_k = span (1/s_k) / sum_j (1/s_j).  The new
 * gaps are (1 - eta) D_k + eta D*_k; the betas are their running sums from beta[0].  With a
 * pair that had no attempt nothing changes.  Equal rates are the fixed point. */
void or_pt_adapt(int M, double *beta, const uint64_t *n_acc, const uint64_t *n_att, double eta) {
    if (M < 3) return;
    for (int k = 0; k + 1 < M; ++k)
        if (n_att[k] == 0) return;
    double span = beta[M - 1] - beta[0];
    double *gap = (double *)malloc(sizeof(double) * (size_t)(M - 1));
    double *inv_s = (double *)malloc(sizeof(double) * (size_t)(M - 1));
    double sum = 0.0;
    for (int k = 0; k + 1 < M; ++k) {
        double a = (double)n_acc[k] / (double)n_att[k];
        if (a < 0.005) a = 0.005;
        if (a > 0.995) a = 0.995;
        gap[k] = beta[k + 1] - beta[k];
        inv_s[k] = gap[k] / -log(a);
        sum += inv_s[k];
    }
    /* beta[0] and beta[M-1] stay; the interior points are running sums of the new gaps */
    for (int k = 0; k + 2 < M; ++k) {
        double target = span * inv_s[k] / sum;
        beta[k + 1] = beta[k] + ((1.0 - eta) * gap[k] + eta * target);
    }
    free(gap);
    free(inv_s);
}

/* ---------------------------------------------------------------- brute force */
/* Density of states g(u) (u = number of unsatisfied bonds) by enumerating every spin
 * configuration with spin V-1 held up (the global flip doubles each count), in Gray-code
 * order so that consecutive states differ by one spin. */
int or_dos_bruteforce(int dim, int L, const int8_t *J, uint64_t *g) {
    int V = or_volume(dim, L), nb = or_nbonds(dim, L);
    if (V > 30) return -1;
    int8_t *S = (int8_t *)malloc((size_t)V);
    for (int i = 0; i < V; ++i) S[i] = 1;
    for (int u = 0; u <= nb; ++u) g[u] = 0;
    int E = or_energy(dim, L, J, S);
    uint64_t nstates = 1ull << (V - 1);
    g[(E + nb) / 2] += 2;
    for (uint64_t k = 1; k < nstates; ++k) {
        int i = __builtin_ctzll(k);          /* Gray code: flip the lowest set bit of k */
        E += 2 * S[i] * local_field(dim, L, J, S, i);
        S[i] = (int8_t)-S[i];
        g[(E + nb) / 2] += 2;
    }
    free(S);
    return 0;
}
