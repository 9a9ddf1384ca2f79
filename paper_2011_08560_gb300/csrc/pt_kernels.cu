// pt_kernels.cu -- a6 + a7: parallel tempering (Sec. II, PT; Eq. "temperatureexchange").
//
// M replicas of every realization, one per temperature slot k (beta ascending with k, slot
// 0 hottest; every realization has its own temperature set).  Each sweep: a Metropolis sweep
// of every slot colour class by colour class (even L: the checkerboard, sites with even
// coordinate sum first; odd L: three colours, see pt_colour), then replica exchange between
// slots (k, k+1) for k = t mod 2, t mod 2 + 2, ..., then one round-trip check per replica
// (Sec. III, PT variant: between E_g and an energy typical of a high temperature, E_hot).
//
// Layout.  Realizations come in groups of 32 (realization id 32g + b is bit b); the
// configuration at slot k of a group is one multi-spin-coded word per site.  Exchanges move
// configurations (not temperatures) with masked XOR swaps of whole words.
//
// Acceptance.  For a site word the unsatisfied-bond count of every bit is a bit-sliced sum;
// bits with dE <= 0 flip.  Each uphill bit b compares its 32-bit random number r_b with its
// own threshold (slot k, its realization's beta_k, its class); r_b's bit 31-m is bit b of
// random word m (Philox4x32-10 of counter (8i + m/4, t, g, 4 | k<<8), word m&3), and the
// thresholds are stored the same way, as bit planes: plane m of class c holds bit 31-m of
// the 32 realizations' thresholds.  The comparison runs over planes from the most
// significant one: the first 8 without branches, the rest only while a bit is undecided.
//
// Parallel work.  One thread-block cluster per group: CS CTAs, each owning M/CS consecutive
// slots in shared memory.  Energies are recomputed after every sweep (bit-sliced counters,
// warp bit-matrix transpose, popcount); exchanges between slots owned by different CTAs read
// and write the neighbour CTA's shared memory (distributed shared memory) between cluster
// barriers.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "eamc.h"
#include "eamc_ctx.cuh"
#include "eamc_internal.cuh"

namespace cg = cooperative_groups;
using namespace eamc;

struct PtRt {
    int32_t phase, n_rt;
    int64_t t_first, t_last;
    int32_t e_min, pad;
};

struct PtState {
    int dim = 0, L = 0, V = 0, nb = 0, M = 0, n_real = 0, n_groups = 0, cs = 1;
    uint32_t rid0 = 0;
    uint64_t t = 0;
    uint64_t t_win = 0;            // start of the exchange-count window (pt_adapt)
    uint32_t *d_spins = nullptr;   // [g][k][V]
    uint32_t *d_bonds = nullptr;   // [g][nb]
    int32_t *d_E = nullptr;        // [g][k][32]
    int32_t *d_label = nullptr;    // [g][k][32]
    PtRt *d_rt = nullptr;          // [g][label][32]
    int32_t *d_bounds = nullptr;   // [g][32][2] (e_g, e_hot)
    double *d_beta = nullptr;      // [g][k][32] inverse temperatures
    uint32_t *d_planes = nullptr;  // [g][k][32 planes][4] Metropolis thresholds (classes 0..2, pad)
    uint32_t *d_xacc = nullptr;    // [g][k][32] accepted exchanges of pair (k, k+1) in the window
    unsigned long long *d_swaps = nullptr;  // [M-1]
    int *d_err = nullptr;
};

namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t maj3(uint32_t a, uint32_t b, uint32_t c) {
    return (a & b) | (a & c) | (b & c);
}

// 32x32 bit-matrix transpose across a warp: afterwards lane t holds, in bit s, bit t of
// what lane s held
__device__ __forceinline__ uint32_t warp_transpose(uint32_t x, int lane) {
    const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int j = 16 >> s;
        const uint32_t m = masks[s];
        const uint32_t y = __shfl_xor_sync(kFull, x, j);
        x = (lane & j) ? ((x & ~m) | ((y & ~m) >> j)) : ((x & m) | ((y & m) << j));
    }
    return x;
}

template <int DIM, int L>
struct PtGeo {
    static constexpr int NR = DIM == 3 ? L * L : L;
    static constexpr int V = NR * L;
    static constexpr int NB = DIM * V;
    static constexpr int HALF = V / 2;  // sites of one colour
};

// neighbour of site i along axis d (0 x, 1 y, 2 z), direction +1 / -1
template <int DIM, int L>
__device__ __forceinline__ int pt_nbr(int i, int d, int sgn) {
    int x = i % L, y = (i / L) % L, z = DIM == 3 ? i / (L * L) : 0;
    if (d == 0) x = (x + sgn + L) % L;
    else if (d == 1) y = (y + sgn + L) % L;
    else z = (z + sgn + L) % L;
    return x + L * (y + L * z);
}

// Colour of a site for the PT sweep.  Even L: (x + y + z) mod 2.  Odd L: the sum of per-axis
// colours mod 3, an axis position x having colour x mod 3 except the last one (x = L-1) when
// L = 1 (mod 3), which takes 1 so that it differs from both neighbours L-2 and 0; a step to a
// neighbour then changes the sum by 1 or 2 (mod 3), so no two neighbours share a colour.
template <int DIM, int L>
__device__ __forceinline__ int pt_colour(int i) {
    const int x = i % L, y = (i / L) % L, z = DIM == 3 ? i / (L * L) : 0;
    if constexpr ((L & 1) == 0) {
        return (x + y + z) & 1;
    } else {
        auto ax = [](int c) { return (c == L - 1 && (L - 1) % 3 == 0) ? 1 : c % 3; };
        return (ax(x) + ax(y) + (DIM == 3 ? ax(z) : 0)) % 3;
    }
}

__device__ __forceinline__ uint32_t quantize_prob(double p) {
    if (p >= 1.0) return kAlways;
    const double q = floor(p * 4294967296.0);
    return (q >= 4294967294.0) ? 0xFFFFFFFEu : (uint32_t)q;
}

constexpr int kTailQ = 32;  // open comparisons a warp defers per colour phase

struct PtArgs {
    uint32_t *spins;
    const uint32_t *bonds;
    int32_t *E;
    int32_t *label;
    PtRt *rt;
    const int32_t *bounds;
    const uint32_t *planes;
    const double *beta;
    uint32_t *xacc;
    unsigned long long *swaps;
    int M, spc, n_real;
    uint32_t rid0;
    uint64_t t0, n_sweeps;
    int count_rt;
    PhiloxKey key;
};

template <int DIM, int L>
__global__ void __launch_bounds__(256, 1) pt_kernel(PtArgs a) {
    using G = PtGeo<DIM, L>;
    constexpr int V = G::V, NB = G::NB, HALF = G::HALF;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int g = blockIdx.x / (int)cluster.num_blocks();
    const int spc = a.spc, k0 = rank * spc, M = a.M;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;

    constexpr int NCOL = (L & 1) ? 3 : 2;
    extern __shared__ __align__(16) uint32_t sm[];
    uint4 *P = reinterpret_cast<uint4 *>(sm);  // [spc][32] threshold planes (class 0, 1, 2, pad)
    uint32_t *S = sm + spc * 128;           // [spc][V]
    uint32_t *J = S + spc * V;              // [NB], J[i*DIM + d]
    int32_t *Es = (int32_t *)(J + NB);      // [spc][32]
    int32_t *Ls = Es + spc * 32;            // [spc][32]
    uint32_t *Amask = (uint32_t *)(Ls + spc * 32);  // [spc] exchange masks of owned pairs
    // per-warp queue of site words whose comparison is still open after 8 planes:
    // [nwarps][kTailQ] x (site | slot << 16, acc, und, C0, C1, C2)
    uint32_t *TQ = Amask + spc;
    int32_t *Ep = (int32_t *)(TQ + nwarps * kTailQ * 6);   // [nwarps][spc][32] partial counts
    uint32_t *Xc = (uint32_t *)(Ep + nwarps * spc * 32);  // [spc][32] accepted exchanges, this launch
    int32_t *Bd = (int32_t *)(Xc + spc * 32);             // [32][2] round-trip bounds (e_g, e_hot)
    double *Db = reinterpret_cast<double *>((reinterpret_cast<uintptr_t>(Bd + 64) + 7) & ~uintptr_t(7));  // [spc][32]
    // round-trip records of the replica labels k0 .. k0+spc-1 ("home" labels of this CTA), for
    // the launch; a label's record is updated by whichever CTA holds that replica, through
    // distributed shared memory
    PtRt *Rh = reinterpret_cast<PtRt *>(Db + spc * 32);    // [spc][32]
    int32_t *Cl = (int32_t *)(Rh + spc * 32);  // odd L: sites by colour [V], then offsets [4]

    const uint32_t group_rid0 = a.rid0 + 32u * (uint32_t)g;
    const int nvalid = min(32, a.n_real - 32 * g);
    const uint32_t valid = nvalid >= 32 ? kFull : ((1u << nvalid) - 1u);

    for (int k = tid; k < spc * V; k += blockDim.x)
        S[k] = a.spins[((size_t)g * M + k0) * V + k];
    for (int k = tid; k < NB; k += blockDim.x) J[k] = a.bonds[(size_t)g * NB + k];
    for (int k = tid; k < spc * 32; k += blockDim.x) {
        Es[k] = a.E[((size_t)g * M + k0) * 32 + k];
        Ls[k] = a.label[((size_t)g * M + k0) * 32 + k];
    }
    for (int k = tid; k < spc * 128; k += blockDim.x) sm[k] = a.planes[((size_t)g * M + k0) * 128 + k];
    // per launch: beta_{k+1} - beta_k of every owned pair and realization, the round-trip bounds,
    // zeroed exchange counters (added to the global ones at the end)
    for (int q = tid; q < spc * 32; q += blockDim.x) {
        const int k = k0 + (q >> 5), b = q & 31;
        Db[q] = (k + 1 < M) ? a.beta[((size_t)g * M + k + 1) * 32 + b] - a.beta[((size_t)g * M + k) * 32 + b] : 0.0;
        Xc[q] = 0u;
    }
    for (int q = tid; q < 64; q += blockDim.x) Bd[q] = a.bounds[(size_t)g * 64 + q];
    for (int q = tid; q < spc * 32; q += blockDim.x) Rh[q] = a.rt[((size_t)g * M + k0) * 32 + q];
    if constexpr ((L & 1) != 0) {
        if (tid == 0) {  // colour classes in lexicographic order (a few thousand steps per launch)
            int n = 0;
            for (int c = 0; c < NCOL; ++c) {
                Cl[V + c] = n;
                for (int i = 0; i < V; ++i)
                    if (pt_colour<DIM, L>(i) == c) Cl[n++] = i;
            }
            Cl[V + NCOL] = n;
        }
    }
    __syncthreads();
    cluster.sync();

    for (uint64_t s = 0; s < a.n_sweeps; ++s) {
        const uint64_t t = a.t0 + s;
        const uint32_t tt = (uint32_t)t;
        // ---- checkerboard Metropolis sweep of every owned slot
        // planes 8..31 of one site word: drawn only while a bit is still undecided
        auto finish = [&](int i, int ks, uint32_t C0, uint32_t C1, uint32_t C2, uint32_t acc, uint32_t und) {
            const uint32_t c2 = (uint32_t)g + (a.rid0 >> 5), c3 = 4u | ((uint32_t)(k0 + ks) << 8);
            const uint4 *Pk = P + ks * 32;
            uint4 w4 = make_uint4(0, 0, 0, 0);
            for (int m = 8; m < 32 && und; ++m) {
                if ((m & 3) == 0)
                    w4 = philox4x32_10(make_uint4((uint32_t)(8 * i + (m >> 2)), tt, c2, c3), a.key);
                const uint32_t R = uint4_get(w4, m & 3);
                const uint4 q = Pk[m];
                const uint32_t Tm = (C0 & q.x) | (C1 & q.y) | (C2 & q.z);
                acc |= und & ~R & Tm;
                und &= ~(R ^ Tm);
            }
            return acc;
        };
        uint32_t *tq = TQ + warp * kTailQ * 6;
        for (int colour = 0; colour < NCOL; ++colour) {
            const int nc = ((L & 1) == 0) ? HALF : Cl[V + colour + 1] - Cl[V + colour];
            // site words of one colour never neighbour each other, so a word whose comparison
            // is still open after 8 planes (about 6 % of them) can be finished after the others:
            // the warp queues them and finishes them together, one per lane
            int nq = 0;
            for (int item = tid; item < spc * nc; item += blockDim.x) {
                const int ks = item / nc, j = item % nc;
                int i;
                if constexpr ((L & 1) == 0) {
                    const int row = j / (L / 2), xh = j % (L / 2);
                    const int y = row % L, z = DIM == 3 ? row / L : 0;
                    i = 2 * xh + ((colour + y + z) & 1) + L * row;
                } else {
                    i = Cl[Cl[V + colour] + j];
                }
                uint32_t *Sk = S + ks * V;
                const uint32_t si = Sk[i];
                uint32_t u[2 * DIM];
#pragma unroll
                for (int d = 0; d < DIM; ++d) {
                    const int jp = pt_nbr<DIM, L>(i, d, +1), jm = pt_nbr<DIM, L>(i, d, -1);
                    u[2 * d] = si ^ Sk[jp] ^ J[i * DIM + d];
                    u[2 * d + 1] = si ^ Sk[jm] ^ J[jm * DIM + d];
                }
                uint32_t n0, n1, n2;  // bit-sliced count of unsatisfied bonds
                if constexpr (DIM == 3) {
                    const uint32_t s1 = u[0] ^ u[1] ^ u[2], c1 = maj3(u[0], u[1], u[2]);
                    const uint32_t s2 = u[3] ^ u[4] ^ u[5], c2 = maj3(u[3], u[4], u[5]);
                    n0 = s1 ^ s2;
                    const uint32_t c3 = s1 & s2;
                    n1 = c1 ^ c2 ^ c3;
                    n2 = maj3(c1, c2, c3);
                } else {
                    const uint32_t s1 = u[0] ^ u[1] ^ u[2], c1 = maj3(u[0], u[1], u[2]);
                    n0 = s1 ^ u[3];
                    const uint32_t c2 = s1 & u[3];
                    n1 = c1 ^ c2;
                    n2 = c1 & c2;
                }
                // uphill classes: n < DIM unsatisfied bonds (dE = 2*(2*DIM) - 4n > 0)
                uint32_t C[3];
                C[0] = ~n2 & ~n1 & ~n0;
                C[1] = ~n2 & ~n1 & n0;
                C[2] = (DIM == 3) ? (~n2 & n1 & ~n0) : 0u;
                const uint32_t up = C[0] | C[1] | C[2];
                uint32_t acc = ~up;  // dE <= 0 always accepted
                uint32_t und = up & valid;
                const int k = k0 + ks;
                const uint4 *Pk = P + ks * 32;
                // the 8 most significant planes come from two independent Philox calls and are
                // compared without branches; planes 8..31 are drawn only while a bit is still
                // undecided (about 2^-8 per uphill bit)
                const uint32_t c2 = (uint32_t)g + (a.rid0 >> 5), c3 = 4u | ((uint32_t)k << 8);
                const uint4 wa = philox4x32_10(make_uint4((uint32_t)(8 * i), tt, c2, c3), a.key);
                const uint4 wb = philox4x32_10(make_uint4((uint32_t)(8 * i + 1), tt, c2, c3), a.key);
                const uint32_t Rm[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    const uint4 q = Pk[m];
                    const uint32_t Tm = (C[0] & q.x) | (C[1] & q.y) | (C[2] & q.z);
                    acc |= und & ~Rm[m] & Tm;  // r bit 0, threshold bit 1: r < threshold
                    und &= ~(Rm[m] ^ Tm);      // equal bits: still undecided
                }
                (void)c2;
                (void)c3;
                // the lanes of this warp that have an item in this pass of the loop (items are consecutive)
                const int rem = spc * nc - (item - lane);
                const uint32_t live = rem >= 32 ? kFull : ((1u << rem) - 1u);
                const bool open = und != 0u;
                const uint32_t om = __ballot_sync(live, open);
                const int pos = nq + __popc(om & ((1u << lane) - 1u));
                const bool deferred = open && pos < kTailQ;
                if (deferred) {
                    uint32_t *e = tq + pos * 6;
                    e[0] = (uint32_t)i | ((uint32_t)ks << 16);
                    e[1] = acc;
                    e[2] = und;
                    e[3] = C[0];
                    e[4] = C[1];
                    e[5] = C[2];
                } else {
                    if (open) acc = finish(i, ks, C[0], C[1], C[2], acc, und);  // queue full
                    Sk[i] = si ^ (acc & valid);
                }
                nq += __popc(om);
            }
            __syncwarp();
            nq = __shfl_sync(kFull, nq, 0);
            for (int e0 = 0; e0 < min(nq, kTailQ); e0 += 32) {
                const int e = e0 + lane;
                if (e < min(nq, kTailQ)) {
                    const uint32_t *q = tq + e * 6;
                    const int i = (int)(q[0] & 0xFFFFu), ks = (int)(q[0] >> 16);
                    const uint32_t acc = finish(i, ks, q[3], q[4], q[5], q[1], q[2]);
                    S[ks * V + i] ^= acc & valid;
                }
            }
            __syncthreads();
        }
        // ---- energies of the owned slots: u_b = number of unsatisfied bonds of bit b; every
        //      warp leaves its partial counts in Ep, one barrier, then they are summed
        for (int ks = 0; ks < spc; ++ks) {
            const uint32_t *Sk = S + ks * V;
            int part = 0;
            for (int base = warp * 32; base < V; base += nwarps * 32) {
                const int i = base + lane;
                uint32_t c0 = 0, c1 = 0;  // bit-sliced count (0..3) of this site's +d bonds
                if (i < V) {
#pragma unroll
                    for (int d = 0; d < DIM; ++d) {
                        const uint32_t w = Sk[i] ^ Sk[pt_nbr<DIM, L>(i, d, +1)] ^ J[i * DIM + d];
                        c1 ^= c0 & w;  // add one bit into the 2-bit counter (max 3)
                        c0 ^= w;
                    }
                }
                const uint32_t t0w = warp_transpose(c0, lane), t1w = warp_transpose(c1, lane);
                part += __popc(t0w) + 2 * __popc(t1w);
            }
            Ep[(warp * spc + ks) * 32 + lane] = part;
        }
        __syncthreads();
        for (int k = tid; k < spc * 32; k += blockDim.x) {
            int u = 0;
            for (int w = 0; w < nwarps; ++w) u += Ep[w * spc * 32 + k];
            Es[k] = 2 * u - NB;
        }
        cluster.sync();  // every slot's energy is known (and a barrier of this CTA)
        // ---- replica exchange between (k, k+1), k = t mod 2 (mod 2); the owner of k decides,
        //      one warp per owned slot
        {
            for (int ks = warp; ks < spc; ks += nwarps) {
                const int k = k0 + ks;
                uint32_t A = 0u;
                if (((k ^ (int)t) & 1) == 0 && k + 1 < M) {
                    const int kr = (ks + 1 < spc) ? rank : rank + 1;
                    const int ksr = (ks + 1 < spc) ? ks + 1 : 0;
                    int32_t *Er = cluster.map_shared_rank(Es, kr);
                    const int e0 = Es[ks * 32 + lane], e1 = Er[ksr * 32 + lane];
                    bool ok;
                    if (e1 >= e0) {
                        ok = true;
                    } else {
                        // Eq. "temperatureexchange" with this realization's beta_k, beta_k+1
                        const int d = (e0 - e1) / 4;
                        const uint32_t th = quantize_prob(exp(-Db[ks * 32 + lane] * 4.0 * (double)d));
                        const uint4 w = philox4x32_10(make_uint4((uint32_t)k, tt, group_rid0 + lane, 1u), a.key);
                        ok = (th == kAlways) || (w.x < th);
                    }
                    A = __ballot_sync(kFull, ok) & valid;
                    Xc[ks * 32 + lane] += (A >> lane) & 1u;
                }
                if (lane == 0) Amask[ks] = A;
            }
        }
        __syncthreads();
        for (int ks = 0; ks < spc; ++ks) {
            const uint32_t A = Amask[ks];
            if (!A) continue;  // uniform across the CTA
            const int kr = (ks + 1 < spc) ? rank : rank + 1;
            const int ksr = (ks + 1 < spc) ? ks + 1 : 0;
            uint32_t *Sr = cluster.map_shared_rank(S, kr) + ksr * V;
            uint32_t *Sl = S + ks * V;
            for (int i = tid; i < V; i += blockDim.x) {
                const uint32_t d = (Sl[i] ^ Sr[i]) & A;
                Sl[i] ^= d;
                Sr[i] ^= d;
            }
            if (tid < 32 && ((A >> tid) & 1u)) {
                int32_t *Er = cluster.map_shared_rank(Es, kr);
                int32_t *Lr = cluster.map_shared_rank(Ls, kr);
                const int32_t te = Es[ks * 32 + tid];
                Es[ks * 32 + tid] = Er[ksr * 32 + tid];
                Er[ksr * 32 + tid] = te;
                const int32_t tl = Ls[ks * 32 + tid];
                Ls[ks * 32 + tid] = Lr[ksr * 32 + tid];
                Lr[ksr * 32 + tid] = tl;
            }
        }
        cluster.sync();  // exchanges complete everywhere
        // ---- round trips / lowest energy per replica (by label)
        for (int q = tid; q < spc * 32; q += blockDim.x) {
            const int ks = q >> 5, b = q & 31;
            if (!((valid >> b) & 1u)) continue;
            const int lbl = Ls[q], E = Es[q];
            PtRt &r = cluster.map_shared_rank(Rh, lbl / spc)[(lbl % spc) * 32 + b];
            if (E < r.e_min) r.e_min = E;
            if (a.count_rt) {
                const int eg = Bd[2 * b + 0];
                const int ehot = Bd[2 * b + 1];
                if (r.phase == 0) {
                    if (E >= ehot) { r.t_first = (int64_t)t; r.phase = 1; }
                } else if (r.phase == 1) {
                    if (E <= eg) r.phase = 2;
                } else {
                    if (E >= ehot) { r.n_rt += 1; r.t_last = (int64_t)t; r.phase = 1; }
                }
            }
            (void)ks;
        }
        __syncthreads();
    }
    // ---- write back (every CTA of the cluster is done with this CTA's records)
    cluster.sync();
    for (int q = tid; q < spc * 32; q += blockDim.x) a.rt[((size_t)g * M + k0) * 32 + q] = Rh[q];
    for (int q = tid; q < spc * 32; q += blockDim.x) {
        const int k = k0 + (q >> 5);
        if (Xc[q]) {
            a.xacc[((size_t)g * M + k) * 32 + (q & 31)] += Xc[q];
            atomicAdd(&a.swaps[k], (unsigned long long)Xc[q]);
        }
    }
    for (int k = tid; k < spc * V; k += blockDim.x) a.spins[((size_t)g * M + k0) * V + k] = S[k];
    for (int k = tid; k < spc * 32; k += blockDim.x) {
        a.E[((size_t)g * M + k0) * 32 + k] = Es[k];
        a.label[((size_t)g * M + k0) * 32 + k] = Ls[k];
    }
    cluster.sync();
}

// initial state: couplings and per-slot random spins from the seed (or the caller), energies
// by full recomputation, labels = slot.  One warp per (group, slot).
template <int DIM, int L>
__global__ void pt_init_kernel(uint32_t *spins, uint32_t *bonds, int32_t *E, int32_t *label,
                               const int8_t *Jin, int M, int n_real, uint32_t rid0, PhiloxKey key) {
    using G = PtGeo<DIM, L>;
    constexpr int V = G::V, NB = G::NB;
    const int g = blockIdx.x / M, k = blockIdx.x % M, lane = threadIdx.x;
    const uint32_t rid = rid0 + 32u * g + lane;
    const bool act = (int)(32 * g + lane) < n_real;
    uint32_t *sp = spins + ((size_t)g * M + k) * V;
    uint32_t *bd = bonds + (size_t)g * NB;
    if (k == 0) {
        for (int j0 = 0; j0 < NB; j0 += 4) {
            const uint4 w = philox4x32_10(make_uint4((uint32_t)(j0 >> 2), 0u, rid, 3u), key);
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                const int j = j0 + jj;
                if (j < NB) {
                    const bool neg = act && (Jin ? (Jin[(size_t)(32 * g + lane) * NB + j] < 0)
                                                 : ((uint4_get(w, jj) >> 31) != 0));
                    const uint32_t m = __ballot_sync(kFull, neg);
                    if (lane == 0) bd[j] = m;
                }
            }
        }
    }
    for (int i0 = 0; i0 < V; i0 += 4) {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)(i0 >> 2), 0u, rid, 2u | ((uint32_t)k << 8)), key);
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int i = i0 + jj;
            if (i < V) {
                const bool neg = act && ((uint4_get(w, jj) >> 31) != 0);
                const uint32_t m = __ballot_sync(kFull, neg);
                if (lane == 0) sp[i] = m;
            }
        }
    }
    label[((size_t)g * M + k) * 32 + lane] = k;
}

// energies of every (group, slot) from scratch; one warp per (group, slot)
template <int DIM, int L>
__global__ void pt_energy_kernel(const uint32_t *spins, const uint32_t *bonds, int32_t *E, int M) {
    using G = PtGeo<DIM, L>;
    constexpr int V = G::V, NB = G::NB;
    const int g = blockIdx.x / M, k = blockIdx.x % M, lane = threadIdx.x;
    const uint32_t *sp = spins + ((size_t)g * M + k) * V;
    const uint32_t *bd = bonds + (size_t)g * NB;
    int u = 0;
    for (int i = 0; i < V; ++i)
        for (int d = 0; d < DIM; ++d) {
            const uint32_t w = sp[i] ^ sp[pt_nbr<DIM, L>(i, d, +1)] ^ bd[i * DIM + d];
            u += (w >> lane) & 1u;
        }
    E[((size_t)g * M + k) * 32 + lane] = 2 * u - NB;
}

template <int DIM, int L>
cudaError_t pt_launch_all(PtState *p, const int8_t *dJ, ea_ctx *ctx, int what, uint64_t n_sweeps,
                          int count_rt) {
    using G = PtGeo<DIM, L>;
    if (what == 0) {
        pt_init_kernel<DIM, L><<<p->n_groups * p->M, 32, 0, ctx->stream>>>(
            p->d_spins, p->d_bonds, p->d_E, p->d_label, dJ, p->M, p->n_real, p->rid0, ctx->key);
        pt_energy_kernel<DIM, L><<<p->n_groups * p->M, 32, 0, ctx->stream>>>(p->d_spins, p->d_bonds, p->d_E, p->M);
        return cudaGetLastError();
    }
    PtArgs a;
    a.spins = p->d_spins;
    a.bonds = p->d_bonds;
    a.E = p->d_E;
    a.label = p->d_label;
    a.rt = p->d_rt;
    a.bounds = p->d_bounds;
    a.planes = p->d_planes;
    a.beta = p->d_beta;
    a.xacc = p->d_xacc;
    a.swaps = p->d_swaps;
    a.M = p->M;
    a.spc = p->M / p->cs;
    a.n_real = p->n_real;
    a.rid0 = p->rid0;
    a.t0 = p->t;
    a.n_sweeps = n_sweeps;
    a.count_rt = count_rt;
    a.key = ctx->key;
    const int items = a.spc * (G::V / 2);
    const int threads = std::min(256, std::max(64, (items + 31) / 32 * 32));
    const size_t smem = (size_t)(a.spc * 128 + a.spc * G::V + G::NB + a.spc * 32 * 2 + a.spc +
                                 (threads / 32) * (kTailQ * 6 + a.spc * 32) + a.spc * 32 + 64 + 1 + 2 * a.spc * 32 +
                                 a.spc * 32 * (int)(sizeof(PtRt) / 4) + ((L & 1) ? G::V + 4 : 0)) * 4;
    cudaError_t e = cudaFuncSetAttribute(pt_kernel<DIM, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(pt_kernel<DIM, L>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof cfg);
    cfg.gridDim = dim3(p->n_groups * p->cs);
    // up to one thread per site of one colour of the CTA's slots (at most 256, at least 2
    // warps); 512-thread blocks measured slower (barrier cost, register cap)
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = p->cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, pt_kernel<DIM, L>, a);
}

cudaError_t pt_dispatch(PtState *p, const int8_t *dJ, ea_ctx *ctx, int what, uint64_t n_sweeps, int count_rt) {
#define PT_CASE(D, LL) \
    if (p->dim == D && p->L == LL) return pt_launch_all<D, LL>(p, dJ, ctx, what, n_sweeps, count_rt);
    PT_CASE(3, 3) PT_CASE(3, 4) PT_CASE(3, 5) PT_CASE(3, 6) PT_CASE(3, 7) PT_CASE(3, 8) PT_CASE(3, 9)
    PT_CASE(3, 10) PT_CASE(3, 11) PT_CASE(3, 12)
    PT_CASE(2, 3) PT_CASE(2, 4) PT_CASE(2, 5) PT_CASE(2, 6) PT_CASE(2, 7) PT_CASE(2, 8) PT_CASE(2, 9)
    PT_CASE(2, 10) PT_CASE(2, 11) PT_CASE(2, 12)
#undef PT_CASE
    return cudaErrorInvalidValue;
}

// Metropolis threshold planes of every (group, slot): one warp, lane b = realization bit.
// Class n (n unsatisfied bonds, dE = 2z - 4n > 0) accepts with exp(-beta dE) (Sec. II, PT).
__global__ void pt_planes_kernel(const double *__restrict__ beta, int dim, uint32_t *__restrict__ planes) {
    const int gk = blockIdx.x, lane = threadIdx.x;
    const int z = 2 * dim;
    const double b = beta[(size_t)gk * 32 + lane];
    uint32_t thr[3];
#pragma unroll
    for (int n = 0; n < 3; ++n) {
        const int dE = 2 * z - 4 * n;
        thr[n] = (dE <= 0) ? kAlways : quantize_prob(exp(-b * (double)dE));
    }
    uint32_t *out = planes + (size_t)gk * 128;
    for (int m = 0; m < 32; ++m) {
        const int sh = 31 - m;
        const uint32_t p0 = __ballot_sync(kFull, (thr[0] >> sh) & 1u);
        const uint32_t p1 = __ballot_sync(kFull, (thr[1] >> sh) & 1u);
        const uint32_t p2 = __ballot_sync(kFull, (thr[2] >> sh) & 1u);
        if (lane == 0) {
            out[4 * m + 0] = p0;
            out[4 * m + 1] = p1;
            out[4 * m + 2] = p2;
            out[4 * m + 3] = 0u;
        }
    }
}

constexpr int kMaxSlots = 64;

// One step of the constant-exchange-rate adaptation (Sec. II, PT: the temperatures of every
// realization are moved during equilibration until its exchange rates are equal).  One thread
// per realization.  Pair k accepted xacc of att_k attempts in the window: rate A_k clamped to
// [0.005, 0.995], stiffness s_k = -ln A_k / D_k of its gap D_k; the gaps that equalise the rates
// are D*_k = span (1/s_k) / sum_j (1/s_j); new gaps (1 - eta) D_k + eta D*_k, end points fixed.
// A pair without attempts leaves the realization unchanged.  Counts of the window are cleared.
__global__ void pt_adapt_kernel(double *__restrict__ beta, uint32_t *__restrict__ xacc, int M, int n_real,
                                uint64_t t0, uint64_t t1, double eta) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_real) return;
    const size_t g = r / 32, b = r % 32;
    auto at = [&](int k) -> size_t { return (g * M + k) * 32 + b; };
    bool ok = M >= 3;
    double inv_s[kMaxSlots], gap[kMaxSlots];
    double sum = 0.0;
    for (int k = 0; k + 1 < M; ++k) {
        const uint64_t first = t0 + (uint64_t)(((uint64_t)k - t0) & 1u);  // first t >= t0, t = k (mod 2)
        const uint64_t att = (first >= t1) ? 0 : (t1 - 1 - first) / 2 + 1;
        if (att == 0) ok = false;
        if (!ok) break;
        double a = (double)xacc[at(k)] / (double)att;
        a = a < 0.005 ? 0.005 : (a > 0.995 ? 0.995 : a);
        gap[k] = __dsub_rn(beta[at(k + 1)], beta[at(k)]);
        inv_s[k] = gap[k] / -log(a);
        sum = __dadd_rn(sum, inv_s[k]);
    }
    if (ok) {
        const double span = __dsub_rn(beta[at(M - 1)], beta[at(0)]);
        double bk = beta[at(0)];
        for (int k = 0; k + 2 < M; ++k) {
            const double target = __dmul_rn(span, inv_s[k]) / sum;
            bk = __dadd_rn(bk, __dadd_rn(__dmul_rn(__dsub_rn(1.0, eta), gap[k]), __dmul_rn(eta, target)));
            beta[at(k + 1)] = bk;
        }
    }
    for (int k = 0; k < M; ++k) xacc[at(k)] = 0u;
}

}  // namespace

void pt_release(ea_ctx *ctx) {
    if (!ctx || !ctx->pt) return;
    PtState *p = ctx->pt;
    void *ptrs[] = {p->d_spins, p->d_bonds, p->d_E, p->d_label, p->d_rt, p->d_bounds,
                    p->d_beta, p->d_planes, p->d_xacc, p->d_swaps, p->d_err};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    delete p;
    ctx->pt = nullptr;
}

#define PT_CUDA(call)                                        \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
    } while (0)

// host betas [n_real][M] -> device [g][k][32] (bits past n_real copy the group's first
// realization), then the threshold planes
static int pt_upload_betas(ea_ctx *ctx, const double *betas) {
    PtState *p = ctx->pt;
    const size_t G = p->n_groups, M = p->M;
    std::vector<double> h(G * M * 32);
    for (size_t g = 0; g < G; ++g)
        for (size_t k = 0; k < M; ++k)
            for (size_t b = 0; b < 32; ++b) {
                const size_t r = (32 * g + b < (size_t)p->n_real) ? 32 * g + b : 32 * g;
                h[(g * M + k) * 32 + b] = betas[r * M + k];
            }
    PT_CUDA(cudaMemcpyAsync(p->d_beta, h.data(), h.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
    pt_planes_kernel<<<(int)(G * M), 32, 0, ctx->stream>>>(p->d_beta, p->dim, p->d_planes);
    PT_CUDA(cudaGetLastError());
    PT_CUDA(cudaStreamSynchronize(ctx->stream));
    return EA_OK;
}

extern "C" int pt_init(ea_ctx *ctx, int dim, int L, int n_real, uint32_t rid0, int M, const double *betas,
                       const int8_t *couplings_or_null) {
    if (!ctx) return fail(EA_EINVAL, "null context");
    if (dim != 2 && dim != 3) return fail(EA_EINVAL, "dim must be 2 or 3");
    if (L < 3 || L > 12) return fail(EA_EINVAL, "PT needs L in [3, 12]");
    if (n_real <= 0) return fail(EA_EINVAL, "n_real must be positive");
    if (rid0 % 32) return fail(EA_EINVAL, "rid0 must be a multiple of 32 (realizations are packed 32 per word)");
    if (M < 2 || M > 64) return fail(EA_EINVAL, "M must be in [2, 64]");
    if (!betas) return fail(EA_EINVAL, "null betas");
    for (int k = 0; k + 1 < M; ++k)
        if (!(betas[k + 1] > betas[k])) return fail(EA_EINVAL, "betas must increase with the slot index");
    PT_CUDA(cudaSetDevice(ctx->device));
    pt_release(ctx);
    PtState *p = new PtState();
    ctx->pt = p;
    p->dim = dim;
    p->L = L;
    p->V = volume_of(dim, L);
    p->nb = dim * p->V;
    p->M = M;
    p->n_real = n_real;
    p->n_groups = (n_real + 31) / 32;
    p->rid0 = rid0;
    p->cs = 1;
    // the largest cluster (at most 8 CTAs: 16-CTA clusters measured slower) that splits the
    // slots evenly, for the most CTAs per realization group
    for (int c = 8; c >= 2; --c)
        if (M % c == 0) { p->cs = c; break; }
    const size_t G = p->n_groups;
    auto alloc = [&](void **ptr, size_t bytes) -> int {
        if (cudaMalloc(ptr, bytes) != cudaSuccess) return fail(EA_ENOMEM, "PT allocation of %zu bytes failed", bytes);
        cudaMemsetAsync(*ptr, 0, bytes, ctx->stream);
        return EA_OK;
    };
    int rc;
    if ((rc = alloc((void **)&p->d_spins, G * M * p->V * 4)) || (rc = alloc((void **)&p->d_bonds, G * p->nb * 4)) ||
        (rc = alloc((void **)&p->d_E, G * M * 32 * 4)) || (rc = alloc((void **)&p->d_label, G * M * 32 * 4)) ||
        (rc = alloc((void **)&p->d_rt, G * M * 32 * sizeof(PtRt))) ||
        (rc = alloc((void **)&p->d_bounds, G * 32 * 2 * 4)) || (rc = alloc((void **)&p->d_beta, G * M * 32 * 8)) ||
        (rc = alloc((void **)&p->d_planes, G * M * 128 * 4)) || (rc = alloc((void **)&p->d_xacc, G * M * 32 * 4)) ||
        (rc = alloc((void **)&p->d_swaps, (M - 1) * 8)) || (rc = alloc((void **)&p->d_err, 4))) {
        pt_release(ctx);
        return rc;
    }
    // the same temperatures for every realization; bounds default: never reached
    std::vector<double> hbeta((size_t)n_real * M);
    for (int r = 0; r < n_real; ++r)
        for (int k = 0; k < M; ++k) hbeta[(size_t)r * M + k] = betas[k];
    if ((rc = pt_upload_betas(ctx, hbeta.data()))) return rc;
    void *scr;
    const int8_t *dJ = nullptr;
    if (couplings_or_null) {
        if ((rc = ctx_scratch(ctx, (size_t)n_real * p->nb + 256, &scr))) return rc;
        dJ = (const int8_t *)scr;
        PT_CUDA(cudaMemcpyAsync((void *)dJ, couplings_or_null, (size_t)n_real * p->nb, cudaMemcpyHostToDevice,
                                ctx->stream));
    }
    std::vector<int32_t> hb(G * 32 * 2);
    for (size_t q = 0; q < G * 32; ++q) {
        hb[2 * q] = -(1 << 30);   // e_g: never reached
        hb[2 * q + 1] = 1 << 30;  // e_hot: never reached
    }
    PT_CUDA(cudaMemcpyAsync(p->d_bounds, hb.data(), hb.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    PT_CUDA(pt_dispatch(p, dJ, ctx, 0, 0, 0));
    // round-trip records start at phase 0 with e_min = the initial energy
    std::vector<int32_t> hE(G * M * 32);
    PT_CUDA(cudaMemcpyAsync(hE.data(), p->d_E, hE.size() * 4, cudaMemcpyDeviceToHost, ctx->stream));
    PT_CUDA(cudaStreamSynchronize(ctx->stream));
    std::vector<PtRt> hr(G * M * 32);
    for (size_t gg = 0; gg < G; ++gg)
        for (int k = 0; k < M; ++k)
            for (int b = 0; b < 32; ++b) {
                PtRt &r = hr[(gg * M + k) * 32 + b];  // label k starts at slot k
                r.phase = 0;
                r.n_rt = 0;
                r.t_first = -1;
                r.t_last = -1;
                r.e_min = hE[(gg * M + k) * 32 + b];
                r.pad = 0;
            }
    PT_CUDA(cudaMemcpyAsync(p->d_rt, hr.data(), hr.size() * sizeof(PtRt), cudaMemcpyHostToDevice, ctx->stream));
    PT_CUDA(cudaStreamSynchronize(ctx->stream));
    p->t = 0;
    p->t_win = 0;
    return EA_OK;
}

extern "C" int pt_set_betas(ea_ctx *ctx, const double *betas) {
    if (!ctx || !ctx->pt) return fail(EA_ESTATE, "call pt_init first");
    if (!betas) return fail(EA_EINVAL, "null betas");
    const PtState *p = ctx->pt;
    for (int r = 0; r < p->n_real; ++r)
        for (int k = 0; k + 1 < p->M; ++k)
            if (!(betas[(size_t)r * p->M + k + 1] > betas[(size_t)r * p->M + k]))
                return fail(EA_EINVAL, "betas of realization %d must increase with the slot index", r);
    return pt_upload_betas(ctx, betas);
}

extern "C" int pt_get_betas(ea_ctx *ctx, double *betas) {
    if (!ctx || !ctx->pt) return fail(EA_ESTATE, "call pt_init first");
    if (!betas) return fail(EA_EINVAL, "null output");
    const PtState *p = ctx->pt;
    const size_t G = p->n_groups, M = p->M;
    std::vector<double> h(G * M * 32);
    PT_CUDA(cudaMemcpyAsync(h.data(), p->d_beta, h.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
    PT_CUDA(cudaStreamSynchronize(ctx->stream));
    for (int r = 0; r < p->n_real; ++r)
        for (size_t k = 0; k < M; ++k) betas[(size_t)r * M + k] = h[((r / 32) * M + k) * 32 + r % 32];
    return EA_OK;
}

extern "C" int pt_get_exchange_counts(ea_ctx *ctx, uint32_t *accepted, uint64_t *attempted) {
    if (!ctx || !ctx->pt) return fail(EA_ESTATE, "call pt_init first");
    const PtState *p = ctx->pt;
    const size_t G = p->n_groups, M = p->M;
    if (accepted) {
        std::vector<uint32_t> h(G * M * 32);
        PT_CUDA(cudaMemcpyAsync(h.data(), p->d_xacc, h.size() * 4, cudaMemcpyDeviceToHost, ctx->stream));
        PT_CUDA(cudaStreamSynchronize(ctx->stream));
        for (int r = 0; r < p->n_real; ++r)
            for (size_t k = 0; k + 1 < M; ++k) accepted[(size_t)r * (M - 1) + k] = h[((r / 32) * M + k) * 32 + r % 32];
    }
    if (attempted)
        for (size_t k = 0; k + 1 < M; ++k) {
            const uint64_t first = p->t_win + ((k - p->t_win) & 1u);
            attempted[k] = (first >= p->t) ? 0 : (p->t - 1 - first) / 2 + 1;
        }
    return EA_OK;
}

extern "C" int pt_adapt(ea_ctx *ctx, double eta) {
    if (!ctx || !ctx->pt) return fail(EA_ESTATE, "call pt_init first");
    if (!(eta >= 0.0 && eta <= 1.0)) return fail(EA_EINVAL, "eta must be in [0, 1]");
    PtState *p = ctx->pt;
    pt_adapt_kernel<<<(p->n_real + 127) / 128, 128, 0, ctx->stream>>>(p->d_beta, p->d_xacc, p->M, p->n_real,
                                                                       p->t_win, p->t, eta);
    PT_CUDA(cudaGetLastError());
    pt_planes_kernel<<<p->n_groups * p->M, 32, 0, ctx->stream>>>(p->d_beta, p->dim, p->d_planes);
    PT_CUDA(cudaGetLastError());
    PT_CUDA(cudaStreamSynchronize(ctx->stream));
    p->t_win = p->t;
    return EA_OK;
}

extern "C" int pt_set_rt_bounds(ea_ctx *ctx, const int32_t *e_g, const int32_t *e_hot) {
    if (!ctx || !ctx->pt) return fail(EA_ESTATE, "call pt_init first");
    if (!e_g || !e_hot) return fail(EA_EINVAL, "null bounds");
    PtState *p = ctx->pt;
    std::vector<int32_t> hb((size_t)p->n_groups * 64, 0);
    for (size_t q = 0; q < (size_t)p->n_groups * 32; ++q) {
        const bool in = q < (size_t)p->n_real;
        hb[2 * q] = in ? e_g[q] : -(1 << 30);
        hb[2 * q + 1] = in ? e_hot[q] : (1 << 30);
    }
    PT_CUDA(cudaMemcpyAsync(p->d_bounds, hb.data(), hb.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    PT_CUDA(cudaStreamSynchronize(ctx->stream));
    return EA_OK;
}

extern "C" int pt_run(ea_ctx *ctx, uint64_t n_sweeps, int count_roundtrips) {
    if (!ctx || !ctx->pt) return fail(EA_ESTATE, "call pt_init first");
    PtState *p = ctx->pt;
    if (p->t + n_sweeps > (1ull << 32)) return fail(EA_EINVAL, "sweep counter would exceed 2^32");
    if (n_sweeps == 0) return EA_OK;
    PT_CUDA(pt_dispatch(p, nullptr, ctx, 1, n_sweeps, count_roundtrips));
    p->t += n_sweeps;
    return EA_OK;
}

extern "C" int pt_get_state(ea_ctx *ctx, int8_t *spins, int32_t *E, int32_t *labels, uint64_t *t) {
    if (!ctx || !ctx->pt) return fail(EA_ESTATE, "call pt_init first");
    PtState *p = ctx->pt;
    const size_t G = p->n_groups, M = p->M, V = p->V;
    std::vector<uint32_t> hs;
    std::vector<int32_t> hE(G * M * 32), hL(G * M * 32);
    if (spins) {
        hs.resize(G * M * V);
        PT_CUDA(cudaMemcpyAsync(hs.data(), p->d_spins, hs.size() * 4, cudaMemcpyDeviceToHost, ctx->stream));
    }
    PT_CUDA(cudaMemcpyAsync(hE.data(), p->d_E, hE.size() * 4, cudaMemcpyDeviceToHost, ctx->stream));
    PT_CUDA(cudaMemcpyAsync(hL.data(), p->d_label, hL.size() * 4, cudaMemcpyDeviceToHost, ctx->stream));
    PT_CUDA(cudaStreamSynchronize(ctx->stream));
    for (int r = 0; r < p->n_real; ++r) {
        const size_t g = r / 32, b = r % 32;
        for (size_t k = 0; k < M; ++k) {
            if (E) E[r * M + k] = hE[(g * M + k) * 32 + b];
            if (labels) labels[r * M + k] = hL[(g * M + k) * 32 + b];
            if (spins)
                for (size_t i = 0; i < V; ++i)
                    spins[(r * M + k) * V + i] = ((hs[(g * M + k) * V + i] >> b) & 1u) ? -1 : 1;
        }
    }
    if (t) *t = p->t;
    return EA_OK;
}

extern "C" int pt_get_roundtrips(ea_ctx *ctx, ea_pt_stats *out, int reset) {
    if (!ctx || !ctx->pt) return fail(EA_ESTATE, "call pt_init first");
    if (!out) return fail(EA_EINVAL, "null output");
    PtState *p = ctx->pt;
    const size_t G = p->n_groups, M = p->M;
    std::vector<PtRt> hr(G * M * 32);
    PT_CUDA(cudaMemcpyAsync(hr.data(), p->d_rt, hr.size() * sizeof(PtRt), cudaMemcpyDeviceToHost, ctx->stream));
    PT_CUDA(cudaStreamSynchronize(ctx->stream));
    for (int r = 0; r < p->n_real; ++r) {
        const size_t g = r / 32, b = r % 32;
        for (size_t l = 0; l < M; ++l) {
            const PtRt &s = hr[(g * M + l) * 32 + b];
            ea_pt_stats &o = out[r * M + l];
            o.n_rt = s.n_rt;
            o.phase = s.phase;
            o.t_first = s.t_first;
            o.t_last = s.t_last;
            o.e_min = s.e_min;
            o.pad = 0;
        }
    }
    if (reset) {
        std::vector<int32_t> hE(G * M * 32), hL(G * M * 32);
        PT_CUDA(cudaMemcpyAsync(hE.data(), p->d_E, hE.size() * 4, cudaMemcpyDeviceToHost, ctx->stream));
        PT_CUDA(cudaMemcpyAsync(hL.data(), p->d_label, hL.size() * 4, cudaMemcpyDeviceToHost, ctx->stream));
        PT_CUDA(cudaStreamSynchronize(ctx->stream));
        for (size_t g = 0; g < G; ++g)
            for (size_t k = 0; k < M; ++k)
                for (int b = 0; b < 32; ++b) {
                    const int lbl = hL[(g * M + k) * 32 + b];
                    PtRt &s = hr[(g * M + lbl) * 32 + b];
                    s.phase = 0;
                    s.n_rt = 0;
                    s.t_first = -1;
                    s.t_last = -1;
                    s.e_min = hE[(g * M + k) * 32 + b];
                }
        PT_CUDA(cudaMemcpyAsync(p->d_rt, hr.data(), hr.size() * sizeof(PtRt), cudaMemcpyHostToDevice, ctx->stream));
        PT_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    return EA_OK;
}

extern "C" int pt_get_swap_counts(ea_ctx *ctx, uint64_t *out) {
    if (!ctx || !ctx->pt) return fail(EA_ESTATE, "call pt_init first");
    if (!out) return fail(EA_EINVAL, "null output");
    PtState *p = ctx->pt;
    PT_CUDA(cudaMemcpyAsync(out, p->d_swaps, (p->M - 1) * 8, cudaMemcpyDeviceToHost, ctx->stream));
    PT_CUDA(cudaStreamSynchronize(ctx->stream));
    return EA_OK;
}
