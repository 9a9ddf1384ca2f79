// muca_kernels.cu -- sm_103a kernels of the multicanonical (MUCA) hot path.
//
//   init_kernel            a1: disorder, initial spins, energy, descent to E <= E_top
//   (the sweep kernel itself, a2+a3, is in muca_sweep.cu)
//   update_weights_kernel  a4: W <- W P_SH / H (Sec. II iterative procedure), FP64
//   quantize_kernel        a4: ln W -> u32 acceptance thresholds
//   build_ensemble_kernel  a5: flat / power-law / 1/k / canonical weights from ln Omega
//
// One warp = one tile of up to 32 chains of equal (dim, L); in global memory the tile's lattice
// is multi-spin coded (bit `lane` of each word is chain `lane`).
#include <cuda_runtime.h>

#include <cstdint>

#include "eamc_internal.cuh"

namespace eamc {

namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;

// neighbour of site i along d (0..DIM-1) with sign +-1, from coordinates
template <int DIM>
__device__ __forceinline__ int nbr(int i, int L, int d, int sign) {
    int c[3] = {i % L, (i / L) % L, DIM == 3 ? i / (L * L) : 0};
    c[d] = (c[d] + sign + L) % L;
    return c[0] + L * c[1] + L * L * c[2];
}

// ------------------------------------------------------------------------------ a1
// One warp per tile.  Couplings and spins are drawn per lane from the chain's Philox
// counters (or read from the caller's arrays), assembled into words with a ballot, then
// each lane computes u (unsatisfied bonds) and descends to E <= E_top.
template <int DIM>
__global__ void __launch_bounds__(32)
init_kernel(const TileDesc *__restrict__ tiles, int tile0, SlotState *__restrict__ slots,
            uint32_t *__restrict__ spins, uint32_t *__restrict__ bonds,
            const int8_t *__restrict__ Jin, const int8_t *__restrict__ Sin, int in_row0,
            PhiloxKey key, int *__restrict__ err) {
    const int tile = tile0 + blockIdx.x;
    const TileDesc td = tiles[tile];
    const int lane = threadIdx.x;
    const int L = td.L, V = td.V, nb = DIM * V;
    SlotState ss = slots[tile * kTile + lane];
    const bool active = lane < td.n_active;
    const int row = in_row0 + blockIdx.x * td.width + lane;  // row in the caller's arrays
    uint32_t *sp = spins + td.spin_off;
    uint32_t *bd = bonds + td.bond_off;

    int negatives = 0;
    for (int j0 = 0; j0 < nb; j0 += 4) {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)(j0 >> 2), 0u, ss.rid, 3u), key);
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int j = j0 + jj;
            if (j < nb) {
                const bool neg =
                    active && (Jin ? (Jin[(size_t)row * nb + j] < 0) : ((uint4_get(w, jj) >> 31) != 0));
                negatives += neg;
                const uint32_t m = __ballot_sync(kFull, neg);
                if (lane == 0) bd[j] = m;
            }
        }
    }
    for (int i0 = 0; i0 < V; i0 += 4) {
        const uint4 w = philox4x32_10(
            make_uint4((uint32_t)(i0 >> 2), 0u, ss.rid, 2u | (ss.stream << 8)), key);
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int i = i0 + jj;
            if (i < V) {
                const bool neg =
                    active && (Sin ? (Sin[(size_t)row * V + i] < 0) : ((uint4_get(w, jj) >> 31) != 0));
                const uint32_t m = __ballot_sync(kFull, neg);
                if (lane == 0) sp[i] = m;
            }
        }
    }
    __syncwarp();

    // unsatisfied count of this lane's chain at site i
    auto unsat_at = [&](int i) -> int {
        uint32_t u[2 * DIM];
        const uint32_t si = sp[i];
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const int jp = nbr<DIM>(i, L, d, +1), jm = nbr<DIM>(i, L, d, -1);
            u[2 * d] = si ^ sp[jp] ^ bd[i * DIM + d];
            u[2 * d + 1] = si ^ sp[jm] ^ bd[jm * DIM + d];
        }
        int n = 0;
#pragma unroll
        for (int k = 0; k < 2 * DIM; ++k) n += (u[k] >> lane) & 1u;
        return n;
    };

    int u = 0;
    for (int i = 0; i < V; ++i)
        for (int d = 0; d < DIM; ++d) {
            const uint32_t w = sp[i] ^ sp[nbr<DIM>(i, L, d, +1)] ^ bd[i * DIM + d];
            u += (w >> lane) & 1u;
        }
    int E = 2 * u - nb;
    const int parity = negatives & 1;
    const int btop = top_bin(nb, parity);
    const int etop = energy_of_bin(nb, parity, btop);
    bool stuck = false;
    while (__any_sync(kFull, active && !stuck && E > etop)) {
        bool flipped = false;
        for (int i = 0; i < V; ++i) {
            const int n = unsat_at(i);
            const int dE = 2 * (2 * DIM) - 4 * n;
            const bool want = active && !stuck && E > etop && dE < 0;
            const uint32_t m = __ballot_sync(kFull, want);
            __syncwarp();
            if (lane == 0 && m) sp[i] ^= m;
            __syncwarp();
            if (want) { E += dE; flipped = true; }
        }
        if (active && E > etop && !flipped) stuck = true;
    }
    if (stuck) atomicExch(err, 1);
    const bool ok = active && !stuck;  // a stuck chain stays inactive (E above the wall)

    if (ok) {
        ss.parity = parity;
        ss.b_top = btop;
        ss.b = bin_of_energy(nb, E);
        ss.b_min = ss.b;
    } else {
        ss.parity = 0;
        ss.b_top = 0;
        ss.b = 0;
        ss.b_min = 0;
    }
    ss.b_g = kNoBottom;
    ss.e_g = -(1 << 30);
    ss.phase = 0;
    ss.n_rt = 0;
    ss.t_first = -1;
    ss.t_last = -1;
    ss.t = 0;
    ss.requeue = 0;
    ss.active = ok ? 1 : 0;
    slots[tile * kTile + lane] = ss;
}

// ------------------------------------------------------------------------------ a4
__device__ __forceinline__ double ln_profile(int kind, double alpha, double pole, int e_g, int E) {
    if (kind != 1) return 0.0;
    const double Ec = (E < e_g) ? (double)e_g : (double)E;
    return alpha * log(Ec / (pole - (double)e_g) + 1.0);
}

// one block per chain; threads over bins
__device__ void update_weights_one(const TileDesc *__restrict__ tiles, SlotState *__restrict__ slots,
                                   double *__restrict__ lnW, uint32_t *__restrict__ hist,
                                   double2 *__restrict__ acc, int slot);

__global__ void update_weights_kernel(const TileDesc *__restrict__ tiles,
                                      SlotState *__restrict__ slots, double *__restrict__ lnW,
                                      uint32_t *__restrict__ hist, double2 *__restrict__ acc) {
    update_weights_one(tiles, slots, lnW, hist, acc, blockIdx.x);
}

__global__ void update_weights_sel_kernel(const TileDesc *__restrict__ tiles, SlotState *__restrict__ slots,
                                          double *__restrict__ lnW, uint32_t *__restrict__ hist,
                                          double2 *__restrict__ acc, const int32_t *__restrict__ slot_of) {
    update_weights_one(tiles, slots, lnW, hist, acc, slot_of[blockIdx.x]);
}

// Largest table row count: 3D, L = 12 -> (3 * 1728 / 2 >> 1) + 1 bins.
constexpr int kMaxRows = 1297;

// Berg's accumulated error-weighted recursion (B. A. Berg, J. Stat. Phys. 82, 323 (1996), one of
// the iterative procedures Sec. II refers to).  Per pair of neighbouring bins (b, b+1) that were
// both visited this iteration, s = [ln H(b+1) - ln W(b+1)] - [ln H(b) - ln W(b)] estimates
// ln Omega(b+1) - ln Omega(b) with inverse variance g = H(b) H(b+1) / (H(b) + H(b+1));
// acc[b] = {D, G} holds the g-weighted mean of all estimates and the sum of the g.  New weights:
// ln W(b) - ln W(b+1) = ln P_SH(b) - ln P_SH(b+1) + D(b) where G(b) > 0, the plain step's
// difference elsewhere, ln W(b_top) = 0.  Weights constant over the range add no estimates (the
// sweep is then deterministic, every move inside the range being accepted).  A pair of which the
// iteration visited exactly one bin although the accumulated estimate expected at least 10 counts
// on the other side starts over: weights that confine the chain to one side would otherwise
// never be corrected.
__device__ void update_weights_berg(const TileDesc &td, const SlotState &ss, double *__restrict__ w,
                                    const uint32_t *__restrict__ h, double2 *__restrict__ acc, int e_g) {
    __shared__ double diff[kMaxRows];
    const int nb = td.dim * td.V, bt = ss.b_top;
    int changed = 0;
    for (int b = threadIdx.x; b < bt; b += blockDim.x) changed |= (w[b] != w[bt]);
    const bool informative = __syncthreads_or(changed) != 0;
    for (int b = threadIdx.x; b < bt; b += blockDim.x) {
        const double lp0 = ln_profile(ss.kind, ss.alpha, ss.pole, e_g, energy_of_bin(nb, ss.parity, b));
        const double lp1 = ln_profile(ss.kind, ss.alpha, ss.pole, e_g, energy_of_bin(nb, ss.parity, b + 1));
        const uint32_t c0 = h[b], c1 = h[b + 1];
        double2 a = acc[b];
        if (informative && c0 > 0u && c1 > 0u) {
            const double h0 = (double)c0, h1 = (double)c1;
            const double s = __dsub_rn(__dsub_rn(log(h1), w[b + 1]), __dsub_rn(log(h0), w[b]));
            const double g = __ddiv_rn(__dmul_rn(h0, h1), __dadd_rn(h0, h1));
            a.x = __ddiv_rn(__dadd_rn(__dmul_rn(a.y, a.x), __dmul_rn(g, s)), __dadd_rn(a.y, g));
            a.y = __dadd_rn(a.y, g);
            acc[b] = a;
        } else if (informative && a.y > 0.0 && ((c0 > 0u) != (c1 > 0u))) {
            // the chain stayed on one side of the pair although the accumulated estimate
            // expected at least 10 counts on the other: start the pair over (plain step now)
            const double lnexp = (c0 > 0u)
                ? __dadd_rn(__dadd_rn(log((double)c0), a.x), __dsub_rn(w[b + 1], w[b]))
                : __dadd_rn(__dsub_rn(log((double)c1), a.x), __dsub_rn(w[b], w[b + 1]));
            if (lnexp >= 2.302585092994046) {  // ln 10
                a = make_double2(0.0, 0.0);
                acc[b] = a;
            }
        }
        if (a.y > 0.0) {
            diff[b] = __dadd_rn(__dsub_rn(lp0, lp1), a.x);
        } else {
            const double a0 = w[b] + lp0 - log(c0 > 0u ? (double)c0 : 1.0);
            const double a1 = w[b + 1] + lp1 - log(c1 > 0u ? (double)c1 : 1.0);
            diff[b] = a0 - a1;
        }
    }
    __syncthreads();
    // every thread has read the old w it needs; the suffix sum runs in the order of the
    // definition (top bin down), O(bins) on one thread per chain
    if (threadIdx.x == 0) {
        double v = 0.0;
        w[bt] = 0.0;
        for (int b = bt - 1; b >= 0; --b) {
            v = __dadd_rn(v, diff[b]);
            w[b] = v;
        }
    }
}

__device__ void update_weights_one(const TileDesc *__restrict__ tiles, SlotState *__restrict__ slots,
                                   double *__restrict__ lnW, uint32_t *__restrict__ hist,
                                   double2 *__restrict__ acc, int slot) {
    const TileDesc td = tiles[slot / kTile];
    const int lane = slot % kTile;
    SlotState ss = slots[slot];
    if (!ss.active || (ss.kind != 0 && ss.kind != 1)) return;
    const int nb = td.dim * td.V;
    const int e_g = energy_of_bin(nb, ss.parity, ss.b_min);
    double *w = lnW + td.w_base + (uint64_t)lane * td.B;
    uint32_t *h = hist + td.w_base + (uint64_t)lane * td.B;
    if (ss.recursion == 1 && acc) {
        update_weights_berg(td, ss, w, h, acc + td.w_base + (uint64_t)lane * td.B, e_g);
        __syncthreads();
        for (int b = threadIdx.x; b <= ss.b_top; b += blockDim.x) h[b] = 0u;
        if (threadIdx.x == 0) {
            ss.e_g = e_g;
            ss.b_g = ss.b_min;
            slots[slot] = ss;
        }
        return;
    }
    auto next = [&](int b) {
        const int E = energy_of_bin(nb, ss.parity, b);
        const double hb = h[b] > 0u ? (double)h[b] : 1.0;
        return w[b] + ln_profile(ss.kind, ss.alpha, ss.pole, e_g, E) - log(hb);
    };
    const double top = next(ss.b_top);
    __syncthreads();
    // every thread read what it needs (w[b], h[b] of its own bins, and the top bin)
    // before any write; the top value is recomputed, so no second pass is needed
    for (int b = threadIdx.x; b <= ss.b_top; b += blockDim.x) {
        const double v = next(b) - top;
        w[b] = v;
    }
    __syncthreads();
    for (int b = threadIdx.x; b <= ss.b_top; b += blockDim.x) h[b] = 0u;
    if (threadIdx.x == 0) {
        ss.e_g = e_g;
        ss.b_g = ss.b_min;
        slots[slot] = ss;
    }
}

__device__ __forceinline__ void quantize_one(const TileDesc *__restrict__ tiles,
                                             const SlotState *__restrict__ slots,
                                             const double *__restrict__ lnW, uint32_t *__restrict__ thr,
                                             int slot) {
    const TileDesc td = tiles[slot / kTile];
    const int lane = slot % kTile;
    const SlotState ss = slots[slot];
    const double *w = lnW + td.w_base + (uint64_t)lane * td.B;
    uint32_t *t = thr + (td.w_base + (uint64_t)lane * td.B) * 8;
    const int dim = td.dim, btop = ss.active ? ss.b_top : -1;
    for (int b = threadIdx.x; b < td.B; b += blockDim.x) {
        uint32_t v[8];
#pragma unroll
        for (int n = 0; n < 8; ++n) {
            v[n] = 0u;
            const int bn = b + dim - n;
            if (b <= btop && n <= 2 * dim && bn >= 0 && bn <= btop) {
                const double x = w[bn] - w[b];
                if (x >= 0.0) {
                    v[n] = kAlways;
                } else {
                    const double q = floor(exp(x) * 4294967296.0);
                    v[n] = (q >= 4294967294.0) ? 0xFFFFFFFEu : (uint32_t)q;
                }
            }
        }
        uint4 *dst = reinterpret_cast<uint4 *>(t + (size_t)b * 8);
        dst[0] = make_uint4(v[0], v[1], v[2], v[3]);
        dst[1] = make_uint4(v[4], v[5], v[6], v[7]);
    }
}

__global__ void quantize_kernel(const TileDesc *__restrict__ tiles,
                                const SlotState *__restrict__ slots,
                                const double *__restrict__ lnW, uint32_t *__restrict__ thr) {
    quantize_one(tiles, slots, lnW, thr, blockIdx.x);
}

// ------------------------------------------------------------------------------ a5
// one thread per selected chain: ln Omega from the current weights, then the new ensemble
__global__ void build_ensemble_kernel(const TileDesc *__restrict__ tiles, int n_slots,
                                      SlotState *__restrict__ slots,
                                      const uint8_t *__restrict__ sel, int kind, double alpha,
                                      double pole, double beta, double *__restrict__ lnW) {
    const int slot = blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= n_slots || !sel[slot]) return;
    const TileDesc td = tiles[slot / kTile];
    const int lane = slot % kTile;
    SlotState ss = slots[slot];
    if (!ss.active) return;
    const int nb = td.dim * td.V;
    double *w = lnW + td.w_base + (uint64_t)lane * td.B;
    const int e_g = (ss.b_g == kNoBottom) ? energy_of_bin(nb, ss.parity, ss.b_min) : ss.e_g;
    // ln Omega in place: lnO = lnP(current kind) - lnW
    for (int b = 0; b <= ss.b_top; ++b)
        w[b] = ln_profile(ss.kind, ss.alpha, ss.pole, e_g, energy_of_bin(nb, ss.parity, b)) - w[b];
    int bg = bin_of_energy(nb, e_g);
    bg = bg < 0 ? 0 : (bg > ss.b_top ? ss.b_top : bg);  // E_g outside the range: clamp
    if (kind == 0) {
        for (int b = 0; b <= ss.b_top; ++b) w[b] = -w[b];
    } else if (kind == 1) {
        for (int b = 0; b <= ss.b_top; ++b)
            w[b] = ln_profile(1, alpha, pole, e_g, energy_of_bin(nb, ss.parity, b)) - w[b];
    } else if (kind == 2) {
        const double lnO_bg = w[bg];
        double acc = w[bg];
        for (int b = bg; b <= ss.b_top; ++b) {
            if (b > bg) {  // acc = log(exp(acc) + exp(lnO(b)))
                const double o = w[b];
                const double m = acc > o ? acc : o;
                acc = m + log(exp(acc - m) + exp(o - m));
            }
            w[b] = -acc;
        }
        for (int b = 0; b < bg && b <= ss.b_top; ++b) w[b] = w[bg] + lnO_bg - w[b];
    } else {
        for (int b = 0; b <= ss.b_top; ++b)
            w[b] = -beta * (double)energy_of_bin(nb, ss.parity, b);
    }
    const double top = w[ss.b_top];
    for (int b = 0; b <= ss.b_top; ++b) w[b] -= top;
    ss.kind = kind;
    ss.alpha = alpha;
    ss.pole = pole;
    ss.beta = beta;
    if (ss.b_g == kNoBottom) { ss.e_g = e_g; ss.b_g = bin_of_energy(nb, e_g); }
    slots[slot] = ss;
}

// injected tables: every move leaving [0, b_top] (and every unused class) becomes a wall,
// so a chain's bin never leaves its rows whatever the caller wrote
__global__ void enforce_walls_kernel(const TileDesc *__restrict__ tiles,
                                     const SlotState *__restrict__ slots, uint32_t *__restrict__ thr) {
    const int slot = blockIdx.x;
    const TileDesc td = tiles[slot / kTile];
    const int lane = slot % kTile;
    const SlotState ss = slots[slot];
    uint32_t *t = thr + (td.w_base + (uint64_t)lane * td.B) * 8;
    const int btop = ss.active ? ss.b_top : -1;
    for (int k = threadIdx.x; k < td.B * 8; k += blockDim.x) {
        const int b = k >> 3, n = k & 7, bn = b + td.dim - n;
        if (b > btop || n > 2 * td.dim || bn < 0 || bn > btop) t[k] = 0u;
    }
}

// Re-initialises single chains in place (serving: a freed lane takes a new job).  One warp
// per chain; only the chain's own bit of each tile word changes (atomic and / or), so the
// other lanes of the tile are untouched.  Couplings and spins come from the chain's new
// (rid, stream) exactly as in init_kernel, then lane 0 descends to E <= E_top.
template <int DIM>
__global__ void reset_lane_kernel(const TileDesc *__restrict__ tiles, SlotState *__restrict__ slots,
                                  uint32_t *__restrict__ spins, uint32_t *__restrict__ bonds,
                                  double *__restrict__ lnW, uint32_t *__restrict__ hist,
                                  const int32_t *__restrict__ slot_of, const uint32_t *__restrict__ rids,
                                  const uint32_t *__restrict__ streams, PhiloxKey key, int *__restrict__ err) {
    const int slot = slot_of[blockIdx.x];
    const int tile = slot / kTile, who = slot % kTile, lane = threadIdx.x;
    const TileDesc td = tiles[tile];
    const int L = td.L, V = td.V, nb = DIM * V;
    const uint32_t rid = rids[blockIdx.x], stream = streams[blockIdx.x];
    const uint32_t bit = 1u << who;
    uint32_t *sp = spins + td.spin_off;
    uint32_t *bd = bonds + td.bond_off;
    int negatives = 0;
    for (int j0 = 4 * lane; j0 < nb; j0 += 128) {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)(j0 >> 2), 0u, rid, 3u), key);
        for (int jj = 0; jj < 4 && j0 + jj < nb; ++jj) {
            const bool neg = (uint4_get(w, jj) >> 31) != 0;
            negatives += neg;
            if (neg) atomicOr(&bd[j0 + jj], bit);
            else atomicAnd(&bd[j0 + jj], ~bit);
        }
    }
    for (int i0 = 4 * lane; i0 < V; i0 += 128) {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)(i0 >> 2), 0u, rid, 2u | (stream << 8)), key);
        for (int jj = 0; jj < 4 && i0 + jj < V; ++jj) {
            if ((uint4_get(w, jj) >> 31) != 0) atomicOr(&sp[i0 + jj], bit);
            else atomicAnd(&sp[i0 + jj], ~bit);
        }
    }
    for (int off = 16; off > 0; off >>= 1) negatives += __shfl_xor_sync(0xFFFFFFFFu, negatives, off);
    __syncwarp();
    __threadfence_block();
    double *w = lnW + td.w_base + (uint64_t)who * td.B;
    uint32_t *h = hist + td.w_base + (uint64_t)who * td.B;
    for (int b = lane; b < td.B; b += 32) { w[b] = 0.0; h[b] = 0u; }
    if (lane != 0) return;
    auto spin = [&](int i) { return (sp[i] >> who) & 1u; };
    auto unsat_at = [&](int i) {
        int n = 0;
        for (int d = 0; d < DIM; ++d) {
            const int jp = nbr<DIM>(i, L, d, +1), jm = nbr<DIM>(i, L, d, -1);
            n += (int)(spin(i) ^ spin(jp) ^ ((bd[i * DIM + d] >> who) & 1u));
            n += (int)(spin(i) ^ spin(jm) ^ ((bd[jm * DIM + d] >> who) & 1u));
        }
        return n;
    };
    int u = 0;
    for (int i = 0; i < V; ++i)
        for (int d = 0; d < DIM; ++d)
            u += (int)(spin(i) ^ spin(nbr<DIM>(i, L, d, +1)) ^ ((bd[i * DIM + d] >> who) & 1u));
    int E = 2 * u - nb;
    const int parity = negatives & 1;
    const int btop = top_bin(nb, parity);
    const int etop = energy_of_bin(nb, parity, btop);
    bool stuck = false;
    while (E > etop && !stuck) {
        bool flipped = false;
        for (int i = 0; i < V && E > etop; ++i) {
            const int dE = 2 * (2 * DIM) - 4 * unsat_at(i);
            if (dE < 0) { atomicXor(&sp[i], bit); E += dE; flipped = true; }
        }
        if (E > etop && !flipped) stuck = true;
    }
    SlotState ss = slots[slot];
    ss.rid = rid;
    ss.stream = stream;
    ss.parity = parity;
    ss.b_top = btop;
    ss.b = stuck ? 0 : bin_of_energy(nb, E);
    ss.b_min = ss.b;
    ss.b_g = kNoBottom;
    ss.e_g = -(1 << 30);
    ss.phase = 0;
    ss.n_rt = 0;
    ss.t_first = -1;
    ss.t_last = -1;
    ss.t = 0;
    ss.requeue = 0;
    ss.kind = 0;
    ss.recursion = 0;
    ss.active = stuck ? 0 : 1;
    slots[slot] = ss;
    if (stuck) atomicExch(err, 1);
}

// weight update of selected chains only (serving: jobs reach iteration boundaries at
// different times)

__global__ void reset_rt_kernel(const TileDesc *__restrict__ tiles, int n_slots,
                                SlotState *__restrict__ slots, const uint8_t *__restrict__ sel) {
    const int slot = blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= n_slots || !sel[slot]) return;
    SlotState ss = slots[slot];
    ss.phase = 0;
    ss.n_rt = 0;
    ss.t_first = -1;
    ss.t_last = -1;
    ss.requeue = 0;
    ss.b_min = ss.b;
    slots[slot] = ss;
}

// ------------------------------------------------------------------------------ a9 serving
// Per-tick control of the served jobs, one thread per slot, after the tick's sweep launch.  A
// job's schedule is counted in its own ticks (every tick adds its sweeps_per_tick sweeps to the
// chain), so what a job computes does not depend on the jobs that share the device:
//   iterate: every ticks_per_step ticks one weight step (Sec. II); after iter_steps steps the
//            round-trip record restarts with E_g = the lowest energy seen and production begins;
//   produce: a chain that went below E_g is requeued (Sec. III: new E_g, one more weight step,
//            counting restarts) up to max_requeues times; the job is done at rt_target round
//            trips, censored after max_prod_ticks production ticks;
//   a descent that got stuck at admission leaves the chain inactive: the job fails.
// A finished job writes one record into the completion ring and its chain stops.
__global__ void srv_control_kernel(const TileDesc *__restrict__ tiles, int n_slots, SlotState *__restrict__ slots,
                                   JobCtl *__restrict__ ctl, int32_t *__restrict__ flag,
                                   SrvRecord *__restrict__ ring, uint32_t *__restrict__ head, uint32_t ring_cap,
                                   unsigned long long *__restrict__ attempts, uint64_t tick) {
    const int slot = blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= n_slots) return;
    flag[slot] = 0;
    JobCtl c = ctl[slot];
    if (c.phase != kJobIterate && c.phase != kJobProduce) return;
    SlotState ss = slots[slot];
    const TileDesc td = tiles[slot / kTile];
    const int nb = td.dim * td.V;
    int status = 0, f = 0;
    if (!ss.active) {
        status = kJobFailed;
    } else {
        c.ticks += 1;
        atomicAdd(attempts, (unsigned long long)td.V * (unsigned long long)c.sweeps_per_tick);
        if (c.phase == kJobIterate) {
            if (c.ticks % c.ticks_per_step == 0) {
                f = kFlagUpdate;
                c.steps_done += 1;
                if (c.steps_done >= c.iter_steps) {
                    f |= kFlagResetRt;
                    c.phase = kJobProduce;
                    c.prod_ticks = 0;
                }
            }
        } else {
            c.prod_ticks += 1;
            if (ss.requeue && c.requeues < c.max_requeues) {
                f = kFlagUpdate | kFlagResetRt;
                c.requeues += 1;
                c.prod_ticks = 0;
            } else if (ss.n_rt >= c.rt_target) {
                status = kJobDone;
            } else if (c.prod_ticks >= c.max_prod_ticks) {
                status = kJobCensored;
            }
        }
    }
    if (status) {
        SrvRecord r;
        r.job = c.job;
        r.status = status;
        r.slot = slot;
        r.n_rt = ss.n_rt;
        r.requeues = c.requeues;
        r.t_first = ss.t_first;
        r.t_last = ss.t_last;
        r.e_g = ss.e_g;
        r.e_min = energy_of_bin(nb, ss.parity, ss.b_min);
        r.sweeps = ss.t;
        r.tick = tick;
        const uint32_t k = atomicAdd(head, 1u);
        ring[k % ring_cap] = r;
        c.phase = kJobFinished;
        ss.active = 0;
        slots[slot] = ss;
    }
    flag[slot] = f;
    ctl[slot] = c;
}

// weight step of the flagged slots (block per slot), then the round-trip record restarts where
// asked: phase 0, no round trips, the lowest energy from now on; E_g stays as the step set it
__global__ void srv_update_kernel(const TileDesc *__restrict__ tiles, SlotState *__restrict__ slots,
                                  double *__restrict__ lnW, uint32_t *__restrict__ hist,
                                  double2 *__restrict__ acc, const int32_t *__restrict__ flag) {
    const int slot = blockIdx.x;
    const int f = flag[slot];
    if (!(f & kFlagUpdate)) return;
    update_weights_one(tiles, slots, lnW, hist, acc, slot);
    if (!(f & kFlagResetRt)) return;
    __syncthreads();
    if (threadIdx.x == 0) {
        SlotState ss = slots[slot];
        ss.phase = 0;
        ss.n_rt = 0;
        ss.t_first = -1;
        ss.t_last = -1;
        ss.requeue = 0;
        ss.b_min = ss.b;
        slots[slot] = ss;
    }
}

__global__ void quantize_flagged_kernel(const TileDesc *__restrict__ tiles, const SlotState *__restrict__ slots,
                                        const double *__restrict__ lnW, uint32_t *__restrict__ thr,
                                        const int32_t *__restrict__ flag) {
    if (flag[blockIdx.x] == 0) return;
    quantize_one(tiles, slots, lnW, thr, blockIdx.x);
}

// an admitted job: ensemble and recursion of its (freshly reset) chain, empty Berg
// accumulators, the job's schedule; its thresholds are quantised next
__global__ void srv_start_kernel(const TileDesc *__restrict__ tiles, SlotState *__restrict__ slots,
                                 JobCtl *__restrict__ ctl, int32_t *__restrict__ flag, double2 *__restrict__ acc,
                                 const SrvStart *__restrict__ start) {
    const SrvStart j = start[blockIdx.x];
    const int slot = j.slot;
    const TileDesc td = tiles[slot / kTile];
    if (acc) {
        double2 *a = acc + td.w_base + (uint64_t)(slot % kTile) * td.B;
        for (int b = threadIdx.x; b < td.B; b += blockDim.x) a[b] = make_double2(0.0, 0.0);
    }
    if (threadIdx.x != 0) return;
    SlotState ss = slots[slot];
    ss.kind = j.kind;
    ss.alpha = j.alpha;
    ss.pole = j.pole;
    ss.recursion = j.recursion;
    slots[slot] = ss;
    JobCtl c;
    c.job = j.job;
    c.phase = kJobIterate;
    c.sweeps_per_tick = j.sweeps_per_tick;
    c.ticks = 0;
    c.steps_done = 0;
    c.iter_steps = j.iter_steps;
    c.ticks_per_step = j.ticks_per_step;
    c.prod_ticks = 0;
    c.max_prod_ticks = j.max_prod_ticks;
    c.requeues = 0;
    c.max_requeues = j.max_requeues;
    c.rt_target = j.rt_target;
    c.pad = 0;
    ctl[slot] = c;
    flag[slot] = kFlagQuantize;
}

__global__ void srv_cancel_kernel(SlotState *__restrict__ slots, JobCtl *__restrict__ ctl,
                                  const int32_t *__restrict__ slot_of, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int slot = slot_of[k];
    ctl[slot].phase = kJobIdle;
    ctl[slot].job = 0;
    slots[slot].active = 0;
}

}  // namespace

// ------------------------------------------------------------------------------ launchers
cudaError_t launch_init(const TileDesc *d_tiles, int tile0, int n_tiles, int dim,
                        SlotState *d_slots, uint32_t *d_spins, uint32_t *d_bonds,
                        const int8_t *d_J, const int8_t *d_S, int in_row0, PhiloxKey key,
                        int *d_err, cudaStream_t st) {
    if (n_tiles <= 0) return cudaSuccess;
    if (dim == 3)
        init_kernel<3><<<n_tiles, 32, 0, st>>>(d_tiles, tile0, d_slots, d_spins, d_bonds, d_J,
                                               d_S, in_row0, key, d_err);
    else
        init_kernel<2><<<n_tiles, 32, 0, st>>>(d_tiles, tile0, d_slots, d_spins, d_bonds, d_J,
                                               d_S, in_row0, key, d_err);
    return cudaGetLastError();
}

cudaError_t launch_quantize(const TileDesc *d_tiles, int n_tiles, const SlotState *d_slots,
                            const double *d_lnW, uint32_t *d_thr, cudaStream_t st) {
    if (n_tiles <= 0) return cudaSuccess;
    quantize_kernel<<<n_tiles * kTile, 128, 0, st>>>(d_tiles, d_slots, d_lnW, d_thr);
    return cudaGetLastError();
}

cudaError_t launch_enforce_walls(const TileDesc *d_tiles, int n_tiles, const SlotState *d_slots,
                                 uint32_t *d_thr, cudaStream_t st) {
    if (n_tiles <= 0) return cudaSuccess;
    enforce_walls_kernel<<<n_tiles * kTile, 128, 0, st>>>(d_tiles, d_slots, d_thr);
    return cudaGetLastError();
}

cudaError_t launch_update_weights(const TileDesc *d_tiles, int n_tiles, SlotState *d_slots,
                                  double *d_lnW, uint32_t *d_hist, double2 *d_acc, cudaStream_t st) {
    if (n_tiles <= 0) return cudaSuccess;
    update_weights_kernel<<<n_tiles * kTile, 128, 0, st>>>(d_tiles, d_slots, d_lnW, d_hist, d_acc);
    return cudaGetLastError();
}

cudaError_t launch_build_ensemble(const TileDesc *d_tiles, int n_tiles, SlotState *d_slots,
                                  const uint8_t *d_sel, int kind, double alpha, double pole,
                                  double beta, double *d_lnW, cudaStream_t st) {
    if (n_tiles <= 0) return cudaSuccess;
    const int n_slots = n_tiles * kTile;
    build_ensemble_kernel<<<(n_slots + 127) / 128, 128, 0, st>>>(d_tiles, n_slots, d_slots, d_sel,
                                                                 kind, alpha, pole, beta, d_lnW);
    return cudaGetLastError();
}

cudaError_t launch_reset_lanes(const TileDesc *d_tiles, int dim, SlotState *d_slots, uint32_t *d_spins,
                               uint32_t *d_bonds, double *d_lnW, uint32_t *d_hist, const int32_t *d_slot_of,
                               const uint32_t *d_rids, const uint32_t *d_streams, int n, PhiloxKey key,
                               int *d_err, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (dim == 3)
        reset_lane_kernel<3><<<n, 32, 0, st>>>(d_tiles, d_slots, d_spins, d_bonds, d_lnW, d_hist, d_slot_of, d_rids,
                                               d_streams, key, d_err);
    else
        reset_lane_kernel<2><<<n, 32, 0, st>>>(d_tiles, d_slots, d_spins, d_bonds, d_lnW, d_hist, d_slot_of, d_rids,
                                               d_streams, key, d_err);
    return cudaGetLastError();
}

cudaError_t launch_update_weights_sel(const TileDesc *d_tiles, SlotState *d_slots, double *d_lnW,
                                      uint32_t *d_hist, double2 *d_acc, const int32_t *d_slot_of, int n,
                                      cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    update_weights_sel_kernel<<<n, 128, 0, st>>>(d_tiles, d_slots, d_lnW, d_hist, d_acc, d_slot_of);
    return cudaGetLastError();
}

cudaError_t launch_reset_rt(const TileDesc *d_tiles, int n_tiles, SlotState *d_slots,
                            const uint8_t *d_sel, cudaStream_t st) {
    if (n_tiles <= 0) return cudaSuccess;
    const int n_slots = n_tiles * kTile;
    reset_rt_kernel<<<(n_slots + 127) / 128, 128, 0, st>>>(d_tiles, n_slots, d_slots, d_sel);
    return cudaGetLastError();
}

}  // namespace eamc

namespace eamc {

cudaError_t launch_srv_control(const TileDesc *d_tiles, int n_slots, SlotState *d_slots, JobCtl *d_ctl,
                               int32_t *d_flag, SrvRecord *d_ring, uint32_t *d_head, uint32_t ring_cap,
                               unsigned long long *d_attempts, uint64_t tick, cudaStream_t st) {
    if (n_slots <= 0) return cudaSuccess;
    srv_control_kernel<<<(n_slots + 127) / 128, 128, 0, st>>>(d_tiles, n_slots, d_slots, d_ctl, d_flag, d_ring,
                                                              d_head, ring_cap, d_attempts, tick);
    return cudaGetLastError();
}

cudaError_t launch_srv_update(const TileDesc *d_tiles, int n_slots, SlotState *d_slots, double *d_lnW,
                              uint32_t *d_hist, double2 *d_acc, const int32_t *d_flag, cudaStream_t st) {
    if (n_slots <= 0) return cudaSuccess;
    srv_update_kernel<<<n_slots, 128, 0, st>>>(d_tiles, d_slots, d_lnW, d_hist, d_acc, d_flag);
    return cudaGetLastError();
}

cudaError_t launch_quantize_flagged(const TileDesc *d_tiles, int n_slots, const SlotState *d_slots,
                                    const double *d_lnW, uint32_t *d_thr, const int32_t *d_flag, cudaStream_t st) {
    if (n_slots <= 0) return cudaSuccess;
    quantize_flagged_kernel<<<n_slots, 128, 0, st>>>(d_tiles, d_slots, d_lnW, d_thr, d_flag);
    return cudaGetLastError();
}

cudaError_t launch_srv_start(const TileDesc *d_tiles, SlotState *d_slots, JobCtl *d_ctl, int32_t *d_flag,
                             double2 *d_acc, const SrvStart *d_start, int n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    srv_start_kernel<<<n, 128, 0, st>>>(d_tiles, d_slots, d_ctl, d_flag, d_acc, d_start);
    return cudaGetLastError();
}

cudaError_t launch_srv_cancel(SlotState *d_slots, JobCtl *d_ctl, const int32_t *d_slot_of, int n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    srv_cancel_kernel<<<(n + 127) / 128, 128, 0, st>>>(d_slots, d_ctl, d_slot_of, n);
    return cudaGetLastError();
}

}  // namespace eamc
