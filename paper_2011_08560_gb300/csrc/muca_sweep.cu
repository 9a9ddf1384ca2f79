// muca_sweep.cu -- a2 + a3: the multicanonical sweep kernel (the hot loop).
//
// Sequential single-spin-flip generalized Metropolis (Sec. II, Eq. "muca":
// P_acc = min(1, W(E_new)/W(E_old))), sites in lexicographic order, for 32 independent
// chains per warp.  After every attempt the lowest energy and (optionally) the round-trip
// state machine of Sec. III are updated; after every sweep H(E) += 1.
//
// Layout inside the kernel.  Each lane owns one chain and keeps that chain's lattice in
// shared memory as row words: the L sites of a row along x are packed 4 bits apart (a
// "nibble" per site, only its low bit used), lane-interleaved (word k of lane l at
// [k*32 + l]) so every access is bank-conflict free.  For a whole row at once,
//   unsatisfied(bond) = S_i ^ S_j ^ J_ij   is one XOR of row words, and
//   n_unsat(site)     = sum over bonds     is an integer add of row words
// (nibbles never carry: at most 6 bonds).  Only two terms change while a row is swept: the
// bond to the -x neighbour (that site was just updated) and the wrap bond of the last site.
// Both are carried as the two candidate counts nA / nB, so each attempt's critical path is
// select -> compare: the threshold for "previous attempt rejected" and "previous attempt
// accepted" are both loaded before that outcome is known.
//
// Acceptance thresholds thr[b][n] live in shared memory (lane-interleaved, conflict free)
// when the table fits, otherwise they are read through L1 from global memory.
//
// Tile width.  A tile holds W = 32 or 16 chains.  With W < 32 the warp's lanes l, l + W, ...
// all run chain l (same inputs, same arithmetic, same values written to the same shared-memory
// words) and only lanes below W write to global memory.  A narrow tile needs W/32 of the shared
// memory of a full one, which brings the threshold tables of L = 7, 8 into shared memory: fewer
// chains per SM, but each attempt of a chain is faster -- the better choice when the batch has
// fewer chains than the GPU can hold.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "eamc_internal.cuh"

namespace eamc {

namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;
// warps: 0 consumer, 1 bond sums, 2-3 random numbers, kMeasureWarp measurement.  Warp w issues
// on scheduler w % 4: with six warps the measurement (warp 5) shares the bond-sum warp's
// scheduler and warp 4 only takes part in the barriers, so nothing competes with the consumer
// for its scheduler (five warps, measurement on warp 4 beside the consumer, and four, the
// bond-sum warp measuring as well, were both measured slower on the L = 6 batch).
#ifndef EAMC_SWEEP_WARPS
#define EAMC_SWEEP_WARPS 6
#endif
constexpr int kWarps = EAMC_SWEEP_WARPS;
#ifndef EAMC_MEASURE_WARP
#define EAMC_MEASURE_WARP (EAMC_SWEEP_WARPS >= 5 ? EAMC_SWEEP_WARPS - 1 : 1)
#endif
constexpr int kMeasureWarp = EAMC_MEASURE_WARP;
constexpr int kThreads = 32 * kWarps;

template <int L>
using RowT = typename std::conditional<(L <= 8), uint32_t, uint64_t>::type;

template <class T, int L>
__host__ __device__ constexpr T nib_mask() {
    T m = 0;
    for (int x = 0; x < L; ++x) m |= T(1) << (4 * x);
    return m;
}

template <class T, int L>
__host__ __device__ constexpr T width_mask() {
    return (4 * L == 8 * (int)sizeof(T)) ? ~T(0) : ((T(1) << (4 * L)) - 1);
}

// nibble x <- nibble x+1 (mod L)
template <class T, int L>
__device__ __forceinline__ T rot_next(T r) {
    return ((r >> 4) | (r << (4 * L - 4))) & width_mask<T, L>();
}

// nibble x <- nibble x-1 (mod L)
template <class T, int L>
__device__ __forceinline__ T rot_prev(T r) {
    return ((r << 4) | (r >> (4 * L - 4))) & width_mask<T, L>();
}

template <int DIM, int L, int W>
struct Geo {
    static_assert(W == 32 || W == 16 || W == 8, "tile width");
    using T = RowT<L>;
    static constexpr int NR = DIM == 3 ? L * L : L;          // rows along x
    static constexpr int V = NR * L;
    static constexpr int B = ((DIM * V) / 2 >> 1) + 1;       // table rows per chain
    static constexpr int NG = (L + 3) / 4;                   // Philox calls per row
    static constexpr int FIELDS = DIM + 1;                   // S, Jx, Jy, (Jz)
    static constexpr int SUMQ = sizeof(T) == 4 ? 1 : 2;      // uint4 slots for sA,sB,R,JYm
    static constexpr int HQ = SUMQ + NG;                     // uint4 slots per lane per row
    static constexpr int LAG = (L >= 4 && L <= 8) ? 2 : 1;  // rows the producers run ahead
    static constexpr int NBUF = LAG + 1;                      // records in the ring
    static constexpr size_t LATTICE_BYTES = (size_t)FIELDS * NR * W * sizeof(T);
    static constexpr size_t HAND_BYTES = (size_t)NBUF * HQ * W * 16;
    static constexpr size_t RES_BYTES = (size_t)2 * L * W * sizeof(int);  // row offsets, measurement
    static constexpr size_t THR_BYTES = (size_t)(B + 2 * DIM) * 8 * W * sizeof(uint32_t);
    static constexpr size_t BASE_BYTES = LATTICE_BYTES + HAND_BYTES + RES_BYTES;
    // up to 225 KB of the 227 KB a block may use (the rest: static shared memory)
    static constexpr bool SMEM_THR = BASE_BYTES + THR_BYTES <= 225 * 1024;
    static constexpr size_t SMEM = BASE_BYTES + (SMEM_THR ? THR_BYTES : 0);
};

template <bool SMEM>
__device__ __forceinline__ uint32_t load_thr(const uint32_t *p) {
    if constexpr (SMEM) return *p;
    else return __ldg(p);
}

// record slot q of chain ln in a ring buffer of W-chain-wide uint4 slots
template <int W, class T>
__device__ __forceinline__ void put4(uint4 *slots, int q, int ln, T a, T b, T c, T d) {
    if constexpr (sizeof(T) == 4) {
        slots[q * W + ln] = make_uint4(a, b, c, d);
    } else {
        slots[q * W + ln] = make_uint4((uint32_t)a, (uint32_t)(a >> 32), (uint32_t)b, (uint32_t)(b >> 32));
        slots[(q + 1) * W + ln] = make_uint4((uint32_t)c, (uint32_t)(c >> 32), (uint32_t)d, (uint32_t)(d >> 32));
    }
}

template <int W, class T>
__device__ __forceinline__ void get4(const uint4 *slots, int q, int ln, T &a, T &b, T &c, T &d) {
    if constexpr (sizeof(T) == 4) {
        const uint4 v = slots[q * W + ln];
        a = v.x; b = v.y; c = v.z; d = v.w;
    } else {
        const uint4 v = slots[q * W + ln], w = slots[(q + 1) * W + ln];
        a = ((T)v.y << 32) | v.x; b = ((T)v.w << 32) | v.z;
        c = ((T)w.y << 32) | w.x; d = ((T)w.w << 32) | w.z;
    }
}

// kWarps warps per tile.  Warp 0 (consumer) runs the sequential accept / reject chain of the 32
// chains.  Warps 1..3 (producers) work LAG rows ahead of it: warp 1 sums, per site, the
// unsatisfied-bond indicators of the bonds that cannot change while the consumer sweeps that
// row; warps 2 and 3 draw the row's random words (Philox call g of the row from warp 2 + g % 2).
// Warp kMeasureWarp measures, one row behind the consumer: from the row offsets the consumer
// leaves after each attempt it keeps the lowest energy, the round-trip state and the histogram.
// One block barrier per row; records live in a ring of LAG + 1 buffers, results in two.  At the
// end of a row the consumer already loads the candidate thresholds of the next row's first
// attempt (the next record is in its registers), so a row starts with a decision.
//
// Running LAG rows ahead is exact as long as every row a record reads as final has been swept:
// besides the -y row (which the consumer adds itself), the last row of a plane (y = L-1) reads
// the plane's first row, L-1 rows back, so LAG <= L-2; the -z row is L rows back.
template <int DIM, int L, int W>
__device__ __forceinline__ void sweep_tile(const TileDesc &td, int tile, SlotState *__restrict__ slots,
                                           uint32_t *__restrict__ spins,
                                           const uint32_t *__restrict__ bonds,
                                           const uint32_t *__restrict__ thr,
                                           uint32_t *__restrict__ hist, uint64_t n_sweeps,
                                           PhiloxKey key, int count_rt, unsigned *__restrict__ diag,
                                           unsigned char *smem_raw) {
    using G = Geo<DIM, L, W>;
    using T = typename G::T;
    constexpr int NR = G::NR, LAG = G::LAG, NBUF = G::NBUF;
    constexpr T NIB = nib_mask<T, L>();
    constexpr T LASTNIB = T(1) << (4 * (L - 1));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // ln: this lane's chain in the tile; lanes ln, ln + W, ... run the same chain and only the
    // first (lane < W, `owner`) writes to global memory
    const int ln = lane & (W - 1);
    const bool owner = lane < W;

    // ---- stage the lattice as nibble-packed row words, chain-interleaved: word k of chain ln
    //      at [k*W + ln].  Nibble x of a row word is site x of that row.
    T *sm = reinterpret_cast<T *>(smem_raw);
    T *Rs = sm;                  // spins, nibble = 1 if S = -1
    T *JXs = sm + NR * W;        // bond (x, x+1) has J = -1
    T *JYs = sm + 2 * NR * W;    // bond (x,y)-(x,y+1)
    T *JZs = sm + 3 * NR * W;    // bond (x,y,z)-(x,y,z+1)   (DIM == 3)
    uint4 *hand = reinterpret_cast<uint4 *>(smem_raw + G::LATTICE_BYTES);
    int *res = reinterpret_cast<int *>(smem_raw + G::LATTICE_BYTES + G::HAND_BYTES);  // [2][L][W]
    const uint32_t *gsp = spins + td.spin_off;
    const uint32_t *gbd = bonds + td.bond_off;
    for (int row = warp; row < NR; row += kWarps) {
        T r = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
        for (int x = 0; x < L; ++x) {
            const int i = row * L + x;
            r |= T((gsp[i] >> ln) & 1u) << (4 * x);
            jx |= T((gbd[i * DIM + 0] >> ln) & 1u) << (4 * x);
            jy |= T((gbd[i * DIM + 1] >> ln) & 1u) << (4 * x);
            if constexpr (DIM == 3) jz |= T((gbd[i * DIM + 2] >> ln) & 1u) << (4 * x);
        }
        Rs[row * W + ln] = r;
        JXs[row * W + ln] = jx;
        JYs[row * W + ln] = jy;
        if constexpr (DIM == 3) JZs[row * W + ln] = jz;
    }

    const int slot = tile * kTile + ln;
    SlotState ss = slots[slot];
    const bool active = ss.active != 0;
    const uint64_t lrow = td.w_base + (uint64_t)ln * G::B;
    // element (b, n) of this chain's table at byte offset b * RSB + n * NSB from `tab`; rows
    // -DIM .. B-1+DIM are addressable (padding), so a speculative row one move away from a
    // valid row never needs a clamp
    constexpr int NSB = G::SMEM_THR ? 4 * W : 4;
    constexpr int RSB = 8 * NSB;
    const char *tab;
    if constexpr (G::SMEM_THR) {
        uint32_t *TH = reinterpret_cast<uint32_t *>(smem_raw + G::LATTICE_BYTES + G::HAND_BYTES + G::RES_BYTES);
        if (warp == 1) {
            // the 32 / W lanes of a chain stage every (32 / W)-th bin each
            constexpr int NM = 32 / W;
            const int mi = lane / W;
            const uint4 *src = reinterpret_cast<const uint4 *>(thr + lrow * 8);
            for (int b = mi; b < G::B; b += NM) {
                const uint4 a = src[2 * b], c = src[2 * b + 1];
                uint32_t *d = TH + (b + DIM) * 8 * W + ln;
                d[0] = a.x; d[W] = a.y; d[2 * W] = a.z; d[3 * W] = a.w;
                d[4 * W] = c.x; d[5 * W] = c.y; d[6 * W] = c.z; d[7 * W] = c.w;
            }
            for (int k = mi; k < DIM * 8; k += NM) {
                TH[k * W + ln] = 0u;
                TH[((G::B + DIM) * 8 + k) * W + ln] = 0u;
            }
        }
        tab = reinterpret_cast<const char *>(TH + DIM * 8 * W + ln);
    } else {
        tab = reinterpret_cast<const char *>(thr + lrow * 8);
    }
    const uint64_t t0 = ss.t;
    const uint64_t total = n_sweeps * (uint64_t)NR;  // rows to sweep

    __syncthreads();
    // every warp passes exactly 1 + total + 1 block barriers
    if (warp >= 1) {
        // ---- producers: record of row `row` (sweep index tt) into ring buffer `k`
        auto produce = [&](int row, int y, int z, uint32_t tt, int k) {
            uint4 *buf = hand + k * G::HQ * W;
            if (warp >= 2) {  // random words: Philox call g covers sites x = 4g .. 4g+3
                // stored as min(r, 2^32 - 2) (an inactive chain: 2^32 - 1), so that the
                // consumer's single test r < th is the rule "r < th or th = always" of an
                // active chain and never accepts for an inactive one; thresholds below
                // "always" are at most 2^32 - 2, which the clamp does not reach
                const uint32_t c3 = ss.stream << 8;
#pragma unroll
                for (int g = warp - 2; g < G::NG; g += 2) {
                    uint4 w = philox4x32_10(make_uint4((uint32_t)(4 * row + g), tt, ss.rid, c3), key);
                    w.x = active ? min(w.x, kAlways - 1u) : kAlways;
                    w.y = active ? min(w.y, kAlways - 1u) : kAlways;
                    w.z = active ? min(w.z, kAlways - 1u) : kAlways;
                    w.w = active ? min(w.w, kAlways - 1u) : kAlways;
                    buf[(G::SUMQ + g) * W + ln] = w;
                }
                return;
            }
            const int ryp = (y == L - 1) ? row - (L - 1) : row + 1;
            const T R = Rs[row * W + ln];
            const T u_xp = R ^ rot_next<T, L>(R) ^ JXs[row * W + ln];  // bond (x, x+1) at nibble x
            const T u_xm = rot_prev<T, L>(u_xp);                        // bond (x-1, x) at nibble x
            T stable = (R ^ Rs[ryp * W + ln] ^ JYs[row * W + ln]) + (u_xp & ~LASTNIB);
            if constexpr (DIM == 3) {
                const int rzm = (z == 0) ? row + (L - 1) * L : row - L;
                const int rzp = (z == L - 1) ? row - (L - 1) * L : row + L;
                stable += (R ^ Rs[rzp * W + ln] ^ JZs[row * W + ln]) +
                          (R ^ Rs[rzm * W + ln] ^ JZs[rzm * W + ln]);
            }
            // the -y row: the consumer's previous row (added there) unless (3D, y = 0), where
            // it is the plane's last row, not yet swept
            T jym = 0;
            const int rym = (y == 0) ? row + (L - 1) : row - 1;
            if (DIM == 3 && y == 0) stable += R ^ Rs[rym * W + ln] ^ JYs[rym * W + ln];
            else jym = JYs[rym * W + ln];
            const T sA = stable + u_xm;
            // nibble 0 of sB is never used (site 0 has no dynamic -x bond): its bit 3 carries
            // the stale wrap bond of site L-1
            const T wbit = (u_xp >> (4 * (L - 1))) & T(1);
            const T sB = ((stable + (u_xm ^ NIB)) & ~T(0xF)) | (wbit << 3);
            put4<W, T>(buf, 0, ln, sA, sB, R, jym);
        };
        int row = 0, y = 0, z = 0, kb = 0;
        uint64_t s = 0;
        auto advance = [&]() {
            if (++y == L) { y = 0; ++z; }
            if (++row == NR) { row = 0; y = 0; z = 0; ++s; }
            if (++kb == NBUF) kb = 0;
        };
        const bool producer = warp <= 3;
        for (int j = 0; producer && j < LAG && (uint64_t)j < total; ++j) {  // the first LAG records
            produce(row, y, z, (uint32_t)(t0 + s), kb);
            advance();
        }
        // ---- measurement (warp kMeasureWarp), one row behind the consumer: lowest energy, round trips
        //      (Sec. III) and, after every sweep, H(E) += 1
        int phase = ss.phase, nrt = ss.n_rt;
        int64_t tf = ss.t_first, tl = ss.t_last;
        const int topB = ss.b_top * RSB, botB = ss.b_g * RSB;
        int pmin = ss.b_min * RSB, pnow = ss.b * RSB;
        uint32_t *hist_l = hist + lrow;
        int mrow = 0;
        uint64_t ms = 0;
        bool out_of_range = false;  // a bin outside [0, b_top]: a broken invariant, reported via diag
        auto measure = [&](int buf) {
            const int *r = res + buf * L * W + ln;
            int lo = 0x7FFFFFFF, hi = -0x7FFFFFFF;
            uint32_t mtop = 0u, mbot = 0u;
#pragma unroll
            for (int x = 0; x < L; ++x) {
                const int pr = r[x * W];
                lo = min(lo, pr);
                hi = max(hi, pr);
                mtop |= (uint32_t)(pr >= topB) << x;
                mbot |= (uint32_t)(pr <= botB) << x;
                if (x == L - 1) pnow = pr;
            }
            pmin = min(pmin, lo);
            out_of_range |= (lo < 0) | (hi > topB);
            // the attempts of the row in order: a transition at the first attempt that meets
            // the current phase's condition (E <= E_g heading down, E >= E_top otherwise), the
            // next one looked for after it
            if (count_rt && active && ((phase == 1) ? mbot : mtop) != 0u) {
                const int64_t t = (int64_t)(t0 + ms);
                int x0 = 0;
                while (x0 < L) {
                    const uint32_t m = ((phase == 1) ? mbot : mtop) >> x0;
                    if (m == 0u) break;
                    x0 += __ffs(m);  // one past the attempt that meets the condition
                    if (phase == 0) { tf = t; phase = 1; }
                    else if (phase == 1) { phase = 2; }
                    else { nrt += 1; tl = t; phase = 1; }
                }
            }
            if (++mrow == NR) {
                mrow = 0;
                ++ms;
                if (active && owner) atomicAdd(&hist_l[pnow / RSB], 1u);  // no return value: no wait
            }
        };
        for (uint64_t k = 0; k < total; ++k) {
            // barrier k: records up to k+LAG-1 are complete, the consumer is done with record
            // k-1 (whose buffer takes record k+LAG) and has left the result of row k-1
            __syncthreads();
            if (producer && k + LAG < total) {
                produce(row, y, z, (uint32_t)(t0 + s), kb);
                advance();
            }
            if (warp == kMeasureWarp && k > 0) measure((int)((k - 1) & 1));
        }
        __syncthreads();
        if (warp == kMeasureWarp) {
            if (total > 0) measure((int)((total - 1) & 1));
            ss.b = pnow / RSB;
            ss.b_min = pmin / RSB;
            ss.phase = phase;
            ss.n_rt = nrt;
            ss.t_first = tf;
            ss.t_last = tl;
            ss.t = t0 + n_sweeps;
            if (count_rt && active && energy_of_bin(DIM * G::V, ss.parity, ss.b_min) < ss.e_g) ss.requeue = 1;
            if (owner) slots[slot] = ss;
            if (diag && __any_sync(kFull, active && out_of_range) && lane == 0) atomicOr(diag, 1u);
        }
        return;
    }

    // ---- consumer
    // the previous attempt, applied lazily: row it was evaluated at (rq), row delta if it was
    // accepted (dq) and whether it was (pa)
    int rq = ss.b * RSB, dq = 0, pa = 0;
    T Rprev = Rs[(NR - 1) * W + ln];
    int row = 0, y = 0, kb = 0;
    // the record of the row to sweep; with LAG >= 2 the next one is complete one barrier early
    // and is read while the current row runs
    T nsA, nsB, nR, njym;
    uint4 nrr[G::NG];
    auto load_rec = [&](int b) {
        const uint4 *buf = hand + b * G::HQ * W;
        get4<W, T>(buf, 0, ln, nsA, nsB, nR, njym);
#pragma unroll
        for (int g = 0; g < G::NG; ++g) nrr[g] = buf[(G::SUMQ + g) * W + ln];
    };
    // candidate thresholds of the next attempt; with LAG >= 2 the last attempt of a row already
    // loads those of the next row's first attempt (its record is in registers by then)
    uint32_t thA = 0u, thB = 0u;
    bool have_next = false;
    for (uint64_t k = 0; k < total; ++k) {
        __syncthreads();  // barrier k: record k is complete
        if (LAG == 1 || k == 0) load_rec(kb);
        T sA = nsA, sB = nsB;
        const T R = nR, jym = njym;
        uint4 rr[G::NG];
#pragma unroll
        for (int g = 0; g < G::NG; ++g) rr[g] = nrr[g];
        if (++kb == NBUF) kb = 0;
        if (LAG >= 2 && k + 1 < total) load_rec(kb);
        if (DIM == 2 || y > 0) {
            const T uym = R ^ Rprev ^ jym;
            sA += uym;
            sB += uym;
        }
        const int wbit = (int)((sB >> 3) & 1u);
        T accN = 0;  // nibble x = 1 if this chain flipped site x of the row
        int *resb = res + (int)(k & 1) * L * W + ln;
        // software pipeline: iteration x resolves attempt x from acc(x-1), issues both
        // candidate threshold loads of attempt x+1 (they need only acc(x-1)), then compares
        int nA = (int)(sA & 0xF), nB = nA;
        if (!have_next) {
            thA = load_thr<G::SMEM_THR>(reinterpret_cast<const uint32_t *>(tab + rq + nA * NSB));
            thB = load_thr<G::SMEM_THR>(reinterpret_cast<const uint32_t *>(tab + rq + dq + nB * NSB));
        }
        have_next = false;
        // does the next row add its -y bond (the row just finished) itself?
        const int y_next = (y + 1 == L || row + 1 == NR) ? 0 : y + 1;
        const bool next_uym = (DIM == 2 || y_next > 0);
#pragma unroll
        for (int x = 0; x < L; ++x) {
            // what does not depend on the previous decision comes first: both candidate deltas
            // of this attempt and all four candidate addresses of the next attempt's loads; the
            // previous decision then only selects
            const int rB = rq + dq;
            const int dxA = (DIM - nA) * RSB, dxB = (DIM - nB) * RSB;
            int nA1 = 0, nB1 = 0;
            bool next = false;
            if (x + 1 < L) {
                nA1 = (int)((sA >> (4 * (x + 1))) & 0xF);
                nB1 = (int)((sB >> (4 * (x + 1))) & 0xF);
                if (x + 1 == L - 1) {  // bond to site 0 of the row, flipped at x = 0 or not
                    const int w = wbit ^ (int)(accN & 1u);
                    nA1 += w;
                    nB1 += w;
                }
                next = true;
            } else if (LAG >= 2 && k + 1 < total) {
                // first attempt of the next row: its class needs that row's record and, through
                // the -y bond, only site 0 of this row (final since attempt 0); both candidate
                // bins depend on this attempt
                const T rfin0 = (R ^ accN) & T(1);
                nA1 = nB1 = (int)(nsA & 0xF) + (next_uym ? (int)((nR ^ rfin0 ^ njym) & T(1)) : 0);
                next = true;
                have_next = true;
            }
            const int offA = nA1 * NSB, offB = nB1 * NSB;
            const int aA0 = rq + offA, aB0 = rq + dxA + offB, aA1 = rB + offA, aB1 = rB + dxB + offB;
            // the next attempt's loads go out before this attempt's threshold is used, so that
            // their latency overlaps this decision (a warp issues in order)
            uint32_t ldA = 0u, ldB = 0u;
            if (next) {
                ldA = load_thr<G::SMEM_THR>(reinterpret_cast<const uint32_t *>(tab + (pa ? aA1 : aA0)));
                ldB = load_thr<G::SMEM_THR>(reinterpret_cast<const uint32_t *>(tab + (pa ? aB1 : aB0)));
            }
            const uint32_t th = pa ? thB : thA;
            const int rx = pa ? rB : rq;
            const int dx = pa ? dxB : dxA;
            if (next) {
                thA = ldA;
                thB = ldB;
            }
            if (x + 1 < L) {
                nA = nA1;
                nB = nB1;
            }
            const uint32_t r = uint4_get(rr[x >> 2], x & 3);
            const bool acc = r < th;  // r clamped by the producer (see there)
            accN |= T(acc ? 1u : 0u) << (4 * x);
            resb[x * W] = acc ? rx + dx : rx;  // row offset after the attempt, for the measurement
            rq = rx;
            dq = dx;
            pa = acc ? 1 : 0;
        }
        const T Rfin = R ^ accN;
        Rs[row * W + ln] = Rfin;
        Rprev = Rfin;
        if (++y == L) y = 0;
        if (++row == NR) {
            row = 0;
            y = 0;
        }
    }
    __syncthreads();
    // spins back to the multi-spin-coded global layout
    constexpr uint32_t kOwned = W == 32 ? kFull : ((1u << W) - 1u);
    for (int r2 = 0; r2 < NR; ++r2) {
        const T Rw = Rs[r2 * W + ln];
#pragma unroll
        for (int x = 0; x < L; ++x) {
            const uint32_t m = __ballot_sync(kFull, ((Rw >> (4 * x)) & 1u) != 0) & kOwned;
            if (lane == 0) spins[td.spin_off + r2 * L + x] = m;
        }
    }
}

// Tile widths compiled per lattice size: 32 for every L; in 3D also 16 for L = 7, 8, whose
// threshold tables then fit in shared memory.  (Width 8 would do the same for L = 9, 10, but
// with both narrow families in this kernel it no longer fits in 255 registers without spills.)
__host__ __device__ constexpr bool width_compiled(int dim, int L, int W) {
    return W == 32 || (dim == 3 && W == 16 && (L == 7 || L == 8));
}

// kWarps warps per tile; the tile's (L, width) selects the body.
// Direct mode (queue == nullptr): block b sweeps tile tile_list[b] (or b).  Persistent mode:
// a grid sized to the resident capacity pulls positions of tile_list (longest tiles first)
// from the counter *queue until n_work positions are taken.
template <int DIM>
__device__ __forceinline__ void sweep_one(const TileDesc *__restrict__ tiles, int tile, SlotState *slots,
                                          uint32_t *spins, const uint32_t *bonds, const uint32_t *thr,
                                          uint32_t *hist, uint64_t n_sweeps, PhiloxKey key, int count_rt,
                                          unsigned *diag, unsigned char *smem_raw) {
    const TileDesc td = tiles[tile];
    const uint64_t n_tile = n_sweeps * (uint64_t)(td.sweep_mul > 0 ? td.sweep_mul : 1);
#define EAMC_BODY(LL, WW) \
    sweep_tile<DIM, LL, WW>(td, tile, slots, spins, bonds, thr, hist, n_tile, key, count_rt, diag, smem_raw)
#define EAMC_CASE(LL)                                                              \
    case LL:                                                                       \
        if constexpr (width_compiled(DIM, LL, 16)) {                               \
            if (td.width == 16) { EAMC_BODY(LL, 16); break; }                      \
        }                                                                          \
        if constexpr (width_compiled(DIM, LL, 8)) {                                \
            if (td.width == 8) { EAMC_BODY(LL, 8); break; }                       \
        }                                                                          \
        EAMC_BODY(LL, 32);                                                         \
        break;
    switch (td.L) {
        EAMC_CASE(3) EAMC_CASE(4) EAMC_CASE(5) EAMC_CASE(6) EAMC_CASE(7)
        EAMC_CASE(8) EAMC_CASE(9) EAMC_CASE(10) EAMC_CASE(11) EAMC_CASE(12)
        default: break;
    }
#undef EAMC_CASE
#undef EAMC_BODY
}

template <int DIM>
__global__ void __launch_bounds__(kThreads, 1)
muca_sweep_kernel(const TileDesc *__restrict__ tiles, const int32_t *__restrict__ tile_list, int n_work,
                  int *__restrict__ queue, SlotState *__restrict__ slots, uint32_t *__restrict__ spins,
                  const uint32_t *__restrict__ bonds, const uint32_t *__restrict__ thr,
                  uint32_t *__restrict__ hist, uint64_t n_sweeps, PhiloxKey key, int count_rt,
                  unsigned *__restrict__ diag) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (!queue) {
        const int tile = tile_list ? tile_list[blockIdx.x] : (int)blockIdx.x;
        sweep_one<DIM>(tiles, tile, slots, spins, bonds, thr, hist, n_sweeps, key, count_rt, diag, smem_raw);
        return;
    }
    __shared__ int s_pos;
    for (;;) {
        if (threadIdx.x == 0) s_pos = atomicAdd(queue, 1);
        __syncthreads();
        const int pos = s_pos;
        __syncthreads();  // every thread has read s_pos before it is overwritten
        if (pos >= n_work) break;
        sweep_one<DIM>(tiles, tile_list[pos], slots, spins, bonds, thr, hist, n_sweeps, key, count_rt, diag,
                       smem_raw);
        __syncthreads();  // every warp is done with this tile's shared memory
    }
}

template <int DIM, int W>
size_t smem_for_w(int L) {
    switch (L) {
        case 3: return Geo<DIM, 3, W>::SMEM;
        case 4: return Geo<DIM, 4, W>::SMEM;
        case 5: return Geo<DIM, 5, W>::SMEM;
        case 6: return Geo<DIM, 6, W>::SMEM;
        case 7: return Geo<DIM, 7, W>::SMEM;
        case 8: return Geo<DIM, 8, W>::SMEM;
        case 9: return Geo<DIM, 9, W>::SMEM;
        case 10: return Geo<DIM, 10, W>::SMEM;
        case 11: return Geo<DIM, 11, W>::SMEM;
        case 12: return Geo<DIM, 12, W>::SMEM;
        default: return 0;
    }
}

template <int DIM, int W>
bool thr_smem_w(int L) {
    switch (L) {
        case 3: return Geo<DIM, 3, W>::SMEM_THR;
        case 4: return Geo<DIM, 4, W>::SMEM_THR;
        case 5: return Geo<DIM, 5, W>::SMEM_THR;
        case 6: return Geo<DIM, 6, W>::SMEM_THR;
        case 7: return Geo<DIM, 7, W>::SMEM_THR;
        case 8: return Geo<DIM, 8, W>::SMEM_THR;
        case 9: return Geo<DIM, 9, W>::SMEM_THR;
        case 10: return Geo<DIM, 10, W>::SMEM_THR;
        case 11: return Geo<DIM, 11, W>::SMEM_THR;
        case 12: return Geo<DIM, 12, W>::SMEM_THR;
        default: return false;
    }
}

}  // namespace

size_t sweep_smem_bytes(int dim, int L, int width) {
    if (!sweep_width_supported(dim, L, width)) return 0;
    if (dim == 3) return width == 32 ? smem_for_w<3, 32>(L) : width == 16 ? smem_for_w<3, 16>(L) : smem_for_w<3, 8>(L);
    return smem_for_w<2, 32>(L);
}

bool sweep_width_supported(int dim, int L, int width) {
    return L >= 3 && L <= 12 && (dim == 2 || dim == 3) && width_compiled(dim, L, width);
}

bool sweep_thresholds_in_smem(int dim, int L, int width) {
    if (!sweep_width_supported(dim, L, width)) return false;
    if (dim == 3) return width == 32 ? thr_smem_w<3, 32>(L) : width == 16 ? thr_smem_w<3, 16>(L) : thr_smem_w<3, 8>(L);
    return thr_smem_w<2, 32>(L);
}

// Raises the kernel's dynamic shared-memory limit when needed (a host call that is not stream
// work, so it happens before any graph capture that launches the kernel).
cudaError_t prepare_sweeps(int dim, size_t smem) {
    static int set_limit[4] = {0, 0, 0, 0};
    if ((int)smem <= set_limit[dim]) return cudaSuccess;
    const cudaError_t e = dim == 3
        ? cudaFuncSetAttribute(muca_sweep_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
        : cudaFuncSetAttribute(muca_sweep_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) set_limit[dim] = (int)smem;
    return e;
}

cudaError_t launch_sweeps(const TileDesc *d_tiles, const int32_t *d_tile_list, int n_blocks, int n_work,
                          int *d_queue, int dim, size_t smem, SlotState *d_slots, uint32_t *d_spins,
                          const uint32_t *d_bonds, const uint32_t *d_thr, uint32_t *d_hist, uint64_t n_sweeps,
                          PhiloxKey key, int count_rt, unsigned *d_diag, cudaStream_t st) {
    if (n_blocks <= 0 || n_sweeps == 0) return cudaSuccess;
    cudaError_t e;
    if (d_queue) {
        e = cudaMemsetAsync(d_queue, 0, sizeof(int), st);
        if (e != cudaSuccess) return e;
    }
    if ((e = prepare_sweeps(dim, smem)) != cudaSuccess) return e;
    if (dim == 3) {
        muca_sweep_kernel<3><<<n_blocks, kThreads, smem, st>>>(d_tiles, d_tile_list, n_work, d_queue, d_slots, d_spins,
                                                         d_bonds, d_thr, d_hist, n_sweeps, key, count_rt, d_diag);
    } else {
        muca_sweep_kernel<2><<<n_blocks, kThreads, smem, st>>>(d_tiles, d_tile_list, n_work, d_queue, d_slots, d_spins,
                                                         d_bonds, d_thr, d_hist, n_sweeps, key, count_rt, d_diag);
    }
    return cudaGetLastError();
}

int sweep_blocks_per_sm(int dim, size_t smem) {
    int nb = 0;
    if (dim == 3)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, muca_sweep_kernel<3>, kThreads, smem);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, muca_sweep_kernel<2>, kThreads, smem);
    return nb > 0 ? nb : 1;
}

}  // namespace eamc
