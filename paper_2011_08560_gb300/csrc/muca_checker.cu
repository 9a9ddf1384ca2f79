// muca_checker.cu -- a2 + a3 in the colour order (the checkerboard for even L): the
// multicanonical sweep (Sec. II, Eq. "muca") with the sites of a sweep taken colour by colour,
// each colour in lexicographic order, for 32, 16, 8 or 4 independent chains per tile, one lane
// per chain (a narrow tile's chains on 32 / width lanes each).  Odd L (three colours, the PT
// colouring) runs in the same kernel: a row has a varying number of sites of a colour, so each
// row gets the largest number of attempt slots and the unused ones are padding that moves
// nothing and never accepts; each (pass, row)'s sites come from tables made once per launch.
//
// In a colour pass no two attempted sites are neighbours, so the class n of every attempt
// (unsatisfied bonds, the move changes the bin by dim - n) is fixed when the pass begins.  The
// only sequential coupling of a chain's attempts is its energy bin: attempt i+1's threshold is
// thr[b][n_{i+1}] with b = b_i or b_i + dim - n_i, so both candidates are loaded before
// attempt i is decided and the decision only selects.  That leaves one class extraction, two
// loads, two selects and a compare per attempt on the consumer warp (the lexicographic order
// has to carry two candidate classes as well, because consecutive sites are neighbours).
//
// Eight warps; warp w issues on scheduler w % 4: 0 the consumer, alone on its scheduler; 1 and 5
// the classes of a record's rows; 3 and 6 their random words (the Philox calls are the heaviest
// producer work, so they sit on two schedulers; a narrow tile deals the rows to the lane groups
// of these warps as well); 2 the measurement (lowest energy, round trips, histogram), one record
// behind the consumer; 4 and 7 only take part in the barriers.  A record is RPR consecutive rows
// of one pass (two to eight, by size): the colour-c sites of those rows, RPR L / 2 attempts for
// even L, with each attempt's class as its table offset n * NSB (16 bits) and its random word.
// The consumer leaves the bin after every attempt for the measurement.  Within a pass the producers may run any number of records ahead (the classes
// read only the other colour's spins and each site's own spin, which its own record changes), so
// they run LAG records ahead; at the start of a pass one extra barrier lets them refill, because
// the first plane's classes read the last plane of the previous pass.
//
// Random words (the colour-order streams): the j-th colour-c site of row r takes word j&3 of
// Philox call (4 r + j/4, t, rid, (5 + c) | stream << 8).
//
// Lattice layout: row words with one nibble per site, chain-interleaved: the spins (bit 0) and
// the bonds (Jx, Jy, Jz at bits 0, 1, 2); thresholds lane-interleaved in shared memory when they
// fit, else read through L1.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "eamc_internal.cuh"

namespace eamc {

namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr int kCkWarps = 8;
constexpr int kCkMeasure = 2;
constexpr int kCkThreads = 32 * kCkWarps;
// warp roles: classes of a record's rows (warps 1, 5), their random words (warps 3, 6)
__device__ __forceinline__ bool ck_classes(int warp) { return warp == 1 || warp == 5; }
__device__ __forceinline__ bool ck_random(int warp) { return warp == 3 || warp == 6; }

template <int L>
using CkRow = typename std::conditional<(L <= 8), uint32_t, uint64_t>::type;

template <class T, int L>
__device__ __forceinline__ constexpr T ck_mask() {
    return (4 * L == 8 * (int)sizeof(T)) ? ~T(0) : ((T(1) << (4 * L)) - 1);
}

// nibble x <- nibble x+1 (mod L), and nibble x <- nibble x-1
template <class T, int L>
__device__ __forceinline__ T ck_next(T r) {
    return ((r >> 4) | (r << (4 * L - 4))) & ck_mask<T, L>();
}
template <class T, int L>
__device__ __forceinline__ T ck_prev(T r) {
    return ((r << 4) | (r >> (4 * L - 4))) & ck_mask<T, L>();
}

// odd L: the colour of a site is (ax(x) + ax(y) + ax(z)) mod 3 with ax(c) = c mod 3, except
// ax(L-1) = 1 when L - 1 is a multiple of 3 (the PT colouring); the colour-c sites of a row with
// (c - ax(y) - ax(z)) mod 3 = s are the x with ax(x) = s
__host__ __device__ constexpr int ck_ax(int L, int c) { return (c == L - 1 && (L - 1) % 3 == 0) ? 1 : c % 3; }
__host__ __device__ constexpr int ck_sites_max(int L) {  // most colour-c sites in one row
    int m = 0;
    for (int s = 0; s < 3; ++s) {
        int n = 0;
        for (int x = 0; x < L; ++x) n += ck_ax(L, x) == s;
        m = n > m ? n : m;
    }
    return m;
}

template <int DIM, int L, int W>
struct CkGeo {
    static_assert(W == 32 || W == 16 || W == 8 || W == 4, "tile width");
    using T = CkRow<L>;
    static constexpr int NCOL = (L & 1) ? 3 : 2;    // colour passes per sweep
    static constexpr int NR = DIM == 3 ? L * L : L;  // rows along x
    static constexpr int V = NR * L;
    static constexpr int B = ((DIM * V) / 2 >> 1) + 1;
    // attempt slots per row: the colour-c sites of a row, the last ones padding where the row has
    // fewer (odd L: a padding slot moves nothing and never accepts)
    static constexpr int HALF = (L & 1) ? ck_sites_max(L) : L / 2;
    static_assert(HALF <= 4 || (L & 1) == 0, "one Philox call per row and pass for odd L");
    static constexpr int NGC = (HALF + 3) / 4;      // Philox calls per row and pass
    // rows per record (fewer, longer records spread the per-record cost of the barrier and the
    // hand-over over more attempts; measured per size, longer records where they cost the other
    // sizes of the same kernel nothing through its register allocation): 3D even L eight at
    // L = 8, six at L = 6, else four where the rows divide into fours, else two; odd L a plane's L
    // rows (the whole lattice for 2D and L = 3) up to L = 9, else two, the last record of a pass
    // padded with rows of padding slots
    static constexpr int RPR = (L & 1) ? (L <= 9 ? (NR <= 9 ? NR : L) : 2)
                                       : (DIM == 3 && L == 8) ? 8
                                       : (DIM == 3 && L == 6) ? 6
                                       : ((NR % 4 == 0 && (L <= 8 || DIM == 3)) ? 4 : 2);
    static constexpr int NA = RPR * HALF;           // attempts per record
    static_assert(NA <= 32, "the measurement keeps a record's attempts in 32-bit masks");
    static constexpr int NP = (NR + RPR - 1) / RPR;  // records per pass
    static constexpr int OW = (HALF + 1) / 2;       // 32-bit words of 16-bit class offsets per row
    static constexpr int OFFQ = (RPR * OW + 3) / 4; // uint4 slots of class offsets (row h at word h * OW)
    static constexpr int HQ = OFFQ + RPR * NGC;     // uint4 slots per lane per record
    static constexpr int LAG = NP >= 3 ? 2 : 1;     // records the producers run ahead
    // ring of records, indexed by the record count over the whole launch: record g is read by
    // the consumer after barrier g (and preloaded after g-1) while record g+LAG is written; one
    // buffer more than that needs (measured faster)
    static constexpr int NBUF = LAG + 2;
    static constexpr int FIELDS = 2;                // S, and the bonds (Jx, Jy, Jz at bits 0, 1, 2 of a site's nibble)
    static constexpr size_t LATTICE_BYTES = (size_t)FIELDS * NR * W * sizeof(T);
    static constexpr size_t HAND_BYTES = (size_t)NBUF * HQ * W * 16;
    static constexpr size_t RES_BYTES = (size_t)2 * NA * W * sizeof(int);  // bin row offset after each attempt, two records
    static constexpr size_t THR_BYTES = (size_t)(B + 2 * DIM) * 8 * W * sizeof(uint32_t);
    // odd L: each (pass, row)'s colour sites as nibble positions, padding slots at 0 for the
    // consumer and 0xFF for the producers (two tables; rows of a pass padded to whole records)
    static constexpr int NPR = NP * RPR;
    static constexpr size_t FSH_BYTES = (L & 1) ? ((size_t)2 * NCOL * NPR * 4 + 15) / 16 * 16 : 0;
    static constexpr size_t BASE_BYTES = LATTICE_BYTES + HAND_BYTES + RES_BYTES + FSH_BYTES;
    static constexpr bool SMEM_THR = BASE_BYTES + THR_BYTES <= 225 * 1024;
    static constexpr size_t SMEM = BASE_BYTES + (SMEM_THR ? THR_BYTES : 0);
    // thresholds addressed by 32-bit shared addresses; measured with the same launches: L = 6 in
    // tiles of 32 2.5 % faster, L = 10 in tiles of 8 1.5 % faster, L = 8 in tiles of 16 2.5 % slower
    static constexpr bool SADDR = SMEM_THR && !(L == 8 && W == 16);
};

// a threshold at byte offset a: in shared memory either at the 32-bit shared address a (SADDR: the
// table base is already in a, so the selected address is the load's operand) or at tab + a; in
// global memory at tab + a
template <bool SMEM, bool SADDR>
__device__ __forceinline__ uint32_t ck_thr(const char *tab, int a) {
    if constexpr (SMEM && SADDR) {
        uint32_t v;
        asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
        return v;
    } else if constexpr (SMEM) {
        return *reinterpret_cast<const uint32_t *>(tab + a);
    } else {
        return __ldg(reinterpret_cast<const uint32_t *>(tab + a));
    }
}

template <int DIM, int L, int W>
__device__ __forceinline__ void checker_tile(const TileDesc &td, int tile, SlotState *__restrict__ slots,
                                             uint32_t *__restrict__ spins, const uint32_t *__restrict__ bonds,
                                             const uint32_t *__restrict__ thr, uint32_t *__restrict__ hist,
                                             uint64_t n_sweeps, PhiloxKey key, int count_rt,
                                             unsigned *__restrict__ diag, unsigned char *smem_raw) {
    using G = CkGeo<DIM, L, W>;
    using T = typename G::T;
    constexpr int NR = G::NR, NP = G::NP, HALF = G::HALF, NGC = G::NGC, LAG = G::LAG, NBUF = G::NBUF;
    constexpr int RPR = G::RPR, NA = G::NA, NCOL = G::NCOL;
    constexpr bool ODD = (L & 1) != 0;
    constexpr bool PADROWS = (NR % RPR) != 0;  // the last record of a pass has rows of padding (odd L only)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ln = lane & (W - 1);  // chain of this lane; lanes ln + W, ... mirror it
    const bool owner = lane < W;

    T *Rs = reinterpret_cast<T *>(smem_raw);  // spins, nibble x = 1 if S = -1
    // bonds of a row, nibble x: bit 0 J(x, x+1) = -1, bit 1 J(y, y+1) = -1, bit 2 J(z, z+1) = -1
    T *JBs = Rs + NR * W;
    uint4 *hand = reinterpret_cast<uint4 *>(smem_raw + G::LATTICE_BYTES);
    int *res = reinterpret_cast<int *>(smem_raw + G::LATTICE_BYTES + G::HAND_BYTES);  // [2 records][NA][W]
    uint32_t *ftab = reinterpret_cast<uint32_t *>(smem_raw + G::LATTICE_BYTES + G::HAND_BYTES + G::RES_BYTES);
    // the colour shift of row r in pass c: its colour sites are x0 + 2j (even L, x0 = the shift)
    // or the x with ax(x) = s (odd L)
    auto row_shift = [](int c, int r) -> int {
        const int y = r % L, z = DIM == 3 ? r / L : 0;
        if constexpr (ODD) return ((c - ck_ax(L, y) - (DIM == 3 ? ck_ax(L, z) : 0)) % 3 + 3) % 3;
        else return (c + y + z) & 1;
    };
    if constexpr (ODD) {  // the consumer's per-row flip positions, once per launch
        for (int e = threadIdx.x; e < NCOL * G::NPR; e += blockDim.x) {
            const int c = e / G::NPR, r = e % G::NPR;
            uint32_t v = 0u, raw = 0xFFFFFFFFu;
            if (r < NR) {
                const int sh = row_shift(c, r);
                int n = 0;
                for (int x = 0; x < L; ++x)
                    if (ck_ax(L, x) == sh) {
                        v |= (uint32_t)x << (8 * n);
                        raw = (raw & ~(0xFFu << (8 * n))) | ((uint32_t)x << (8 * n));
                        ++n;
                    }
            }
            ftab[e] = v;  // unused slots: position 0 (they never accept)
            ftab[NCOL * G::NPR + e] = raw;
        }
    }
    const uint32_t *gsp = spins + td.spin_off;
    const uint32_t *gbd = bonds + td.bond_off;
    for (int row = warp; row < NR; row += kCkWarps) {
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
        JBs[row * W + ln] = jx | (jy << 1) | (jz << 2);
    }

    const int slot = tile * kTile + ln;
    SlotState ss = slots[slot];
    const bool active = ss.active != 0;
    const uint64_t lrow = td.w_base + (uint64_t)ln * G::B;
    // element (b, n) of this chain's table at byte offset b * RSB + n * NSB from `tab`; rows
    // -DIM .. B-1+DIM are addressable (zero padding), so a candidate row one move away from a
    // valid row needs no clamp.  Bin row offsets carry the base rb0: the table's 32-bit shared
    // address when it is read by shared addresses (SADDR), else 0
    constexpr int NSB = G::SMEM_THR ? 4 * W : 4;
    constexpr int RSB = 8 * NSB;
    const char *tab;
    if constexpr (G::SMEM_THR) {
        uint32_t *TH = reinterpret_cast<uint32_t *>(smem_raw + G::BASE_BYTES);
        if (warp == 1) {
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
    const int rb0 = G::SADDR ? (int)__cvta_generic_to_shared(tab) : 0;
    const uint64_t t0 = ss.t;
    const uint64_t n_pass = n_sweeps * NCOL;  // colour passes

    __syncthreads();
    // Every warp passes the same barriers: one after staging, per pass one fill barrier and NP
    // record barriers, one at the end.
    if (warp >= 1) {
        // ---- producers: record p of colour pass c (sweep t) into ring buffer k
        auto produce = [&](int c, int p, uint32_t t, int k) {
            uint4 *buf = hand + k * G::HQ * W;
            const int r0 = RPR * p;
            // a role's rows are dealt to its workers, the 32 / W lane groups of its two warps (a
            // narrow tile's lanes above W would otherwise repeat lanes 0 .. W-1): worker wk takes
            // rows wk, wk + NWK, ...; a loop of RH iterations with a guard keeps the trip count a
            // constant
            constexpr int NWK = 2 * (32 / W);
            constexpr int RH = (RPR + NWK - 1) / NWK;
            const int wk = (warp >= 4 ? 32 / W : 0) + lane / W;
            if (ck_random(warp)) {  // clamped as in the lexicographic kernel; padding: never accepts
                const uint32_t c3 = (uint32_t)(5 + c) | (ss.stream << 8);
#pragma unroll
                for (int hi = 0; hi < RH; ++hi) {
                    const int h = wk + hi * NWK;
                    if ((RPR % NWK) != 0 && h >= RPR) break;
                    const int r = r0 + h;
                    if constexpr (!ODD && !PADROWS) {  // every slot is a site
#pragma unroll
                        for (int g = 0; g < NGC; ++g) {
                            uint4 w = philox4x32_10(make_uint4((uint32_t)(4 * r + g), t, ss.rid, c3), key);
                            w.x = active ? min(w.x, kAlways - 1u) : kAlways;
                            w.y = active ? min(w.y, kAlways - 1u) : kAlways;
                            w.z = active ? min(w.z, kAlways - 1u) : kAlways;
                            w.w = active ? min(w.w, kAlways - 1u) : kAlways;
                            buf[(G::OFFQ + h * NGC + g) * W + ln] = w;
                        }
                    } else {
                        // odd L: the row's sites, the bytes of its list that are not 0xFF
                        const int nreal = r >= NR ? 0 : (ODD ? 4 - __popc((ftab[(NCOL + c) * G::NPR + r] >> 7) & 0x01010101u) : HALF);
#pragma unroll
                        for (int g = 0; g < NGC; ++g) {
                            uint4 w = make_uint4(kAlways, kAlways, kAlways, kAlways);
                            if (4 * g < nreal) {
                                w = philox4x32_10(make_uint4((uint32_t)(4 * r + g), t, ss.rid, c3), key);
                                const bool ok = active;
                                w.x = (ok && 4 * g + 0 < nreal) ? min(w.x, kAlways - 1u) : kAlways;
                                w.y = (ok && 4 * g + 1 < nreal) ? min(w.y, kAlways - 1u) : kAlways;
                                w.z = (ok && 4 * g + 2 < nreal) ? min(w.z, kAlways - 1u) : kAlways;
                                w.w = (ok && 4 * g + 3 < nreal) ? min(w.w, kAlways - 1u) : kAlways;
                            }
                            buf[(G::OFFQ + h * NGC + g) * W + ln] = w;
                        }
                    }
                }
                return;
            }
            // classes of row h (nibble 2j of s: the j-th colour site), stored as table offsets
            // n * NSB, 16 bits per attempt, the row's offsets from word h * OW
#pragma unroll
            for (int hi = 0; hi < RH; ++hi) {
            const int h = wk + hi * NWK;
            if ((RPR % NWK) != 0 && h >= RPR) break;
            const int r = r0 + h;
            if (PADROWS && r >= NR) {  // padding row: class dim in every slot (no move)
#pragma unroll
                for (int q = 0; q < G::OW; ++q) {
                    const int wd = h * G::OW + q;
                    reinterpret_cast<uint32_t *>(buf + (wd >> 2) * W + ln)[wd & 3] =
                        (uint32_t)(DIM * NSB) * 0x00010001u;
                }
                continue;
            }
            T s;
            uint32_t xs = 0u;  // odd L: the row's colour sites (bytes, 0xFF padding)
            {
                const int y = r % L, z = DIM == 3 ? r / L : 0;
                constexpr T M1 = ck_mask<T, L>() & (T)0x1111111111111111ull;  // bit 0 of every nibble
                const T R = Rs[r * W + ln], JB = JBs[r * W + ln];
                const T uxp = R ^ ck_next<T, L>(R) ^ (JB & M1);
                const int ryp = (y == L - 1) ? r - (L - 1) : r + 1;
                const int rym = (y == 0) ? r + (L - 1) : r - 1;
                T sum = uxp + ck_prev<T, L>(uxp) + (R ^ Rs[ryp * W + ln] ^ ((JB >> 1) & M1)) +
                        (R ^ Rs[rym * W + ln] ^ ((JBs[rym * W + ln] >> 1) & M1));
                if constexpr (DIM == 3) {
                    const int rzp = (z == L - 1) ? r - (L - 1) * L : r + L;
                    const int rzm = (z == 0) ? r + (L - 1) * L : r - L;
                    sum += (R ^ Rs[rzp * W + ln] ^ ((JB >> 2) & M1)) + (R ^ Rs[rzm * W + ln] ^ ((JBs[rzm * W + ln] >> 2) & M1));
                }
                if constexpr (ODD) {
                    s = sum;
                    xs = ftab[(NCOL + c) * G::NPR + r];
                } else {
                    s = sum >> (4 * row_shift(c, r));  // nibble 2j: the j-th colour site
                }
            }
            uint32_t off[G::OW];
#pragma unroll
            for (int q = 0; q < G::OW; ++q) off[q] = 0u;
#pragma unroll
            for (int j = 0; j < HALF; ++j) {
                uint32_t n;
                if constexpr (ODD) {
                    const uint32_t x = (xs >> (8 * j)) & 0xFFu;
                    n = x == 0xFFu ? (uint32_t)DIM : (uint32_t)((s >> (4 * x)) & 0xF);
                } else {
                    n = (uint32_t)((s >> (8 * j)) & 0xF);
                }
                off[j >> 1] |= (n * NSB) << (16 * (j & 1));
            }
#pragma unroll
            for (int q = 0; q < G::OW; ++q) {
                const int wd = h * G::OW + q;
                reinterpret_cast<uint32_t *>(buf + (wd >> 2) * W + ln)[wd & 3] = off[q];
            }
            }
        };
        const bool producer = ck_classes(warp) || ck_random(warp);
        // ---- measurement, one record behind the consumer
        int phase = ss.phase, nrt = ss.n_rt;
        int64_t tf = ss.t_first, tl = ss.t_last;
        const int topB = rb0 + ss.b_top * RSB, botB = rb0 + ss.b_g * RSB;
        int pmin = rb0 + ss.b_min * RSB, pnow = rb0 + ss.b * RSB;
        bool out_of_range = false;
        uint64_t mrec = 0;  // records measured
        auto measure = [&](uint64_t gm) {  // record gm: the bin row offset after each of its attempts
            const int *r = res + (int)(gm & 1) * NA * W + ln;
            int lo = 0x7FFFFFFF, hi = -0x7FFFFFFF;
            uint32_t mtop = 0u, mbot = 0u;
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                const int pr = r[a * W];
                lo = min(lo, pr);
                hi = max(hi, pr);
                mtop |= (uint32_t)(pr >= topB) << a;
                mbot |= (uint32_t)(pr <= botB) << a;
                if (a == NA - 1) pnow = pr;
            }
            pmin = min(pmin, lo);
            out_of_range |= (lo < rb0) | (hi > topB);
            const uint64_t sweep = mrec / (NCOL * NP);
            if (count_rt && active && ((phase == 1) ? mbot : mtop) != 0u) {
                const int64_t t = (int64_t)(t0 + sweep);
                int a0 = 0;
                while (a0 < NA) {
                    const uint32_t m = ((phase == 1) ? mbot : mtop) >> a0;
                    if (m == 0u) break;
                    a0 += __ffs(m);
                    if (phase == 0) { tf = t; phase = 1; }
                    else if (phase == 1) { phase = 2; }
                    else { nrt += 1; tl = t; phase = 1; }
                }
            }
            if (++mrec % (NCOL * NP) == 0 && active && owner) atomicAdd(&hist[lrow + (pnow - rb0) / RSB], 1u);
        };
        uint64_t g = 0;  // records the consumer has been given
        for (uint64_t q = 0; q < n_pass; ++q) {
            const int c = (int)(q % NCOL);
            const uint32_t t = (uint32_t)(t0 + q / NCOL);
            __syncthreads();  // fill barrier: the previous pass is complete
            if (warp == kCkMeasure && g > 0) measure(g - 1);
            if (producer)
                for (int p = 0; p < LAG; ++p) produce(c, p, t, (int)((g + p) % NBUF));
            for (int k = 0; k < NP; ++k) {
                __syncthreads();  // record barrier k: records .. k+LAG-1 complete, consumer done with k-1
                if (producer && k + LAG < NP) produce(c, k + LAG, t, (int)((g + LAG) % NBUF));
                if (warp == kCkMeasure && k > 0) measure(g - 1);
                ++g;
            }
        }
        __syncthreads();
        if (warp == kCkMeasure) {
            if (g > 0) measure(g - 1);
            ss.b = (pnow - rb0) / RSB;
            ss.b_min = (pmin - rb0) / RSB;
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
    // the previous attempt, applied lazily: row offset it was evaluated at (rq), offset change if
    // it was accepted (dq) and whether it was (pa)
    int rq = rb0 + ss.b * RSB, dq = 0;
    bool pa = false;
    uint32_t thA = 0u, thB = 0u;  // candidate thresholds of the next attempt (previous rejected / accepted)
    uint4 noff[G::OFFQ], nrr[RPR * NGC];  // the next record (read one barrier early)
    auto load_rec = [&](uint64_t gk) {
        const uint4 *buf = hand + (int)(gk % NBUF) * G::HQ * W;
#pragma unroll
        for (int q = 0; q < G::OFFQ; ++q) noff[q] = buf[q * W + ln];
#pragma unroll
        for (int i = 0; i < RPR * NGC; ++i) nrr[i] = buf[(G::OFFQ + i) * W + ln];
    };
    uint64_t g = 0;
    for (uint64_t q = 0; q < n_pass; ++q) {
        const int c = (int)(q % NCOL);
        __syncthreads();  // fill barrier
        bool have_next = false;
        for (int k = 0; k < NP; ++k, ++g) {
            __syncthreads();  // record barrier k
            if (LAG == 1 || k == 0) load_rec(g);
            uint32_t off[4 * G::OFFQ];  // 16-bit class offset of attempt (h, j) at bits 16 (j & 1) of off[h OW + j / 2]
#pragma unroll
            for (int q = 0; q < G::OFFQ; ++q) {
                off[4 * q] = noff[q].x; off[4 * q + 1] = noff[q].y; off[4 * q + 2] = noff[q].z; off[4 * q + 3] = noff[q].w;
            }
            uint4 rr[RPR * NGC];
#pragma unroll
            for (int i = 0; i < RPR * NGC; ++i) rr[i] = nrr[i];
            const bool more = k + 1 < NP;  // a next record in this pass
            if (LAG >= 2 && more) load_rec(g + 1);
            const int r0 = RPR * k;
            int on = (int)(off[0] & 0xFFFFu);  // this attempt's class offset
            if (!have_next) {
                thA = ck_thr<G::SMEM_THR, G::SADDR>(tab, rq + on);
                thB = ck_thr<G::SMEM_THR, G::SADDR>(tab, rq + dq + on);
            }
            have_next = false;
            int *resb = res + (int)(g & 1) * NA * W + ln;
            // even L: bit 8j of flipped[h] is the row's j-th colour site (spread at the row's end);
            // odd L: the site's own nibble, at the shifts fsh of the row's colour sites
            T flipped[RPR], rold[RPR];  // rold: the record's spin rows, read before its attempts
            uint32_t fsh[RPR];
#pragma unroll
            for (int h = 0; h < RPR; ++h) {
                flipped[h] = 0;
                rold[h] = (!PADROWS || r0 + h < NR) ? Rs[(r0 + h) * W + ln] : T(0);
                if constexpr (ODD) fsh[h] = ftab[c * G::NPR + r0 + h];  // padding slots at x = 0: they never accept
            }
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                const int h = a / HALF, j = a % HALF;
                // the next attempt's class offset: this record's, or the next record's first
                int off1 = 0;
                bool next = true;
                if (a + 1 < NA) {
                    const int h1 = (a + 1) / HALF, j1 = (a + 1) % HALF, wd = h1 * G::OW + (j1 >> 1);
                    off1 = (int)((off[wd] >> (16 * (j1 & 1))) & 0xFFFFu);
                } else if (LAG >= 2 && more) {
                    off1 = (int)(noff[0].x & 0xFFFFu);
                    have_next = true;
                } else {
                    next = false;
                }
                const int dx = DIM * RSB - 8 * on;  // bin change if accepted: (dim - n) rows
                const int rB = rq + dq;
                // all four candidate addresses first; the previous decision only selects.  The
                // next attempt's loads are issued before this attempt's threshold is used, so that
                // their latency overlaps this decision (a warp issues in order)
                const int aA0 = rq + off1, aA1 = rB + off1, aB0 = aA0 + dx, aB1 = aA1 + dx;
                uint32_t nA = 0u, nB = 0u;
                if (next) {
                    nA = ck_thr<G::SMEM_THR, G::SADDR>(tab, pa ? aA1 : aA0);
                    nB = ck_thr<G::SMEM_THR, G::SADDR>(tab, pa ? aB1 : aB0);
                }
                const uint32_t th = pa ? thB : thA;
                const int rx = pa ? rB : rq;
                const uint32_t r = uint4_get(rr[h * NGC + (j >> 2)], j & 3);
                const bool acc = r < th;  // r clamped by the producer
                if constexpr (ODD) {
                    flipped[h] |= T(acc ? 1u : 0u) << (4 * ((fsh[h] >> (8 * j)) & 0xFu));
                } else {
                    flipped[h] |= T(acc ? 1u : 0u) << (8 * j);
                }
                resb[a * W] = acc ? rx + dx : rx;  // bin row offset after the attempt, for the measurement
                rq = rx;
                dq = dx;
                pa = acc;
                on = off1;
                if (next) {
                    thA = nA;
                    thB = nB;
                }
            }
#pragma unroll
            for (int h = 0; h < RPR; ++h) {
                const int r = r0 + h;
                if (!PADROWS || r < NR) {  // padding rows have no spins
                    if constexpr (ODD) Rs[r * W + ln] = rold[h] ^ flipped[h];
                    else Rs[r * W + ln] = rold[h] ^ (flipped[h] << (4 * row_shift(c, r)));
                }
            }
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

// Kernels for the even sizes, the odd sizes and both: a context of one parity gets a kernel whose
// register allocation is that of its own sizes (the odd sizes' larger records need more); a
// context holding both gets one launch for all its tiles.  MODE 0 even, 1 odd, 2 both.
template <int DIM, int MODE>
__global__ void __launch_bounds__(kCkThreads, 1)
muca_checker_kernel(const TileDesc *__restrict__ tiles, SlotState *__restrict__ slots, uint32_t *__restrict__ spins,
                    const uint32_t *__restrict__ bonds, const uint32_t *__restrict__ thr,
                    uint32_t *__restrict__ hist, uint64_t n_sweeps, PhiloxKey key, int count_rt,
                    unsigned *__restrict__ diag) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const TileDesc td = tiles[blockIdx.x];
    const bool odd = (td.L & 1) != 0;
    if (((MODE == 0 || MODE == 3) && odd) || (MODE == 1 && !odd)) return;  // the whole CTA, before any barrier
    const uint64_t n_tile = n_sweeps * (uint64_t)(td.sweep_mul > 0 ? td.sweep_mul : 1);
#define EAMC_CK(LL, WW) checker_tile<DIM, LL, WW>(td, blockIdx.x, slots, spins, bonds, thr, hist, n_tile, key, count_rt, diag, smem_raw)
    // narrow tiles (3D): 16 chains at L = 4..8, 8 at L = 4..10, 4 at L = 11, 12, each chain on
    // 32 / width lanes, so that the thresholds fit in shared memory (L >= 7) or a batch spreads
    // over more SMs, each with a smaller share of the producer work (L <= 8)
    if (td.width != 32) {
        if constexpr (DIM == 3) {
            if constexpr (MODE == 1 || MODE == 2) {
                if (td.width == 16 && td.L == 7) EAMC_CK(7, 16);
                else if (td.width == 8 && td.L == 7) EAMC_CK(7, 8);
                else if (td.width == 16 && td.L == 5) EAMC_CK(5, 16);
                else if (td.width == 8 && td.L == 5) EAMC_CK(5, 8);
                else if (td.width == 8 && td.L == 9) EAMC_CK(9, 8);
                else if (td.width == 4 && td.L == 11) EAMC_CK(11, 4);
            }
            if constexpr (MODE != 1) {
                if (td.width == 16 && td.L == 8) EAMC_CK(8, 16);
                else if (td.width == 8 && td.L == 8) EAMC_CK(8, 8);
                else if (td.width == 8 && td.L == 10) EAMC_CK(10, 8);
                else if (td.width == 4 && td.L == 12) EAMC_CK(12, 4);
            }
            // the small even sizes' narrow tiles in forms of their own (MODE 3, and 2 for both
            // parities): compiled into the even-size form they cost L = 8 1 % through its code
            if constexpr (MODE >= 2) {
                if (td.width == 16 && td.L == 4) EAMC_CK(4, 16);
                else if (td.width == 8 && td.L == 4) EAMC_CK(4, 8);
                else if (td.width == 16 && td.L == 6) EAMC_CK(6, 16);
                else if (td.width == 8 && td.L == 6) EAMC_CK(6, 8);
            }
        }
        return;
    }
    if constexpr (MODE == 1 || MODE == 2) {
        switch (td.L) {
            case 3: EAMC_CK(3, 32); break;
            case 5: EAMC_CK(5, 32); break;
            case 7: EAMC_CK(7, 32); break;
            case 9: EAMC_CK(9, 32); break;
            case 11: EAMC_CK(11, 32); break;
            default: break;
        }
    }
    if constexpr (MODE != 1) {
        switch (td.L) {
            case 4: EAMC_CK(4, 32); break;
            case 6: EAMC_CK(6, 32); break;
            case 8: EAMC_CK(8, 32); break;
            case 10: EAMC_CK(10, 32); break;
            case 12: EAMC_CK(12, 32); break;
            default: break;
        }
    }
#undef EAMC_CK
}

template <int DIM, int MODE>
cudaError_t ck_launch(int n_tiles, size_t smem, cudaStream_t st, const TileDesc *d_tiles, SlotState *d_slots,
                      uint32_t *d_spins, const uint32_t *d_bonds, const uint32_t *d_thr, uint32_t *d_hist,
                      uint64_t n_sweeps, PhiloxKey key, int count_rt, unsigned *d_diag) {
    static size_t set_limit = 0;
    if (smem > set_limit) {
        const cudaError_t e = cudaFuncSetAttribute(muca_checker_kernel<DIM, MODE>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        set_limit = smem;
    }
    muca_checker_kernel<DIM, MODE><<<n_tiles, kCkThreads, smem, st>>>(d_tiles, d_slots, d_spins, d_bonds, d_thr,
                                                                       d_hist, n_sweeps, key, count_rt, d_diag);
    return cudaGetLastError();
}

template <int DIM, int W>
size_t checker_smem_w(int L) {
    switch (L) {
        case 3: return CkGeo<DIM, 3, W>::SMEM;
        case 4: return CkGeo<DIM, 4, W>::SMEM;
        case 5: return CkGeo<DIM, 5, W>::SMEM;
        case 6: return CkGeo<DIM, 6, W>::SMEM;
        case 7: return CkGeo<DIM, 7, W>::SMEM;
        case 8: return CkGeo<DIM, 8, W>::SMEM;
        case 9: return CkGeo<DIM, 9, W>::SMEM;
        case 10: return CkGeo<DIM, 10, W>::SMEM;
        case 11: return CkGeo<DIM, 11, W>::SMEM;
        case 12: return CkGeo<DIM, 12, W>::SMEM;
        default: return 0;
    }
}

}  // namespace

size_t checker_smem_bytes(int dim, int L, int width) {
    if (L < 3 || L > 12) return 0;
    if (width != 32) {
        if (dim != 3) return 0;
        if (width == 16) {
            switch (L) {
                case 4: return CkGeo<3, 4, 16>::SMEM;
                case 5: return CkGeo<3, 5, 16>::SMEM;
                case 6: return CkGeo<3, 6, 16>::SMEM;
                case 7: return CkGeo<3, 7, 16>::SMEM;
                case 8: return CkGeo<3, 8, 16>::SMEM;
                default: return 0;
            }
        }
        if (width == 8) {
            switch (L) {
                case 4: return CkGeo<3, 4, 8>::SMEM;
                case 5: return CkGeo<3, 5, 8>::SMEM;
                case 6: return CkGeo<3, 6, 8>::SMEM;
                case 7: return CkGeo<3, 7, 8>::SMEM;
                case 8: return CkGeo<3, 8, 8>::SMEM;
                case 9: return CkGeo<3, 9, 8>::SMEM;
                case 10: return CkGeo<3, 10, 8>::SMEM;
                default: return 0;
            }
        }
        if (width == 4) return L == 11 ? CkGeo<3, 11, 4>::SMEM : (L == 12 ? CkGeo<3, 12, 4>::SMEM : 0);
        return 0;
    }
    if (width != 32) return 0;
    return dim == 3 ? checker_smem_w<3, 32>(L) : checker_smem_w<2, 32>(L);
}

int checker_parity_class(int dim, int L, int width) {
    if (L & 1) return 2;
    return (dim == 3 && width != 32 && L <= 6) ? 4 : 1;
}

bool checker_thresholds_in_smem(int dim, int L, int width) {
    if (checker_smem_bytes(dim, L, width) == 0) return false;
#define EAMC_TS(D, LL, WW) if (dim == D && L == LL && width == WW) return CkGeo<D, LL, WW>::SMEM_THR;
    EAMC_TS(3, 7, 16) EAMC_TS(3, 8, 16) EAMC_TS(3, 8, 8) EAMC_TS(3, 4, 16) EAMC_TS(3, 5, 16) EAMC_TS(3, 6, 16)
    EAMC_TS(3, 4, 8) EAMC_TS(3, 5, 8) EAMC_TS(3, 6, 8) EAMC_TS(3, 7, 8) EAMC_TS(3, 9, 8) EAMC_TS(3, 10, 8) EAMC_TS(3, 11, 4) EAMC_TS(3, 12, 4)
    EAMC_TS(3, 3, 32) EAMC_TS(3, 4, 32) EAMC_TS(3, 5, 32) EAMC_TS(3, 6, 32) EAMC_TS(3, 7, 32) EAMC_TS(3, 8, 32)
    EAMC_TS(3, 9, 32) EAMC_TS(3, 10, 32) EAMC_TS(3, 11, 32) EAMC_TS(3, 12, 32)
    EAMC_TS(2, 3, 32) EAMC_TS(2, 4, 32) EAMC_TS(2, 5, 32) EAMC_TS(2, 6, 32) EAMC_TS(2, 7, 32) EAMC_TS(2, 8, 32)
    EAMC_TS(2, 9, 32) EAMC_TS(2, 10, 32) EAMC_TS(2, 11, 32) EAMC_TS(2, 12, 32)
#undef EAMC_TS
    return false;
}

cudaError_t launch_sweeps_checker(const TileDesc *d_tiles, int n_tiles, int dim, size_t smem, SlotState *d_slots,
                                  uint32_t *d_spins, const uint32_t *d_bonds, const uint32_t *d_thr,
                                  uint32_t *d_hist, uint64_t n_sweeps, PhiloxKey key, int count_rt,
                                  unsigned *d_diag, cudaStream_t st, int parities) {
    if (n_tiles <= 0 || n_sweeps == 0 || parities == 0) return cudaSuccess;
    // bit 0 even sizes, bit 1 odd sizes, bit 2 the small even sizes' narrow tiles
    const bool odd = (parities & 2) != 0, small = (parities & 4) != 0;
    const int mode = odd ? ((parities & 5) ? 2 : 1) : (small ? 3 : 0);
#define EAMC_CKL(D, M) ck_launch<D, M>(n_tiles, smem, st, d_tiles, d_slots, d_spins, d_bonds, d_thr, d_hist, n_sweeps, key, count_rt, d_diag)
    if (dim == 3) {
        switch (mode) {
            case 0: return EAMC_CKL(3, 0);
            case 1: return EAMC_CKL(3, 1);
            case 3: return EAMC_CKL(3, 3);
            default: return EAMC_CKL(3, 2);
        }
    }
    return mode == 0 ? EAMC_CKL(2, 0) : (mode == 1 ? EAMC_CKL(2, 1) : EAMC_CKL(2, 2));
#undef EAMC_CKL
}

}  // namespace eamc
