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
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "eamc_internal.cuh"

namespace eamc {

namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;

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

template <int DIM, int L>
struct Geo {
    using T = RowT<L>;
    static constexpr int NR = DIM == 3 ? L * L : L;          // rows along x
    static constexpr int V = NR * L;
    static constexpr int B = ((DIM * V) / 2 >> 1) + 1;       // table rows per chain
    static constexpr int NG = (L + 3) / 4;                   // Philox calls per row
    static constexpr int FIELDS = DIM + 2;                   // S, Jx, Jx(shifted), Jy, (Jz)
    static constexpr size_t LATTICE_BYTES = (size_t)FIELDS * NR * 32 * sizeof(T);
    static constexpr size_t THR_BYTES = (size_t)B * 8 * 32 * sizeof(uint32_t);
    static constexpr bool SMEM_THR = LATTICE_BYTES + THR_BYTES <= 200 * 1024;
    static constexpr size_t SMEM = LATTICE_BYTES + (SMEM_THR ? THR_BYTES : 0);
};

template <bool SMEM>
__device__ __forceinline__ uint32_t load_thr(const uint32_t *p) {
    if constexpr (SMEM) return *p;
    else return __ldg(p);
}

template <int DIM, int L>
__device__ __forceinline__ void sweep_tile(const TileDesc &td, int tile, SlotState *__restrict__ slots,
                                           uint32_t *__restrict__ spins,
                                           const uint32_t *__restrict__ bonds,
                                           const uint32_t *__restrict__ thr,
                                           uint32_t *__restrict__ hist, uint64_t n_sweeps,
                                           PhiloxKey key, int count_rt, unsigned char *smem_raw) {
    using G = Geo<DIM, L>;
    using T = typename G::T;
    constexpr int NR = G::NR;
    constexpr T NIB = nib_mask<T, L>();
    constexpr T LASTNIB = T(1) << (4 * (L - 1));
    const int lane = threadIdx.x;

    // ---- stage this lane's lattice as nibble-packed row words
    T *sm = reinterpret_cast<T *>(smem_raw);
    T *Rs = sm;                  // spins, nibble x = 1 if S = -1
    T *JXs = sm + NR * 32;       // nibble x: bond (x, x+1) has J = -1
    T *JXms = sm + 2 * NR * 32;  // nibble x: bond (x-1, x) has J = -1
    T *JYs = sm + 3 * NR * 32;   // nibble x: bond (x,y)-(x,y+1)
    T *JZs = sm + 4 * NR * 32;   // nibble x: bond (x,y,z)-(x,y,z+1)   (DIM == 3)
    const uint32_t *gsp = spins + td.spin_off;
    const uint32_t *gbd = bonds + td.bond_off;
    for (int row = 0; row < NR; ++row) {
        T r = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
        for (int x = 0; x < L; ++x) {
            const int i = row * L + x;
            r |= T((gsp[i] >> lane) & 1u) << (4 * x);
            jx |= T((gbd[i * DIM + 0] >> lane) & 1u) << (4 * x);
            jy |= T((gbd[i * DIM + 1] >> lane) & 1u) << (4 * x);
            if constexpr (DIM == 3) jz |= T((gbd[i * DIM + 2] >> lane) & 1u) << (4 * x);
        }
        Rs[row * 32 + lane] = r;
        JXs[row * 32 + lane] = jx;
        JXms[row * 32 + lane] = rot_prev<T, L>(jx);
        JYs[row * 32 + lane] = jy;
        if constexpr (DIM == 3) JZs[row * 32 + lane] = jz;
    }

    const int slot = tile * kTile + lane;
    SlotState ss = slots[slot];
    const bool active = ss.active != 0;
    const uint64_t lrow = td.w_base + (uint64_t)lane * G::B;
    // element (b, n) of this lane's table at tab[b * RS + n * NS]
    constexpr int NS = G::SMEM_THR ? 32 : 1;
    constexpr int RS = 8 * NS;
    const uint32_t *tab;
    if constexpr (G::SMEM_THR) {
        uint32_t *TH = reinterpret_cast<uint32_t *>(smem_raw + G::LATTICE_BYTES);
        const uint4 *src = reinterpret_cast<const uint4 *>(thr + lrow * 8);
        for (int b = 0; b < G::B; ++b) {
            const uint4 a = src[2 * b], c = src[2 * b + 1];
            uint32_t *d = TH + b * 256 + lane;
            d[0] = a.x; d[32] = a.y; d[64] = a.z; d[96] = a.w;
            d[128] = c.x; d[160] = c.y; d[192] = c.z; d[224] = c.w;
        }
        tab = TH + lane;
    } else {
        tab = thr + lrow * 8;
    }
    __syncwarp();

    int bmin = ss.b_min, phase = ss.phase, nrt = ss.n_rt;
    const int btop = ss.b_top, bg = ss.b_g;
    int64_t tf = ss.t_first, tl = ss.t_last;
    const uint64_t t0 = ss.t;
    const uint32_t rid = ss.rid, c3 = ss.stream << 8;
    uint32_t *hist_l = hist + lrow;
    // outcome of the previous attempt, applied lazily: bin before it (bq), its unsatisfied
    // count (pn) and whether it was accepted (pa)
    int bq = ss.b, pn = DIM, pa = 0;
    int bnow = ss.b;

    for (uint64_t s = 0; s < n_sweeps; ++s) {
        const uint64_t t = t0 + s;
        const uint32_t tt = (uint32_t)t;
        int y = 0, z = 0;
        for (int row = 0; row < NR; ++row) {
            const int rym = (y == 0) ? row + (L - 1) : row - 1;
            const int ryp = (y == L - 1) ? row - (L - 1) : row + 1;
            const T R = Rs[row * 32 + lane];
            const T u_yp = R ^ Rs[ryp * 32 + lane] ^ JYs[row * 32 + lane];
            const T u_ym = R ^ Rs[rym * 32 + lane] ^ JYs[rym * 32 + lane];
            const T u_xp = R ^ rot_next<T, L>(R) ^ JXs[row * 32 + lane];
            const T u_xm = R ^ rot_prev<T, L>(R) ^ JXms[row * 32 + lane];
            T sum = u_yp + u_ym + (u_xp & ~LASTNIB);
            if constexpr (DIM == 3) {
                const int rzm = (z == 0) ? row + (L - 1) * L : row - L;
                const int rzp = (z == L - 1) ? row - (L - 1) * L : row + L;
                sum += (R ^ Rs[rzp * 32 + lane] ^ JZs[row * 32 + lane]) +
                       (R ^ Rs[rzm * 32 + lane] ^ JZs[rzm * 32 + lane]);
            }
            const T sumA = sum + u_xm;          // -x bond as before the row
            const T sumB = sum + (u_xm ^ NIB);  // -x bond toggled by a flip of site x-1
            uint4 rr[G::NG];
#pragma unroll
            for (int g = 0; g < G::NG; ++g)
                rr[g] = philox4x32_10(make_uint4((uint32_t)(4 * row + g), tt, rid, c3), key);
            T accN = 0;  // nibble x = 1 if this chain flipped site x of the row
#pragma unroll
            for (int x = 0; x < L; ++x) {
                int nA = (int)((sumA >> (4 * x)) & 0xF);
                int nB = (x == 0) ? nA : (int)((sumB >> (4 * x)) & 0xF);
                if (x == L - 1) {  // bond to site 0 of the row, flipped at x = 0 or not
                    const int w = (int)((u_xp >> (4 * (L - 1))) & 1u) ^ (int)(accN & 1u);
                    nA += w;
                    nB += w;
                }
                const int bA = bq;
                const int bB = min(max(bq + DIM - pn, 0), G::B - 1);
                const uint32_t thA = load_thr<G::SMEM_THR>(tab + bA * RS + nA * NS);
                const uint32_t thB = load_thr<G::SMEM_THR>(tab + bB * RS + nB * NS);
                const int n = pa ? nB : nA;
                const uint32_t th = pa ? thB : thA;
                const int bx = pa ? bB : bA;
                const uint32_t r = uint4_get(rr[x >> 2], x & 3);
                const bool acc = active && (th == kAlways || r < th);
                accN |= T(acc ? 1u : 0u) << (4 * x);
                bnow = acc ? bx + DIM - n : bx;
                bmin = min(bmin, bnow);
                if (count_rt && active) {
                    const bool trig = (phase == 1) ? (bnow <= bg) : (bnow >= btop);
                    if (trig) {
                        if (phase == 0) { tf = (int64_t)t; phase = 1; }
                        else if (phase == 1) { phase = 2; }
                        else { nrt += 1; tl = (int64_t)t; phase = 1; }
                    }
                }
                pa = acc ? 1 : 0;
                pn = n;
                bq = bx;
            }
            Rs[row * 32 + lane] = R ^ accN;
            if (++y == L) { y = 0; ++z; }
        }
        if (active) hist_l[bnow] += 1u;
    }
    __syncwarp();
    // spins back to the multi-spin-coded global layout
    for (int row = 0; row < NR; ++row) {
        const T R = Rs[row * 32 + lane];
#pragma unroll
        for (int x = 0; x < L; ++x) {
            const uint32_t m = __ballot_sync(kFull, ((R >> (4 * x)) & 1u) != 0);
            if (lane == 0) spins[td.spin_off + row * L + x] = m;
        }
    }
    ss.b = bnow;
    ss.b_min = bmin;
    ss.phase = phase;
    ss.n_rt = nrt;
    ss.t_first = tf;
    ss.t_last = tl;
    ss.t = t0 + n_sweeps;
    if (count_rt && active && energy_of_bin(DIM * G::V, ss.parity, bmin) < ss.e_g) ss.requeue = 1;
    slots[slot] = ss;
}

// One warp (32 chains of one tile) per block; the tile's L selects the compiled body.
template <int DIM>
__global__ void __launch_bounds__(32, 1)
muca_sweep_kernel(const TileDesc *__restrict__ tiles, const int32_t *__restrict__ tile_list,
                  SlotState *__restrict__ slots, uint32_t *__restrict__ spins,
                  const uint32_t *__restrict__ bonds, const uint32_t *__restrict__ thr,
                  uint32_t *__restrict__ hist, uint64_t n_sweeps, PhiloxKey key, int count_rt) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tile = tile_list ? tile_list[blockIdx.x] : (int)blockIdx.x;
    const TileDesc td = tiles[tile];
#define EAMC_CASE(LL)                                                                      \
    case LL:                                                                               \
        sweep_tile<DIM, LL>(td, tile, slots, spins, bonds, thr, hist, n_sweeps, key, count_rt, \
                            smem_raw);                                                     \
        break;
    switch (td.L) {
        EAMC_CASE(3) EAMC_CASE(4) EAMC_CASE(5) EAMC_CASE(6) EAMC_CASE(7)
        EAMC_CASE(8) EAMC_CASE(9) EAMC_CASE(10) EAMC_CASE(11) EAMC_CASE(12)
        default: break;
    }
#undef EAMC_CASE
}

template <int DIM>
size_t smem_for(int L) {
    switch (L) {
        case 3: return Geo<DIM, 3>::SMEM;
        case 4: return Geo<DIM, 4>::SMEM;
        case 5: return Geo<DIM, 5>::SMEM;
        case 6: return Geo<DIM, 6>::SMEM;
        case 7: return Geo<DIM, 7>::SMEM;
        case 8: return Geo<DIM, 8>::SMEM;
        case 9: return Geo<DIM, 9>::SMEM;
        case 10: return Geo<DIM, 10>::SMEM;
        case 11: return Geo<DIM, 11>::SMEM;
        case 12: return Geo<DIM, 12>::SMEM;
        default: return 0;
    }
}

}  // namespace

size_t sweep_smem_bytes(int dim, int L) { return dim == 3 ? smem_for<3>(L) : smem_for<2>(L); }

cudaError_t launch_sweeps(const TileDesc *d_tiles, const int32_t *d_tile_list, int n_blocks, int dim,
                          size_t smem, SlotState *d_slots, uint32_t *d_spins, const uint32_t *d_bonds,
                          const uint32_t *d_thr, uint32_t *d_hist, uint64_t n_sweeps, PhiloxKey key,
                          int count_rt, cudaStream_t st) {
    if (n_blocks <= 0 || n_sweeps == 0) return cudaSuccess;
    cudaError_t e;
    if (dim == 3) {
        e = cudaFuncSetAttribute(muca_sweep_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        muca_sweep_kernel<3><<<n_blocks, 32, smem, st>>>(d_tiles, d_tile_list, d_slots, d_spins, d_bonds,
                                                         d_thr, d_hist, n_sweeps, key, count_rt);
    } else {
        e = cudaFuncSetAttribute(muca_sweep_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        muca_sweep_kernel<2><<<n_blocks, 32, smem, st>>>(d_tiles, d_tile_list, d_slots, d_spins, d_bonds,
                                                         d_thr, d_hist, n_sweeps, key, count_rt);
    }
    return cudaGetLastError();
}

}  // namespace eamc
