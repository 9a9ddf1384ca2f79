// muca_colour.cu -- a2 + a3 in the colour order for odd L: the multicanonical sweep with the
// sites of a sweep taken colour class by colour class (the PT colouring, three classes for odd
// L), each class in lexicographic order.  Even L (the checkerboard) runs in muca_checker.cu.
//
// The paper fixes no order of the attempts within a sweep.  In this order no two sites of a
// colour pass are neighbours, so every attempt's class n (unsatisfied bonds; the move changes
// the bin by dim - n) is fixed when the pass begins; the only sequential coupling between the
// attempts of a pass is the energy bin of the chain (Eq. "muca": the acceptance depends on
// W(E_new)/W(E_old)).  That is used here as follows.  One warp runs one chain, taking the
// attempts of a pass in blocks of K = 4.  Lane l assumes that the block starts at bin lo + l,
// where lo is the lowest bin the block can start from given the bin at the start of the
// previous block (the possible starts span at most 3K + 1 <= 13 bins).  For every attempt i of
// the block, lane l loads the threshold of bin mlo + l (mlo = lo minus the block's largest
// possible descent) and a ballot gives the acceptance mask of attempt i over 32 bins, which
// covers every bin a path of the block can visit from any possible start.  Each lane then walks
// the block from its own start bin through the masks (registers only), and one shuffle from the
// lane of the actual start gives the block's end bin and its accepted attempts.  So the
// dependency from one block to the next is a shuffle; the threshold loads and the walks of the
// next block overlap with it.  The decisions are the same as taking the attempts one after the
// other.  Round trips, the lowest bin and the range checks are per-attempt rules (Sec. III); a
// block whose bin range [start + descent, start + ascent] stays clear of the top, the bottom
// E_g and the lowest bin so far cannot change them, any other block is replayed attempt by
// attempt from its accepted moves.
//
// Random words (the colour-order streams): the j-th colour-c site of row r takes word j&3 of
// Philox call (4 r + j/4, t, rid, (5 + c) | stream << 8); for odd L <= 11 a row has at most four
// sites of a colour, so one call per row and colour.
//
// Layout.  A CTA of C warps (C <= 8) takes chains c0 .. c0+C-1 of one tile (bit c of the tile's
// multi-spin-coded words).  Shared memory: the tile's spin and coupling words (flips of a
// chain are atomic XORs of its bit), and per chain its thresholds transposed class-major
// (T[n][b], so that a window of bins is contiguous), the sweep's random words by colour site
// (each colour's segment padded to a multiple of K with words that never accept), and the
// classes of the current pass (padded with class dim: no move).  At the end of a launch each
// CTA XORs its own bits' changes into the global spin words.
#include <cuda_runtime.h>

#include <cstdint>

#include "eamc_internal.cuh"

namespace eamc {

namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr int kBlk = 4;  // attempts resolved together

template <int DIM, int L>
struct CGeo {
    static_assert((L & 1) != 0 && L <= 11, "odd L up to 11: at most four sites of a colour per row");
    static constexpr int NR = DIM == 3 ? L * L : L;
    static constexpr int V = NR * L;
    static constexpr int B = ((DIM * V) / 2 >> 1) + 1;
    static constexpr int NCOL = 3;
    static constexpr int NMAX = V;                    // sites of the largest colour (bound)
    static constexpr int RWN = ((V + 3) & ~3) + 4 * NCOL;  // random words, padded segments
    static constexpr int NCB = (((NMAX + 3) & ~3) + 15) & ~15;  // class bytes of a pass, padded
    static constexpr int NFB = ((NCB / 4) + 15) & ~15;           // accepted-attempt nibbles, a byte per block
    // shared memory: S, S0 [V], J [DIM*V], colour offsets [4], segment bases [4], sites by
    // colour [V] and random-word index of each site [V]; per chain: T [8][B], Rw [RWN],
    // Nc [NCB], Fb [NFB]
    static constexpr size_t TILE_BYTES = (size_t)(2 + DIM) * V * 4 + (size_t)2 * V * 2 + 32;
    static constexpr size_t CHAIN_BYTES = (size_t)8 * B * 4 + (size_t)RWN * 4 + NCB + NFB;
    static size_t smem(int C) { return ((TILE_BYTES + 15) & ~(size_t)15) + (size_t)C * CHAIN_BYTES; }
};

// colour of site (x, y, z) (the PT colouring: neighbours never share a colour)
template <int DIM, int L>
__device__ __forceinline__ int ccolour_xyz(int x, int y, int z) {
    auto ax = [](int c) { return (c == L - 1 && (L - 1) % 3 == 0) ? 1 : c % 3; };
    return (ax(x) + ax(y) + (DIM == 3 ? ax(z) : 0)) % 3;
}

template <int DIM, int L>
__device__ __forceinline__ int ccolour(int i) {
    return ccolour_xyz<DIM, L>(i % L, (i / L) % L, DIM == 3 ? i / (L * L) : 0);
}

// unsatisfied bonds of chain bit c at site i = (x, y, z): bond (i, i + e_d) has coupling word
// Jw[i*DIM + d]
template <int DIM, int L>
__device__ __forceinline__ int unsat_count(const uint32_t *S, const uint32_t *Jw, int i, int x, int y, int z, int c) {
    const uint32_t si = S[i];
    const int ixp = x == L - 1 ? i - (L - 1) : i + 1, ixm = x == 0 ? i + (L - 1) : i - 1;
    const int iyp = y == L - 1 ? i - L * (L - 1) : i + L, iym = y == 0 ? i + L * (L - 1) : i - L;
    uint32_t n = ((si ^ S[ixp] ^ Jw[i * DIM + 0]) >> c & 1u) + ((si ^ S[ixm] ^ Jw[ixm * DIM + 0]) >> c & 1u) +
                 ((si ^ S[iyp] ^ Jw[i * DIM + 1]) >> c & 1u) + ((si ^ S[iym] ^ Jw[iym * DIM + 1]) >> c & 1u);
    if constexpr (DIM == 3) {
        const int izp = z == L - 1 ? i - L * L * (L - 1) : i + L * L, izm = z == 0 ? i + L * L * (L - 1) : i - L * L;
        n += ((si ^ S[izp] ^ Jw[i * DIM + 2]) >> c & 1u) + ((si ^ S[izm] ^ Jw[izm * DIM + 2]) >> c & 1u);
    }
    return (int)n;
}

template <int DIM, int L>
__device__ void colour_tile(const TileDesc &td, int tile, int c0, int C, SlotState *__restrict__ slots,
                            uint32_t *__restrict__ spins, const uint32_t *__restrict__ bonds,
                            const uint32_t *__restrict__ thr, uint32_t *__restrict__ hist, uint64_t n_sweeps,
                            PhiloxKey key, int count_rt, unsigned *__restrict__ diag, unsigned char *smem_raw) {
    using G = CGeo<DIM, L>;
    constexpr int V = G::V, B = G::B, NR = G::NR, NCOL = G::NCOL;
    constexpr uint32_t kDimBytes = 0x01010101u * (uint32_t)DIM;  // four padding attempts
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *S = reinterpret_cast<uint32_t *>(smem_raw);
    uint32_t *S0 = S + V;
    uint32_t *Jw = S0 + V;
    int *Coff = reinterpret_cast<int *>(Jw + DIM * V);          // [4] colour offsets in CL,
    int *RBo = Coff + 4;                                        // [4] random-word segment bases,
    uint16_t *CL = reinterpret_cast<uint16_t *>(RBo + 4);       // [V] sites by colour,
    uint16_t *RI = CL + V;                                      // [V] random-word index of a site
    unsigned char *chain_base = smem_raw + ((G::TILE_BYTES + 15) & ~(size_t)15);

    // ---- the tile's lattice words (all threads), colour lists
    for (int k = threadIdx.x; k < V; k += blockDim.x) {
        const uint32_t w = spins[td.spin_off + k];
        S[k] = w;
        S0[k] = w;
    }
    for (int k = threadIdx.x; k < DIM * V; k += blockDim.x) Jw[k] = bonds[td.bond_off + k];
    {
        if (threadIdx.x < 32) {  // warp 0 compacts each colour's sites in lexicographic order
            const int ln = threadIdx.x;
            int n = 0, rb = 0;
            for (int c = 0; c < NCOL; ++c) {
                const int start = n;  // the same in every lane
                if (ln == 0) { Coff[c] = start; RBo[c] = rb; }
                for (int i0 = 0; i0 < V; i0 += 32) {
                    const int i = i0 + ln;
                    const bool in = i < V && ccolour<DIM, L>(i) == c;
                    const uint32_t bal = __ballot_sync(kFull, in);
                    const int pos = n + __popc(bal & ((1u << ln) - 1u));
                    if (in) { CL[pos] = (uint16_t)i; RI[i] = (uint16_t)(rb + pos - start); }
                    n += __popc(bal);
                    __syncwarp();
                }
                rb += (n - start + 3) & ~3;
            }
            if (ln == 0) { Coff[NCOL] = n; RBo[NCOL] = rb; }
        }
    }
    __syncthreads();

    const int c = c0 + warp;  // this warp's chain (lane of the tile)
    if (warp >= C || c >= td.width) return;
    const int slot = tile * kTile + c;
    SlotState ss = slots[slot];
    const uint64_t t0 = ss.t;
    if (!ss.active) {
        if (lane == 0) {
            ss.t = t0 + n_sweeps;
            slots[slot] = ss;
        }
        return;
    }
    uint32_t *T = reinterpret_cast<uint32_t *>(chain_base + (size_t)warp * G::CHAIN_BYTES);  // [8][B]
    uint32_t *Rw = T + 8 * B;                                                               // [RWN]
    uint8_t *Nc = reinterpret_cast<uint8_t *>(Rw + G::RWN);                                 // [NCB]
    uint8_t *Fb = Nc + G::NCB;                                                              // [NFB]
    const uint64_t lrow = td.w_base + (uint64_t)c * td.B;
    // thresholds, transposed to class-major
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(thr + lrow * 8);
        for (int b = lane; b < B; b += 32) {
            const uint4 a = src[2 * b], q = src[2 * b + 1];
            T[0 * B + b] = a.x; T[1 * B + b] = a.y; T[2 * B + b] = a.z; T[3 * B + b] = a.w;
            T[4 * B + b] = q.x; T[5 * B + b] = q.y; T[6 * B + b] = q.z; T[7 * B + b] = q.w;
        }
    }
    // colour c's sites, their number and the base of its random-word segment
    auto n_of = [&](int colour) -> int { return Coff[colour + 1] - Coff[colour]; };
    auto rb_of = [&](int colour) -> int { return RBo[colour]; };
    // padding of each segment: random words that accept nothing
    for (int colour = 0; colour < NCOL; ++colour) {
        const int n = n_of(colour), pad = ((n + 3) & ~3) - n;
        if (lane < pad) Rw[rb_of(colour) + n + lane] = kAlways;
    }
    const uint32_t bitc = 1u << c;
    int b = ss.b, bmin = ss.b_min;
    int phase = ss.phase, nrt = ss.n_rt;
    int64_t tf = ss.t_first, tl = ss.t_last;
    const int btop = ss.b_top, bbot = count_rt ? ss.b_g : -1;
    bool out_of_range = false;
    __syncwarp();

    // the lane walks of one block: lane l starts at bin mlo - neg + l; returns its end position
    // (bits 0..7, relative to mlo) and its accepted attempts (bits 8..11)
    auto walk = [&](uint32_t w, uint4 r, int mlo, int neg) -> uint32_t {
        const int bin = min(max(mlo + lane, 0), B - 1);
        const uint32_t *tb = T + bin;
        uint32_t X = (uint32_t)(lane - neg);
        const uint32_t rr[kBlk] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int i = 0; i < kBlk; ++i) {
            const int n = (int)((w >> (8 * i)) & 7u);
            const uint32_t M = __ballot_sync(kFull, rr[i] < tb[n * B]);
            X += (__funnelshift_r(M, 0u, X) & 1u) * (uint32_t)(DIM - n + (256 << i));
        }
        return X;
    };

    for (uint64_t s = 0; s < n_sweeps; ++s) {
        const uint32_t tt = (uint32_t)(t0 + s);
        // ---- the sweep's random words: call (4 row, t, rid, (5 + colour) | stream<<8) for each
        //      row and colour, word j to the row's j-th site of that colour; stored by colour
        //      site and clamped to 2^32 - 2 so that "r < threshold" is the whole rule
        for (int q = lane; q < NR * NCOL; q += 32) {
            const int row = q / NCOL, colour = q % NCOL;
            const uint4 w = philox4x32_10(
                make_uint4((uint32_t)(4 * row), tt, ss.rid, (uint32_t)(5 + colour) | (ss.stream << 8)), key);
            const int y = row % L, z = DIM == 3 ? row / L : 0;
            int j = 0;
#pragma unroll
            for (int x = 0; x < L; ++x) {
                if (ccolour_xyz<DIM, L>(x, y, z) == colour) {
                    Rw[RI[row * L + x]] = min(uint4_get(w, j & 3), kAlways - 1u);
                    ++j;
                }
            }
        }
        __syncwarp();
        for (int colour = 0; colour < NCOL; ++colour) {
            const int ncs = n_of(colour), nq = (ncs + 3) & ~3, nblk = nq / kBlk;
            // classes of this colour's sites from the other colours' current spins, a byte per
            // site: class n (bits 0-2), largest descent max(n - dim, 0) (bits 3-4) and ascent
            // max(dim - n, 0) (bits 5-6) in bins; padding: class dim, no move
            auto site_xyz = [&](int k, int &x, int &y, int &z) -> int {
                const int i = CL[Coff[colour] + k];
                x = i % L;
                y = (i / L) % L;
                z = DIM == 3 ? i / (L * L) : 0;
                return i;
            };
            for (int k = lane; k < nq; k += 32) {
                int n = DIM;
                if (k < ncs) {
                    int x, y, z;
                    const int i = site_xyz(k, x, y, z);
                    n = unsat_count<DIM, L>(S, Jw, i, x, y, z, c);
                }
                Nc[k] = (uint8_t)(n | (max(n - DIM, 0) << 3) | (max(DIM - n, 0) << 5));
            }
            __syncwarp();
            const uint32_t *Nw = reinterpret_cast<const uint32_t *>(Nc);
            const uint4 *Rq = reinterpret_cast<const uint4 *>(Rw + rb_of(colour));
            // a block's largest descent (as a negative number of bins) and ascent
            auto descent = [](uint32_t w) { return -(int)__dp4a((w >> 3) & 0x03030303u, 0x01010101u, 0u); };
            auto ascent = [](uint32_t w) { return (int)__dp4a((w >> 5) & 0x03030303u, 0x01010101u, 0u); };
            int lowT = max(bmin - 1, bbot);  // a path at or below this bin may change bmin / round trips

            int bs = b;  // bin at the start of the current block
            uint32_t w_c = Nw[0];
            int neg_c = descent(w_c);
            int lo_c = bs, mlo_c = bs + neg_c;
            uint32_t X_c = walk(w_c, Rq[0], mlo_c, neg_c);
            int hiT = btop - ascent(w_c);  // a block starting at or above this bin may reach the top
#pragma unroll 2
            for (int j = 0; j < nblk; ++j) {
                // the next block's walks, from the lowest bin it can start at
                uint32_t w_n = kDimBytes, X_n = 0u;
                int neg_n = 0, lo_n = 0, mlo_n = 0, hiT_n = btop;
                if (j + 1 < nblk) {
                    w_n = Nw[j + 1];
                    neg_n = descent(w_n);
                    hiT_n = btop - ascent(w_n);
                    lo_n = bs + neg_c;
                    mlo_n = lo_n + neg_n;
                    X_n = walk(w_n, Rq[j + 1], mlo_n, neg_n);
                }
                // this block's outcome: the walk of the lane that starts at the actual bin
                const uint32_t Xs = __shfl_sync(kFull, X_c, bs - lo_c);
                const int be = mlo_c + (int)(Xs & 0xFFu);
                const uint32_t flips = (Xs >> 8) & 0xFu;
                Fb[j] = (uint8_t)(Xs >> 8);  // the same value from every lane
                if (bs >= hiT || bs + neg_c <= lowT) {
                    // near an end of the range: the per-attempt rules, attempt by attempt
                    int p = bs;
                    const int64_t tnow = (int64_t)(t0 + s);
#pragma unroll
                    for (int i = 0; i < kBlk; ++i) {
                        p += (int)((flips >> i) & 1u) * (DIM - (int)((w_c >> (8 * i)) & 7u));
                        bmin = min(bmin, p);
                        out_of_range |= (p < 0) | (p > btop);
                        if (count_rt) {
                            if (phase == 0) {
                                if (p >= btop) { tf = tnow; phase = 1; }
                            } else if (phase == 1) {
                                if (p <= bbot) phase = 2;
                            } else if (p >= btop) {
                                nrt += 1; tl = tnow; phase = 1;
                            }
                        }
                    }
                    lowT = max(bmin - 1, bbot);
                }
                bs = be;
                w_c = w_n; neg_c = neg_n; hiT = hiT_n; lo_c = lo_n; mlo_c = mlo_n; X_c = X_n;
            }
            b = bs;
            __syncwarp();
            // this pass's flips: colour site k was attempt k mod 4 of block k / 4
            for (int k = lane; k < ncs; k += 32) {
                if ((Fb[k >> 2] >> (k & 3)) & 1u) {
                    int x, y, z;
                    atomicXor(&S[site_xyz(k, x, y, z)], bitc);
                }
            }
            __syncwarp();
        }
        if (lane == 0) atomicAdd(&hist[lrow + b], 1u);  // no return value: no wait
    }
    __syncwarp();
    // this chain's spin changes into the global words (other chains of the tile are other bits)
    for (int k = lane; k < V; k += 32) {
        const uint32_t ch = (S[k] ^ S0[k]) & bitc;
        if (ch) atomicXor(&spins[td.spin_off + k], ch);
    }
    if (lane == 0) {
        ss.b = b;
        ss.b_min = bmin;
        ss.phase = phase;
        ss.n_rt = nrt;
        ss.t_first = tf;
        ss.t_last = tl;
        ss.t = t0 + n_sweeps;
        if (count_rt && energy_of_bin(DIM * V, ss.parity, ss.b_min) < ss.e_g) ss.requeue = 1;
        slots[slot] = ss;
        if (diag && out_of_range) atomicOr(diag, 1u);
    }
}

template <int DIM>
__global__ void __launch_bounds__(256, 1)
muca_colour_kernel(const TileDesc *__restrict__ tiles, int n_sub, int C, SlotState *__restrict__ slots,
                   uint32_t *__restrict__ spins, const uint32_t *__restrict__ bonds,
                   const uint32_t *__restrict__ thr, uint32_t *__restrict__ hist, uint64_t n_sweeps, PhiloxKey key,
                   int count_rt, unsigned *__restrict__ diag) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tile = blockIdx.x / n_sub, c0 = (blockIdx.x % n_sub) * C;
    const TileDesc td = tiles[tile];
    if (c0 >= td.width || (td.L & 1) == 0) return;  // the whole CTA, before any barrier (even L: checkerboard kernel)
    const uint64_t n_tile = n_sweeps * (uint64_t)(td.sweep_mul > 0 ? td.sweep_mul : 1);
#define EAMC_CCASE(LL)                                                                                        \
    case LL:                                                                                                  \
        colour_tile<DIM, LL>(td, tile, c0, C, slots, spins, bonds, thr, hist, n_tile, key, count_rt, diag, \
                             smem_raw);                                                                       \
        break;
    switch (td.L) {
        EAMC_CCASE(3) EAMC_CCASE(5) EAMC_CCASE(7) EAMC_CCASE(9) EAMC_CCASE(11)
        default: break;
    }
#undef EAMC_CCASE
}

template <int DIM>
size_t colour_smem_dim(int L, int C) {
    switch (L) {
        case 3: return CGeo<DIM, 3>::smem(C);
        case 5: return CGeo<DIM, 5>::smem(C);
        case 7: return CGeo<DIM, 7>::smem(C);
        case 9: return CGeo<DIM, 9>::smem(C);
        case 11: return CGeo<DIM, 11>::smem(C);
        default: return 0;
    }
}

}  // namespace

size_t colour_smem_bytes(int dim, int L, int C) { return dim == 3 ? colour_smem_dim<3>(L, C) : colour_smem_dim<2>(L, C); }

cudaError_t launch_sweeps_colour(const TileDesc *d_tiles, int n_tiles, int C, int dim, size_t smem, SlotState *d_slots,
                                 uint32_t *d_spins, const uint32_t *d_bonds, const uint32_t *d_thr, uint32_t *d_hist,
                                 uint64_t n_sweeps, PhiloxKey key, int count_rt, unsigned *d_diag, cudaStream_t st) {
    if (n_tiles <= 0 || n_sweeps == 0) return cudaSuccess;
    if (C < 1 || C > 8 || (32 % C) != 0) return cudaErrorInvalidValue;
    static size_t set_limit[4] = {0, 0, 0, 0};
    cudaError_t e;
    if (smem > set_limit[dim]) {
        e = dim == 3 ? cudaFuncSetAttribute(muca_colour_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                     : cudaFuncSetAttribute(muca_colour_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        set_limit[dim] = smem;
    }
    const int n_sub = 32 / C;
    const int grid = n_tiles * n_sub;
    if (dim == 3)
        muca_colour_kernel<3><<<grid, 32 * C, smem, st>>>(d_tiles, n_sub, C, d_slots, d_spins, d_bonds, d_thr, d_hist,
                                                         n_sweeps, key, count_rt, d_diag);
    else
        muca_colour_kernel<2><<<grid, 32 * C, smem, st>>>(d_tiles, n_sub, C, d_slots, d_spins, d_bonds, d_thr, d_hist,
                                                         n_sweeps, key, count_rt, d_diag);
    return cudaGetLastError();
}

}  // namespace eamc
