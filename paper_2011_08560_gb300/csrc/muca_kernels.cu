// muca_kernels.cu -- sm_103a kernels of the multicanonical (MUCA) hot path.
//
//   init_kernel            a1: disorder, initial spins, energy, descent to E <= E_top
//   muca_sweep_kernel      a2+a3: sequential single-spin-flip generalized Metropolis
//                          (Eq. "muca") with histogram, lowest energy and round trips
//   update_weights_kernel  a4: W <- W P_SH / H (Sec. II iterative procedure), FP64
//   quantize_kernel        a4: ln W -> u32 acceptance thresholds
//   build_ensemble_kernel  a5: flat / power-law / 1/k / canonical weights from ln Omega
//
// One warp = one tile of 32 chains of equal (dim, L).  The lattice of the tile is
// multi-spin coded (bit `lane` of each word is chain `lane`) and staged in shared memory,
// so every spin / bond read is a warp-broadcast LDS; each lane then works on its own chain:
// its own Philox stream, energy bin, threshold row and round-trip state.  MUCA is
// sequential within a chain because W depends on the total energy, so all parallelism
// comes from the chains.
#include <cuda_runtime.h>

#include <cstdint>

#include "eamc_internal.cuh"

namespace eamc {

namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t maj3(uint32_t a, uint32_t b, uint32_t c) {
    return (a & b) | (a & c) | (b & c);
}

// bit-sliced number of set bits among the 2*DIM "unsatisfied" words: p0 + 2 p1 + 4 p2
template <int DIM>
__device__ __forceinline__ void count_unsat(const uint32_t *u, uint32_t &p0, uint32_t &p1,
                                            uint32_t &p2) {
    if constexpr (DIM == 3) {
        const uint32_t s1 = u[0] ^ u[1] ^ u[2], c1 = maj3(u[0], u[1], u[2]);
        const uint32_t s2 = u[3] ^ u[4] ^ u[5], c2 = maj3(u[3], u[4], u[5]);
        p0 = s1 ^ s2;
        const uint32_t c3 = s1 & s2;
        p1 = c1 ^ c2 ^ c3;
        p2 = maj3(c1, c2, c3);
    } else {
        const uint32_t s1 = u[0] ^ u[1] ^ u[2], c1 = maj3(u[0], u[1], u[2]);
        p0 = s1 ^ u[3];
        const uint32_t c2 = s1 & u[3];
        p1 = c1 ^ c2;
        p2 = c1 & c2;
    }
}

__device__ __forceinline__ int lane_count(uint32_t p0, uint32_t p1, uint32_t p2, int lane) {
    return (int)(((p0 >> lane) & 1u) | (((p1 >> lane) & 1u) << 1) | (((p2 >> lane) & 1u) << 2));
}

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
    const int row = in_row0 + blockIdx.x * kTile + lane;  // row in the caller's arrays
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

// ------------------------------------------------------------------------------ a2+a3
// smem: spins (V words, padded to 16 B) then per site a bond record: DIM=3 ->
// [J+x, J+y, J+z, 0, J-x, J-y, J-z, 0], DIM=2 -> [J+x, J+y, J-x, J-y]; J-d is the bond to
// the neighbour at -e_d.  The records duplicate each bond so one site needs two LDS.128.
template <int DIM>
__global__ void __launch_bounds__(32)
muca_sweep_kernel(const TileDesc *__restrict__ tiles, SlotState *__restrict__ slots,
                  uint32_t *__restrict__ spins, const uint32_t *__restrict__ bonds,
                  const uint32_t *__restrict__ thr, uint32_t *__restrict__ hist,
                  uint64_t n_sweeps, PhiloxKey key, int count_rt) {
    constexpr int BW = (DIM == 3) ? 8 : 4;
    extern __shared__ __align__(16) uint32_t smem[];
    const TileDesc td = tiles[blockIdx.x];
    const int lane = threadIdx.x;
    const int L = td.L, V = td.V, LL = L * L;
    uint32_t *sp = smem;
    uint32_t *bd = smem + ((V + 3) & ~3);
    for (int k = lane; k < V; k += 32) sp[k] = spins[td.spin_off + k];
    for (int i = lane; i < V; i += 32) {
        const uint32_t *g = bonds + td.bond_off;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            bd[i * BW + d] = g[i * DIM + d];
            bd[i * BW + BW / 2 + d] = g[nbr<DIM>(i, L, d, -1) * DIM + d];
        }
        if (DIM == 3) { bd[i * BW + 3] = 0u; bd[i * BW + 7] = 0u; }
    }
    __syncwarp();

    const int slot = blockIdx.x * kTile + lane;
    SlotState ss = slots[slot];
    const bool active = ss.active != 0;
    const uint32_t *thr_l = thr + (td.w_base + (uint64_t)lane * td.B) * 8;
    uint32_t *hist_l = hist + td.w_base + (uint64_t)lane * td.B;
    int b = ss.b, bmin = ss.b_min, phase = ss.phase, nrt = ss.n_rt;
    const int btop = ss.b_top, bg = ss.b_g;
    int64_t tf = ss.t_first, tl = ss.t_last;
    const uint64_t t0 = ss.t;
    const uint32_t c2 = ss.rid, c3 = ss.stream << 8;

    for (uint64_t s = 0; s < n_sweeps; ++s) {
        const uint32_t tt = (uint32_t)(t0 + s);
        int x = 0, y = 0, z = 0;
        for (int i0 = 0; i0 < V; i0 += 4) {
            const uint4 r4 = philox4x32_10(make_uint4((uint32_t)(i0 >> 2), tt, c2, c3), key);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int i = i0 + j;
                if (i < V) {
                    const uint32_t r = uint4_get(r4, j);
                    const int xm = (x == 0) ? i + (L - 1) : i - 1;
                    const int xp = (x == L - 1) ? i - (L - 1) : i + 1;
                    const int ym = (y == 0) ? i + (LL - L) : i - L;
                    const int yp = (y == L - 1) ? i - (LL - L) : i + L;
                    const uint32_t si = sp[i];
                    const uint4 bp = *reinterpret_cast<const uint4 *>(bd + i * BW);
                    uint32_t u[2 * DIM];
                    if constexpr (DIM == 3) {
                        const int zm = (z == 0) ? i + (V - LL) : i - LL;
                        const int zp = (z == L - 1) ? i - (V - LL) : i + LL;
                        const uint4 bm = *reinterpret_cast<const uint4 *>(bd + i * BW + 4);
                        u[0] = si ^ sp[xp] ^ bp.x;
                        u[1] = si ^ sp[yp] ^ bp.y;
                        u[2] = si ^ sp[zp] ^ bp.z;
                        u[3] = si ^ sp[xm] ^ bm.x;
                        u[4] = si ^ sp[ym] ^ bm.y;
                        u[5] = si ^ sp[zm] ^ bm.z;
                    } else {
                        u[0] = si ^ sp[xp] ^ bp.x;
                        u[1] = si ^ sp[yp] ^ bp.y;
                        u[2] = si ^ sp[xm] ^ bp.z;
                        u[3] = si ^ sp[ym] ^ bp.w;
                    }
                    uint32_t p0, p1, p2;
                    count_unsat<DIM>(u, p0, p1, p2);
                    const int n = lane_count(p0, p1, p2, lane);
                    const uint32_t th = __ldg(thr_l + b * 8 + n);
                    const bool acc = active && (th == kAlways || r < th);
                    const uint32_t m = __ballot_sync(kFull, acc);
                    sp[i] = si ^ m;
                    if (acc) b += DIM - n;
                    bmin = min(bmin, b);
                    if (count_rt && active) {
                        const bool trig = (phase == 1) ? (b <= bg) : (b >= btop);
                        if (trig) {
                            if (phase == 0) { tf = (int64_t)(t0 + s); phase = 1; }
                            else if (phase == 1) { phase = 2; }
                            else { nrt += 1; tl = (int64_t)(t0 + s); phase = 1; }
                        }
                    }
                }
                if (++x == L) { x = 0; if (++y == L) { y = 0; ++z; } }
            }
        }
        if (active) hist_l[b] += 1u;
    }
    __syncwarp();
    for (int k = lane; k < V; k += 32) spins[td.spin_off + k] = sp[k];
    ss.b = b;
    ss.b_min = bmin;
    ss.phase = phase;
    ss.n_rt = nrt;
    ss.t_first = tf;
    ss.t_last = tl;
    ss.t = t0 + n_sweeps;
    if (count_rt && active && energy_of_bin(td.dim * V, ss.parity, bmin) < ss.e_g) ss.requeue = 1;
    slots[slot] = ss;
}

// ------------------------------------------------------------------------------ a4
__device__ __forceinline__ double ln_profile(int kind, double alpha, double pole, int e_g, int E) {
    if (kind != 1) return 0.0;
    const double Ec = (E < e_g) ? (double)e_g : (double)E;
    return alpha * log(Ec / (pole - (double)e_g) + 1.0);
}

// one block per chain; threads over bins
__global__ void update_weights_kernel(const TileDesc *__restrict__ tiles,
                                      SlotState *__restrict__ slots, double *__restrict__ lnW,
                                      uint32_t *__restrict__ hist) {
    const int slot = blockIdx.x;
    const TileDesc td = tiles[slot / kTile];
    const int lane = slot % kTile;
    SlotState ss = slots[slot];
    if (!ss.active || (ss.kind != 0 && ss.kind != 1)) return;
    const int nb = td.dim * td.V;
    const int e_g = energy_of_bin(nb, ss.parity, ss.b_min);
    double *w = lnW + td.w_base + (uint64_t)lane * td.B;
    uint32_t *h = hist + td.w_base + (uint64_t)lane * td.B;
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

__global__ void quantize_kernel(const TileDesc *__restrict__ tiles,
                                const SlotState *__restrict__ slots,
                                const double *__restrict__ lnW, uint32_t *__restrict__ thr) {
    const int slot = blockIdx.x;
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

static size_t sweep_smem_bytes(int dim, int V) {
    const int bw = dim == 3 ? 8 : 4;
    return (size_t)(((V + 3) & ~3) + bw * V) * sizeof(uint32_t);
}

cudaError_t launch_sweeps(const TileDesc *d_tiles, int n_tiles, int dim, int max_V,
                          SlotState *d_slots, uint32_t *d_spins, const uint32_t *d_bonds,
                          const uint32_t *d_thr, uint32_t *d_hist, uint64_t n_sweeps,
                          PhiloxKey key, int count_rt, cudaStream_t st) {
    if (n_tiles <= 0 || n_sweeps == 0) return cudaSuccess;
    const size_t smem = sweep_smem_bytes(dim, max_V);
    cudaError_t e;
    if (dim == 3) {
        e = cudaFuncSetAttribute(muca_sweep_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        muca_sweep_kernel<3><<<n_tiles, 32, smem, st>>>(d_tiles, d_slots, d_spins, d_bonds, d_thr,
                                                        d_hist, n_sweeps, key, count_rt);
    } else {
        e = cudaFuncSetAttribute(muca_sweep_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        muca_sweep_kernel<2><<<n_tiles, 32, smem, st>>>(d_tiles, d_slots, d_spins, d_bonds, d_thr,
                                                        d_hist, n_sweeps, key, count_rt);
    }
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
                                  double *d_lnW, uint32_t *d_hist, cudaStream_t st) {
    if (n_tiles <= 0) return cudaSuccess;
    update_weights_kernel<<<n_tiles * kTile, 128, 0, st>>>(d_tiles, d_slots, d_lnW, d_hist);
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

cudaError_t launch_reset_rt(const TileDesc *d_tiles, int n_tiles, SlotState *d_slots,
                            const uint8_t *d_sel, cudaStream_t st) {
    if (n_tiles <= 0) return cudaSuccess;
    const int n_slots = n_tiles * kTile;
    reset_rt_kernel<<<(n_slots + 127) / 128, 128, 0, st>>>(d_tiles, n_slots, d_slots, d_sel);
    return cudaGetLastError();
}

}  // namespace eamc
