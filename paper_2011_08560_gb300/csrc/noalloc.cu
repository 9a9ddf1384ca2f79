// noalloc.cu -- muca_run_sweeps_noalloc: the MUCA sweep path for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside another framework's memory pool
// or under a strict device-memory budget, plugins that may only touch buffers handed to them,
// and hosts that forbid allocation after start-up.  They hand over their own device buffers
// for inputs and outputs; everything else this path needs (the multi-spin-coded lattices,
// per-chain state, tile descriptors and a padded copy of the threshold tables) lives in one
// file-scope __device__ array of kScratchBytes.  Every GPU that loads the library holds that
// array until the process exits.
//
// Host code may not use the array's name as a device address (on the host it is only a
// stand-in symbol): its address is obtained once per device with cudaGetSymbolAddress while
// that device is current, at the first call on the device, and passed to the kernels.  That
// first call should therefore happen before any stream capture.  All calls share the array
// and it keeps the last call's contents: everything a call relies on is rewritten by that
// call, and calls that overlap on the GPU (other streams, other host threads) race on it.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstring>

#include "eamc.h"
#include "eamc_ctx.cuh"
#include "eamc_internal.cuh"

using namespace eamc;

namespace {

constexpr size_t kScratchBytes = (size_t)4 << 20;  // 4 MiB
constexpr int kMaxChains = 256;                    // 8 tiles of 32 chains
constexpr int kMaxDevices = 64;
constexpr size_t kPad = 64;                        // threshold elements before / after (zero)

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];
// device address of g_scratch per device, resolved at the first call on that device; atomic
// because calls may come from several host threads (they all store the same value)
std::atomic<unsigned char *> g_scratch_dev[kMaxDevices];

struct Layout {
    size_t tiles, slots, spins, bonds, thr, err, end;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

Layout layout_for(int dim, int L, int n_tiles) {
    const int V = volume_of(dim, L), B = rows_of(dim, L);
    Layout l;
    size_t off = 0;
    l.tiles = off; off = align256(off + (size_t)n_tiles * sizeof(TileDesc));
    l.slots = off; off = align256(off + (size_t)n_tiles * kTile * sizeof(SlotState));
    l.spins = off; off = align256(off + (size_t)n_tiles * ((V + 3) & ~3) * 4);
    l.bonds = off; off = align256(off + (size_t)n_tiles * ((dim * V + 3) & ~3) * 4);
    l.thr = off; off = align256(off + ((size_t)n_tiles * kTile * B * 8 + 2 * kPad) * 4);
    l.err = off; off = align256(off + sizeof(int));
    l.end = off;
    return l;
}

// neighbour of site i along d with sign
template <int DIM>
__device__ __forceinline__ int nb_site(int i, int L, int d, int sign) {
    int c[3] = {i % L, (i / L) % L, DIM == 3 ? i / (L * L) : 0};
    c[d] = (c[d] + sign + L) % L;
    return c[0] + L * c[1] + L * L * c[2];
}

// one warp per tile: caller's +-1 arrays -> multi-spin-coded words, tile descriptor and chain
// states (energy from the spins, parity from the couplings), padded copy of the thresholds
template <int DIM>
__global__ void pack_kernel(int L, int n, const uint32_t *__restrict__ rid, const uint32_t *__restrict__ stream,
                            const int8_t *__restrict__ J, const int8_t *__restrict__ S,
                            const uint32_t *__restrict__ thr_in, uint64_t t0, TileDesc *tiles, SlotState *slots,
                            uint32_t *spins, uint32_t *bonds, uint32_t *thr, int *err) {
    const int tile = blockIdx.x, lane = threadIdx.x, c = tile * kTile + lane;
    const bool active = c < n;
    const int V = volume_of(DIM, L), nb = DIM * V, B = rows_of(DIM, L);
    const uint64_t spin_off = (uint64_t)tile * ((V + 3) & ~3), bond_off = (uint64_t)tile * ((nb + 3) & ~3);
    if (lane == 0) {
        TileDesc td;
        td.dim = DIM;
        td.L = L;
        td.V = V;
        td.B = B;
        td.n_active = min(kTile, n - tile * kTile);
        td.sweep_mul = 1;
        td.width = kTile;
        td.pad = 0;
        td.w_base = (uint64_t)tile * kTile * B;
        td.spin_off = spin_off;
        td.bond_off = bond_off;
        tiles[tile] = td;
    }
    uint32_t *sp = spins + spin_off, *bd = bonds + bond_off;
    int negatives = 0;
    for (int j = 0; j < nb; ++j) {
        const bool neg = active && J[(size_t)c * nb + j] < 0;
        negatives += neg;
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, neg);
        if (lane == 0) bd[j] = m;
    }
    for (int i = 0; i < V; ++i) {
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, active && S[(size_t)c * V + i] < 0);
        if (lane == 0) sp[i] = m;
    }
    __syncwarp();
    int u = 0;
    for (int i = 0; i < V; ++i)
        for (int d = 0; d < DIM; ++d)
            u += (int)(((sp[i] ^ sp[nb_site<DIM>(i, L, d, +1)] ^ bd[i * DIM + d]) >> lane) & 1u);
    const int E = 2 * u - nb, parity = negatives & 1;
    const int btop = top_bin(nb, parity);
    const bool inside = E <= energy_of_bin(nb, parity, btop);
    if (active && !inside) atomicExch(err, 1);
    SlotState ss;
    memset(&ss, 0, sizeof ss);
    ss.parity = parity;
    ss.b_top = active ? btop : 0;
    ss.b = (active && inside) ? bin_of_energy(nb, E) : 0;
    ss.b_min = ss.b;
    ss.b_g = kNoBottom;
    ss.e_g = -(1 << 30);
    ss.t_first = -1;
    ss.t_last = -1;
    ss.t = t0;
    ss.rid = active ? rid[c] : 0u;
    ss.stream = active ? stream[c] : 0u;
    ss.active = (active && inside) ? 1 : 0;
    slots[c] = ss;
    // thresholds: this chain's [B][8] rows (zeros for padding lanes)
    uint32_t *dst = thr + kPad + (size_t)c * B * 8;
    for (int k = 0; k < B * 8; ++k) dst[k] = active ? thr_in[(size_t)c * B * 8 + k] : 0u;
}

__global__ void zero_pads(uint32_t *thr, size_t n_elems) {
    const int k = threadIdx.x;
    if (k < (int)kPad) {
        thr[k] = 0u;
        thr[kPad + n_elems + k] = 0u;
    }
}

template <int DIM>
__global__ void unpack_kernel(int L, int n, const SlotState *slots, const uint32_t *spins, int8_t *S, int32_t *E) {
    const int c = blockIdx.x, tile = c / kTile, lane = c % kTile;
    const int V = volume_of(DIM, L), nb = DIM * V;
    const uint32_t *sp = spins + (uint64_t)tile * ((V + 3) & ~3);
    for (int i = threadIdx.x; i < V; i += blockDim.x) S[(size_t)c * V + i] = ((sp[i] >> lane) & 1u) ? -1 : 1;
    if (threadIdx.x == 0) {
        const SlotState ss = slots[c];
        E[c] = energy_of_bin(nb, ss.parity, ss.b);
    }
}

#define NA_CUDA(call)                                        \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
    } while (0)

}  // namespace

extern "C" int muca_run_sweeps_noalloc(int dim, int L, int n, uint64_t seed, const uint32_t *rid,
                                       const uint32_t *stream_id, const int8_t *couplings, int8_t *spins,
                                       int32_t *energies, const uint32_t *thr, uint32_t *hist, uint64_t t0,
                                       uint64_t n_sweeps, void *cuda_stream) {
    if (dim != 2 && dim != 3) return fail(EA_EINVAL, "dim must be 2 or 3");
    if (L < 3 || L > 12) return fail(EA_EINVAL, "L must be in [3, 12]");
    if (n <= 0 || n > kMaxChains) return fail(EA_EINVAL, "n must be in [1, %d] for the no-allocation path", kMaxChains);
    const int n_tiles = (n + kTile - 1) / kTile;
    const Layout lay = layout_for(dim, L, n_tiles);
    if (lay.end > kScratchBytes)
        return fail(EA_EINVAL, "%d chains of L=%d need %zu bytes of scratch, the static array holds %zu", n, L,
                    lay.end, kScratchBytes);
    if (!rid || !stream_id || !couplings || !spins || !energies || !thr || !hist)
        return fail(EA_EINVAL, "null buffer");
    if (t0 > (1ull << 32) || n_sweeps > (1ull << 32) - t0)
        return fail(EA_EINVAL, "sweep counter would exceed 2^32");
    const size_t smem = sweep_smem_bytes(dim, L, kTile);
    int dev = 0;
    NA_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(EA_EINVAL, "device %d out of range", dev);
    unsigned char *base = g_scratch_dev[dev].load(std::memory_order_acquire);
    if (!base) {  // first call on this device: resolve the array's device address
        void *p = nullptr;
        NA_CUDA(cudaGetSymbolAddress(&p, g_scratch));
        base = (unsigned char *)p;
        g_scratch_dev[dev].store(base, std::memory_order_release);
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    TileDesc *tiles = (TileDesc *)(base + lay.tiles);
    SlotState *slots = (SlotState *)(base + lay.slots);
    uint32_t *d_spins = (uint32_t *)(base + lay.spins), *d_bonds = (uint32_t *)(base + lay.bonds);
    uint32_t *d_thr = (uint32_t *)(base + lay.thr);
    int *d_err = (int *)(base + lay.err);
    const size_t thr_elems = (size_t)n_tiles * kTile * rows_of(dim, L) * 8;
    PhiloxKey key{(uint32_t)seed, (uint32_t)(seed >> 32)};
    NA_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), st));
    zero_pads<<<1, (int)kPad, 0, st>>>(d_thr, thr_elems);
    if (dim == 3)
        pack_kernel<3><<<n_tiles, kTile, 0, st>>>(L, n, rid, stream_id, couplings, spins, thr, t0, tiles, slots,
                                                  d_spins, d_bonds, d_thr, d_err);
    else
        pack_kernel<2><<<n_tiles, kTile, 0, st>>>(L, n, rid, stream_id, couplings, spins, thr, t0, tiles, slots,
                                                  d_spins, d_bonds, d_thr, d_err);
    NA_CUDA(cudaGetLastError());
    // a chain outside its range refuses the whole call before any sweep: no output buffer is
    // written, so a caller may fix the input and call again with the same t0
    int herr = 0;
    NA_CUDA(cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    NA_CUDA(cudaStreamSynchronize(st));
    if (herr)
        return fail(EA_EINVAL, "a chain starts above E_top (outside the MUCA range); nothing was run and no "
                               "output was written");
    // the caller's tables get the same walls as tables injected into a context
    // (muca_set_thresholds): moves out of [0, b_top] are rejected whatever the caller wrote
    NA_CUDA(launch_enforce_walls(tiles, n_tiles, slots, d_thr + kPad, st));
    NA_CUDA(launch_sweeps(tiles, nullptr, n_tiles, n_tiles, nullptr, dim, smem, slots, d_spins, d_bonds,
                          d_thr + kPad, hist, n_sweeps, key, 0, nullptr, st));
    if (dim == 3)
        unpack_kernel<3><<<n, 128, 0, st>>>(L, n, slots, d_spins, spins, energies);
    else
        unpack_kernel<2><<<n, 128, 0, st>>>(L, n, slots, d_spins, spins, energies);
    NA_CUDA(cudaGetLastError());
    NA_CUDA(cudaStreamSynchronize(st));
    return EA_OK;
}
