// eamc_api.cu -- the C ABI declared in include/eamc.h: context, device arenas, and the
// marshalling between caller buffers and the multi-spin-coded device layout.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "eamc.h"
#include "eamc_internal.cuh"
#include "eamc_ctx.cuh"

using namespace eamc;

// ------------------------------------------------------------------------------ errors
static thread_local std::string g_last_error;

int eamc::fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int eamc::cuda_fail(cudaError_t e, const char *what) {
    return fail(EA_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

extern "C" const char *ea_last_error(void) { return g_last_error.c_str(); }

#define EA_CUDA(call)                                          \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);    \
    } while (0)

// ------------------------------------------------------------------------------ helpers
namespace {

template <class T>
int grow(T **ptr, size_t *cap, size_t used, size_t need, cudaStream_t st) {
    if (need <= *cap) return EA_OK;
    size_t ncap = std::max(need, *cap * 2);
    T *np = nullptr;
    if (cudaMalloc(&np, ncap * sizeof(T)) != cudaSuccess)
        return fail(EA_ENOMEM, "device allocation of %zu bytes failed", ncap * sizeof(T));
    cudaMemsetAsync(np, 0, ncap * sizeof(T), st);
    if (*ptr && used) {
        cudaError_t e = cudaMemcpyAsync(np, *ptr, used * sizeof(T), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) { cudaFree(np); return cuda_fail(e, "grow copy"); }
    }
    if (*ptr) {
        cudaStreamSynchronize(st);
        cudaFree(*ptr);
    }
    *ptr = np;
    *cap = ncap;
    return EA_OK;
}

// Threshold tables get kThrPad zero elements before and after the used range: the sweep
// kernel may read (never use) a row one move beyond a chain's table.
constexpr size_t kThrPad = 64;

int grow_thr(ea_ctx *ctx, size_t need) {
    if (need <= ctx->thr_cap) return EA_OK;
    size_t ncap = std::max(need, ctx->thr_cap * 2);
    uint32_t *raw = nullptr;
    if (cudaMalloc(&raw, (ncap + 2 * kThrPad) * sizeof(uint32_t)) != cudaSuccess)
        return fail(EA_ENOMEM, "device allocation of the threshold tables failed");
    cudaMemsetAsync(raw, 0, (ncap + 2 * kThrPad) * sizeof(uint32_t), ctx->stream);
    uint32_t *np = raw + kThrPad;
    if (ctx->d_thr && ctx->w_used) {
        cudaError_t e = cudaMemcpyAsync(np, ctx->d_thr, ctx->w_used * 8 * sizeof(uint32_t),
                                        cudaMemcpyDeviceToDevice, ctx->stream);
        if (e != cudaSuccess) { cudaFree(raw); return cuda_fail(e, "grow copy"); }
    }
    if (ctx->d_thr) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ctx->d_thr - kThrPad);
    }
    ctx->d_thr = np;
    ctx->thr_cap = ncap;
    return EA_OK;
}

// rows of per-chain tables <-> a dense [n][stride] staging array
template <class T>
__global__ void gather_rows(const T *__restrict__ table, const uint64_t *__restrict__ off,
                            const int32_t *__restrict__ len, int n, int stride, int width,
                            T *__restrict__ out) {
    const int c = blockIdx.y;
    if (c >= n) return;
    const uint64_t o = off[c] * width;
    const int l = len[c] * width;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < stride; k += gridDim.x * blockDim.x)
        out[(size_t)c * stride + k] = (k < l) ? table[o + k] : T(0);
}

template <class T>
__global__ void scatter_rows(T *__restrict__ table, const uint64_t *__restrict__ off,
                             const int32_t *__restrict__ len, int n, int stride, int width,
                             const T *__restrict__ in) {
    const int c = blockIdx.y;
    if (c >= n) return;
    const uint64_t o = off[c] * width;
    const int l = len[c] * width;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < l; k += gridDim.x * blockDim.x)
        table[o + k] = in[(size_t)c * stride + k];
}

__global__ void unpack_spins(const TileDesc *__restrict__ tiles, const int32_t *__restrict__ slot_of,
                             int n, int stride, const uint32_t *__restrict__ spins,
                             int8_t *__restrict__ out) {
    const int c = blockIdx.y;
    if (c >= n) return;
    const int slot = slot_of[c];
    const TileDesc td = tiles[slot / kTile];
    const int lane = slot % kTile;
    // the whole row is written: sites beyond this chain's V read as 0
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < stride; i += gridDim.x * blockDim.x)
        out[(size_t)c * stride + i] =
            (i >= td.V) ? int8_t(0) : (((spins[td.spin_off + i] >> lane) & 1u) ? int8_t(-1) : int8_t(1));
}

__global__ void set_eg_kernel(const TileDesc *__restrict__ tiles, SlotState *__restrict__ slots,
                              const int32_t *__restrict__ slot_of, int n,
                              const int32_t *__restrict__ e_g) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int slot = slot_of[c];
    const TileDesc td = tiles[slot / kTile];
    SlotState ss = slots[slot];
    const int nb = td.dim * td.V;
    const int eg = e_g ? e_g[c] : energy_of_bin(nb, ss.parity, ss.b_min);
    ss.e_g = eg;
    // bottom bin: the largest bin whose energy is <= e_g
    int b = bin_of_energy(nb, eg);
    while (b >= 0 && energy_of_bin(nb, ss.parity, b) > eg) --b;
    ss.b_g = b;
    slots[slot] = ss;
}

__global__ void set_params_kernel(SlotState *__restrict__ slots, const int32_t *__restrict__ slot_of,
                                  int n, int kind, double alpha, double pole, double beta) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    SlotState &ss = slots[slot_of[c]];
    ss.kind = kind;
    ss.alpha = alpha;
    ss.pole = pole;
    ss.beta = beta;
}

__global__ void rt_out_kernel(const TileDesc *__restrict__ tiles, const SlotState *__restrict__ slots,
                              const int32_t *__restrict__ slot_of, int n,
                              ea_rt_stats *__restrict__ out, ea_chain_desc *__restrict__ desc) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int slot = slot_of[c];
    const TileDesc td = tiles[slot / kTile];
    const SlotState ss = slots[slot];
    const int nb = td.dim * td.V;
    if (out) {
        ea_rt_stats r;
        r.phase = ss.phase;
        r.n_rt = ss.n_rt;
        r.t_first = ss.t_first;
        r.t_last = ss.t_last;
        r.e_min = energy_of_bin(nb, ss.parity, ss.b_min);
        r.e_g = ss.e_g;
        r.requeue = ss.requeue;
        r.pad = 0;
        out[c] = r;
    }
    if (desc) {
        ea_chain_desc d;
        d.dim = td.dim;
        d.L = td.L;
        d.b_top = ss.b_top;
        d.parity = ss.parity;
        d.rid = ss.rid;
        d.stream = ss.stream;
        d.E = energy_of_bin(nb, ss.parity, ss.b);
        d.kind = ss.kind;
        d.t = ss.t;
        desc[c] = d;
    }
}

}  // namespace

// ------------------------------------------------------------------------------ context
int eamc::ctx_scratch(ea_ctx *ctx, size_t bytes, void **out) {
    if (bytes > ctx->scratch_cap) {
        if (ctx->d_scratch) {
            cudaStreamSynchronize(ctx->stream);
            cudaFree(ctx->d_scratch);
            ctx->d_scratch = nullptr;
            ctx->scratch_cap = 0;
        }
        size_t cap = std::max(bytes, (size_t)1 << 20);
        if (cudaMalloc(&ctx->d_scratch, cap) != cudaSuccess)
            return fail(EA_ENOMEM, "scratch allocation of %zu bytes failed", cap);
        ctx->scratch_cap = cap;
    }
    *out = ctx->d_scratch;
    return EA_OK;
}

int eamc::ctx_check_range(ea_ctx *ctx, int chain0, int n) {
    if (!ctx) return fail(EA_EINVAL, "null context");
    if (n < 0 || chain0 < 0 || chain0 + n > (int)ctx->chain_slot.size())
        return fail(EA_EINVAL, "chain range [%d, %d) outside [0, %zu)", chain0, chain0 + n,
                    ctx->chain_slot.size());
    return EA_OK;
}

// uploads per-chain (slot, row offset, row length) of the range into scratch, returns
// device pointers after `extra` bytes of caller scratch
int eamc::ctx_range_meta(ea_ctx *ctx, int chain0, int n, size_t extra, void **scratch,
                         int32_t **d_slot, uint64_t **d_off, int32_t **d_len) {
    size_t a = (extra + 255) & ~(size_t)255;
    size_t need = a + (size_t)n * (sizeof(int32_t) * 2 + sizeof(uint64_t)) + 512;
    void *base;
    int rc = ctx_scratch(ctx, need, &base);
    if (rc) return rc;
    char *p = (char *)base + a;
    uint64_t *off = (uint64_t *)p;
    int32_t *slot = (int32_t *)(p + (size_t)n * sizeof(uint64_t));
    int32_t *len = slot + n;
    std::vector<uint64_t> h_off(n);
    std::vector<int32_t> h_slot(n), h_len(n);
    for (int k = 0; k < n; ++k) {
        const int c = chain0 + k;
        h_slot[k] = ctx->chain_slot[c];
        h_off[k] = ctx->chain_woff[c];
        h_len[k] = ctx->chain_btop[c] + 1;
    }
    if (n > 0) {
        EA_CUDA(cudaMemcpyAsync(off, h_off.data(), n * sizeof(uint64_t), cudaMemcpyHostToDevice, ctx->stream));
        EA_CUDA(cudaMemcpyAsync(slot, h_slot.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
        EA_CUDA(cudaMemcpyAsync(len, h_len.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
        EA_CUDA(cudaStreamSynchronize(ctx->stream));  // host vectors go out of scope
    }
    *scratch = base;
    *d_slot = slot;
    *d_off = off;
    *d_len = len;
    return EA_OK;
}

int eamc::ctx_refresh_chains(ea_ctx *ctx) {
    // host mirror of b_top per chain (needed for row lengths); read back the slot array
    const size_t ns = ctx->tiles.size() * kTile;
    std::vector<SlotState> h(ns);
    if (ns) {
        EA_CUDA(cudaMemcpyAsync(h.data(), ctx->d_slots, ns * sizeof(SlotState), cudaMemcpyDeviceToHost,
                                ctx->stream));
        EA_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    for (size_t c = 0; c < ctx->chain_slot.size(); ++c) ctx->chain_btop[c] = h[ctx->chain_slot[c]].b_top;
    return EA_OK;
}

// tile ids ordered by decreasing lattice volume (longest tiles first, for the work queue)
void eamc::ctx_drop_graph(ea_ctx *ctx) {
    if (ctx->graph_exec || ctx->graph) cudaStreamSynchronize(ctx->stream);
    if (ctx->graph_exec) { cudaGraphExecDestroy(ctx->graph_exec); ctx->graph_exec = nullptr; }
    if (ctx->graph) { cudaGraphDestroy(ctx->graph); ctx->graph = nullptr; }
    ctx->graph_sweeps = 0;
}

int eamc::ctx_rebuild_order(ea_ctx *ctx) {
    const size_t n = ctx->tiles.size();
    std::vector<int32_t> order(n);
    for (size_t t = 0; t < n; ++t) order[t] = (int32_t)t;
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return ctx->tiles[a].V > ctx->tiles[b].V; });
    if (n > ctx->order_cap) {
        if (ctx->d_order) {
            cudaStreamSynchronize(ctx->stream);
            cudaFree(ctx->d_order);
        }
        ctx->d_order = nullptr;
        if (cudaMalloc(&ctx->d_order, n * sizeof(int32_t)) != cudaSuccess)
            return fail(EA_ENOMEM, "tile order allocation failed");
        ctx->order_cap = n;
    }
    EA_CUDA(cudaMemcpyAsync(ctx->d_order, order.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
    EA_CUDA(cudaStreamSynchronize(ctx->stream));
    return EA_OK;
}

extern "C" int ea_create(ea_ctx **out, int device, void *cuda_stream, uint64_t seed) {
    if (!out) return fail(EA_EINVAL, "null output pointer");
    int ndev = 0;
    EA_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(EA_EINVAL, "device %d outside [0, %d)", device, ndev);
    EA_CUDA(cudaSetDevice(device));
    ea_ctx *ctx = new ea_ctx();
    ctx->device = device;
    ctx->stream = (cudaStream_t)cuda_stream;
    ctx->seed = seed;
    ctx->key = PhiloxKey{(uint32_t)seed, (uint32_t)(seed >> 32)};
    cudaError_t e = cudaMalloc(&ctx->d_err, sizeof(int));
    if (e != cudaSuccess) { delete ctx; return cuda_fail(e, "cudaMalloc"); }
    cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream);
    cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, device);
    // d_queue[0]: work-queue counter of persistent sweeps; d_queue[1]: invariant flags set by
    // the sweep kernel (read and cleared by ea_check)
    if (cudaMalloc(&ctx->d_queue, 2 * sizeof(int)) != cudaSuccess) {
        cudaFree(ctx->d_err);
        delete ctx;
        return fail(EA_ENOMEM, "queue allocation failed");
    }
    cudaMemsetAsync(ctx->d_queue, 0, 2 * sizeof(int), ctx->stream);
    *out = ctx;
    return EA_OK;
}

extern "C" void ea_destroy(ea_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    pt_release(ctx);
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    if (ctx->graph) cudaGraphDestroy(ctx->graph);
    if (ctx->d_order) cudaFree(ctx->d_order);
    if (ctx->d_queue) cudaFree(ctx->d_queue);
    void *ptrs[] = {ctx->d_tiles, ctx->d_slots, ctx->d_spins,   ctx->d_bonds, ctx->d_lnW,
                    ctx->d_hist,  ctx->d_thr ? ctx->d_thr - kThrPad : nullptr,
                    ctx->d_scratch, ctx->d_err, ctx->d_Jin, ctx->d_acc};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete ctx;
}

extern "C" int ea_num_chains(const ea_ctx *ctx) { return ctx ? (int)ctx->chain_slot.size() : 0; }

extern "C" int ea_init_disorder(ea_ctx *ctx, int dim, int L, int n, uint32_t rid0, uint32_t stream,
                                const int8_t *couplings, const int8_t *spins_in, int *first_chain) {
    if (!ctx) return fail(EA_EINVAL, "null context");
    if (dim != 2 && dim != 3) return fail(EA_EINVAL, "dim must be 2 or 3 (got %d)", dim);
    if (L < 3 || L > 12) return fail(EA_EINVAL, "L must be in [3, 12] (got %d)", L);
    if (n <= 0) return fail(EA_EINVAL, "n must be positive (got %d)", n);
    if (stream >= (1u << 24)) return fail(EA_EINVAL, "stream must be < 2^24");
    if (ctx->dim && ctx->dim != dim) return fail(EA_EINVAL, "a context holds a single dim");
    EA_CUDA(cudaSetDevice(ctx->device));
    ctx_drop_graph(ctx);  // the arenas may move and the tile set changes
    int smem_optin = 0;
    EA_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
    // the tile width: the configured one where either sweep kernel has it (8 and 4 only the
    // colour-order kernel), else 32
    const int Wc = ctx->tile_width[L];
    const bool lex_w = sweep_width_supported(dim, L, Wc), col_w = checker_smem_bytes(dim, L, Wc) > 0;
    const int W = (lex_w || col_w) ? Wc : kTile;
    const size_t need = std::max(lex_w || W == kTile ? sweep_smem_bytes(dim, L, W) : 0, checker_smem_bytes(dim, L, W));
    if (need > (size_t)smem_optin)
        return fail(EA_EINVAL, "L=%d needs %zu bytes of shared memory per block, the device allows %d", L, need,
                    smem_optin);
    const int V = volume_of(dim, L), B = rows_of(dim, L);
    const int new_tiles = (n + W - 1) / W;
    const int tile0 = (int)ctx->tiles.size();
    const int chain_first = (int)ctx->chain_slot.size();

    // layout of the new tiles
    std::vector<TileDesc> nt(new_tiles);
    size_t spin_used = ctx->spin_used, bond_used = ctx->bond_used, w_used = ctx->w_used;
    for (int t = 0; t < new_tiles; ++t) {
        TileDesc &td = nt[t];
        td.dim = dim;
        td.L = L;
        td.V = V;
        td.B = B;
        td.n_active = std::min(W, n - t * W);
        td.sweep_mul = 1;
        td.width = W;
        td.pad = 0;
        td.w_base = w_used;
        td.spin_off = spin_used;
        td.bond_off = bond_used;
        spin_used += (size_t)((V + 3) & ~3);
        bond_used += (size_t)((dim * V + 3) & ~3);
        w_used += (size_t)kTile * B;
    }
    const size_t ns_old = ctx->tiles.size() * kTile, ns_new = ns_old + (size_t)new_tiles * kTile;
    int rc;
    if ((rc = grow(&ctx->d_tiles, &ctx->tiles_cap, ctx->tiles.size(), ctx->tiles.size() + new_tiles, ctx->stream)) ||
        (rc = grow(&ctx->d_slots, &ctx->slots_cap, ns_old, ns_new, ctx->stream)) ||
        (rc = grow(&ctx->d_spins, &ctx->spins_cap, ctx->spin_used, spin_used, ctx->stream)) ||
        (rc = grow(&ctx->d_bonds, &ctx->bonds_cap, ctx->bond_used, bond_used, ctx->stream)) ||
        (rc = grow(&ctx->d_lnW, &ctx->lnW_cap, ctx->w_used, w_used, ctx->stream)) ||
        (rc = grow(&ctx->d_hist, &ctx->hist_cap, ctx->w_used, w_used, ctx->stream)) ||
        (rc = grow_thr(ctx, w_used * 8)))
        return rc;
    if (ctx->d_acc && (rc = grow(&ctx->d_acc, &ctx->acc_cap, ctx->w_used, w_used, ctx->stream))) return rc;
    EA_CUDA(cudaMemcpyAsync(ctx->d_tiles + tile0, nt.data(), new_tiles * sizeof(TileDesc),
                            cudaMemcpyHostToDevice, ctx->stream));
    // per-slot identity (rid, stream, defaults)
    std::vector<SlotState> hs((size_t)new_tiles * kTile);
    for (size_t s = 0; s < hs.size(); ++s) {
        SlotState &ss = hs[s];
        std::memset(&ss, 0, sizeof ss);
        // chain index within this group (slots beyond the tile width stay inactive)
        const int k = (int)(s / kTile) * W + std::min((int)(s % kTile), W - 1);
        ss.rid = rid0 + (uint32_t)std::min(k, n - 1);
        ss.stream = stream;
        ss.kind = EA_FLAT;
        ss.alpha = -3.6;
        ss.pole = 96.0;
        ss.beta = 1.0;
    }
    EA_CUDA(cudaMemcpyAsync(ctx->d_slots + ns_old, hs.data(), hs.size() * sizeof(SlotState),
                            cudaMemcpyHostToDevice, ctx->stream));
    // optional caller arrays
    const int8_t *dJ = nullptr, *dS = nullptr;
    void *scratch = nullptr;
    const size_t jbytes = couplings ? (size_t)n * dim * V : 0, sbytes = spins_in ? (size_t)n * V : 0;
    if (jbytes + sbytes) {
        if ((rc = ctx_scratch(ctx, jbytes + sbytes + 256, &scratch))) return rc;
        if (couplings) {
            dJ = (const int8_t *)scratch;
            EA_CUDA(cudaMemcpyAsync((void *)dJ, couplings, jbytes, cudaMemcpyHostToDevice, ctx->stream));
        }
        if (spins_in) {
            dS = (const int8_t *)scratch + ((jbytes + 127) & ~(size_t)127);
            EA_CUDA(cudaMemcpyAsync((void *)dS, spins_in, sbytes, cudaMemcpyHostToDevice, ctx->stream));
        }
    }
    EA_CUDA(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
    EA_CUDA(launch_init(ctx->d_tiles, tile0, new_tiles, dim, ctx->d_slots, ctx->d_spins,
                        ctx->d_bonds, dJ, dS, 0, ctx->key, ctx->d_err, ctx->stream));
    int herr = 0;
    EA_CUDA(cudaMemcpyAsync(&herr, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    EA_CUDA(cudaStreamSynchronize(ctx->stream));
    // commit the new tiles
    ctx->dim = dim;
    for (const TileDesc &td : nt) ctx->tiles.push_back(td);
    ctx->spin_used = spin_used;
    ctx->bond_used = bond_used;
    ctx->w_used = w_used;
    ctx->max_V = std::max(ctx->max_V, V);
    if (sweep_width_supported(dim, L, W)) ctx->sweep_smem = std::max(ctx->sweep_smem, sweep_smem_bytes(dim, L, W));
    for (int k = 0; k < n; ++k) {
        const int slot = (tile0 + k / W) * kTile + k % W;
        ctx->chain_slot.push_back(slot);
        ctx->chain_woff.push_back(nt[k / W].w_base + (uint64_t)(k % W) * B);
        ctx->chain_btop.push_back(0);
    }
    if ((rc = ctx_refresh_chains(ctx))) return rc;
    if ((rc = ctx_rebuild_order(ctx))) return rc;
    // flat weights (ln W = 0 already) -> thresholds
    EA_CUDA(launch_quantize(ctx->d_tiles, (int)ctx->tiles.size(), ctx->d_slots, ctx->d_lnW,
                            ctx->d_thr, ctx->stream));
    if (first_chain) *first_chain = chain_first;
    if (herr) return fail(EA_ESTATE, "descent to E_top got stuck in a local minimum");
    return EA_OK;
}

extern "C" int ea_describe(ea_ctx *ctx, int chain0, int n, ea_chain_desc *out) {
    int rc = ctx_check_range(ctx, chain0, n);
    if (rc) return rc;
    if (!out) return fail(EA_EINVAL, "null output");
    if (n == 0) return EA_OK;
    void *scr;
    int32_t *d_slot, *d_len;
    uint64_t *d_off;
    if ((rc = ctx_range_meta(ctx, chain0, n, (size_t)n * sizeof(ea_chain_desc), &scr, &d_slot, &d_off, &d_len)))
        return rc;
    ea_chain_desc *d_out = (ea_chain_desc *)scr;
    rt_out_kernel<<<(n + 127) / 128, 128, 0, ctx->stream>>>(ctx->d_tiles, ctx->d_slots, d_slot, n,
                                                            nullptr, d_out);
    EA_CUDA(cudaGetLastError());
    EA_CUDA(cudaMemcpyAsync(out, d_out, (size_t)n * sizeof(ea_chain_desc), cudaMemcpyDeviceToHost, ctx->stream));
    EA_CUDA(cudaStreamSynchronize(ctx->stream));
    return EA_OK;
}

extern "C" int muca_set_ensemble(ea_ctx *ctx, int chain0, int n, int kind, double alpha,
                                 double pole_dE, double beta) {
    int rc = ctx_check_range(ctx, chain0, n);
    if (rc) return rc;
    if (kind < EA_FLAT || kind > EA_CANON) return fail(EA_EINVAL, "unknown ensemble kind %d", kind);
    if (kind == EA_POWERLAW && !(pole_dE > 0.0)) return fail(EA_EINVAL, "pole_dE must be > 0");
    if (n == 0) return EA_OK;
    void *scr;
    int32_t *d_slot, *d_len;
    uint64_t *d_off;
    if ((rc = ctx_range_meta(ctx, chain0, n, 0, &scr, &d_slot, &d_off, &d_len))) return rc;
    set_params_kernel<<<(n + 127) / 128, 128, 0, ctx->stream>>>(ctx->d_slots, d_slot, n, kind, alpha,
                                                                pole_dE, beta);
    EA_CUDA(cudaGetLastError());
    EA_CUDA(cudaStreamSynchronize(ctx->stream));
    return EA_OK;
}

__global__ void set_recursion_kernel(SlotState *__restrict__ slots, const int32_t *__restrict__ slot_of,
                                     const uint64_t *__restrict__ off, const int32_t *__restrict__ len, int n,
                                     int mode, double2 *__restrict__ acc) {
    const int c = blockIdx.x;
    if (c >= n) return;
    if (acc)
        for (int b = threadIdx.x; b < len[c]; b += blockDim.x) acc[off[c] + b] = make_double2(0.0, 0.0);
    if (threadIdx.x == 0) slots[slot_of[c]].recursion = mode;
}

extern "C" int muca_set_recursion(ea_ctx *ctx, int chain0, int n, int mode) {
    int rc = ctx_check_range(ctx, chain0, n);
    if (rc) return rc;
    if (mode != EA_REC_PLAIN && mode != EA_REC_BERG) return fail(EA_EINVAL, "unknown recursion %d", mode);
    if (n == 0) return EA_OK;
    if (mode == EA_REC_BERG && !ctx->d_acc) {
        ctx_drop_graph(ctx);  // a captured update would not see the new accumulators
        if ((rc = grow(&ctx->d_acc, &ctx->acc_cap, 0, ctx->w_used, ctx->stream))) return rc;
    }
    void *scr;
    int32_t *d_slot, *d_len;
    uint64_t *d_off;
    if ((rc = ctx_range_meta(ctx, chain0, n, 0, &scr, &d_slot, &d_off, &d_len))) return rc;
    set_recursion_kernel<<<n, 128, 0, ctx->stream>>>(ctx->d_slots, d_slot, d_off, d_len, n, mode, ctx->d_acc);
    EA_CUDA(cudaGetLastError());
    EA_CUDA(cudaStreamSynchronize(ctx->stream));
    return EA_OK;
}

static int max_len(ea_ctx *ctx, int chain0, int n) {
    int m = 0;
    for (int k = 0; k < n; ++k) m = std::max(m, ctx->chain_btop[chain0 + k] + 1);
    return m;
}

template <class T>
static int table_io(ea_ctx *ctx, int chain0, int n, T *table, int width, T *host, int stride,
                    bool to_device) {
    int rc = ctx_check_range(ctx, chain0, n);
    if (rc) return rc;
    if (!host) return fail(EA_EINVAL, "null buffer");
    if (n == 0) return EA_OK;
    if (stride < max_len(ctx, chain0, n) * width)
        return fail(EA_EINVAL, "stride %d shorter than a row (%d)", stride, max_len(ctx, chain0, n) * width);
    const size_t bytes = (size_t)n * stride * sizeof(T);
    void *scr;
    int32_t *d_slot, *d_len;
    uint64_t *d_off;
    if ((rc = ctx_range_meta(ctx, chain0, n, bytes, &scr, &d_slot, &d_off, &d_len))) return rc;
    T *stage = (T *)scr;
    dim3 grid((stride + 255) / 256, n);
    if (to_device) {
        EA_CUDA(cudaMemcpyAsync(stage, host, bytes, cudaMemcpyHostToDevice, ctx->stream));
        scatter_rows<T><<<grid, 256, 0, ctx->stream>>>(table, d_off, d_len, n, stride, width, stage);
        EA_CUDA(cudaGetLastError());
        EA_CUDA(cudaStreamSynchronize(ctx->stream));
    } else {
        gather_rows<T><<<grid, 256, 0, ctx->stream>>>(table, d_off, d_len, n, stride, width, stage);
        EA_CUDA(cudaGetLastError());
        EA_CUDA(cudaMemcpyAsync(host, stage, bytes, cudaMemcpyDeviceToHost, ctx->stream));
        EA_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    return EA_OK;
}

extern "C" int muca_set_weights(ea_ctx *ctx, int chain0, int n, const double *lnW, int stride) {
    int rc = table_io<double>(ctx, chain0, n, ctx ? ctx->d_lnW : nullptr, 1, const_cast<double *>(lnW),
                              stride, true);
    if (rc) return rc;
    EA_CUDA(launch_quantize(ctx->d_tiles, (int)ctx->tiles.size(), ctx->d_slots, ctx->d_lnW, ctx->d_thr,
                            ctx->stream));
    return EA_OK;
}

extern "C" int muca_get_weights(ea_ctx *ctx, int chain0, int n, double *lnW, int stride) {
    return table_io<double>(ctx, chain0, n, ctx ? ctx->d_lnW : nullptr, 1, lnW, stride, false);
}

extern "C" int muca_get_recursion_state(ea_ctx *ctx, int chain0, int n, double *out, int stride) {
    if (ctx && !ctx->d_acc) return fail(EA_ESTATE, "no chain of this context uses the Berg recursion");
    return table_io<double>(ctx, chain0, n, ctx ? (double *)ctx->d_acc : nullptr, 2, out, stride, false);
}

extern "C" int muca_set_thresholds(ea_ctx *ctx, int chain0, int n, const uint32_t *thr, int stride) {
    int rc = table_io<uint32_t>(ctx, chain0, n, ctx ? ctx->d_thr : nullptr, 8, const_cast<uint32_t *>(thr),
                                stride, true);
    if (rc) return rc;
    EA_CUDA(launch_enforce_walls(ctx->d_tiles, (int)ctx->tiles.size(), ctx->d_slots, ctx->d_thr, ctx->stream));
    EA_CUDA(cudaStreamSynchronize(ctx->stream));
    return EA_OK;
}

extern "C" int muca_get_thresholds(ea_ctx *ctx, int chain0, int n, uint32_t *thr, int stride) {
    return table_io<uint32_t>(ctx, chain0, n, ctx ? ctx->d_thr : nullptr, 8, thr, stride, false);
}

extern "C" int get_histograms(ea_ctx *ctx, int chain0, int n, uint32_t *out, int stride, int reset) {
    int rc = table_io<uint32_t>(ctx, chain0, n, ctx ? ctx->d_hist : nullptr, 1, out, stride, false);
    if (rc || !reset || n == 0) return rc;
    // clear the rows of the range: scatter zeros
    const size_t bytes = (size_t)n * stride * sizeof(uint32_t);
    void *scr;
    int32_t *d_slot, *d_len;
    uint64_t *d_off;
    if ((rc = ctx_range_meta(ctx, chain0, n, bytes, &scr, &d_slot, &d_off, &d_len))) return rc;
    EA_CUDA(cudaMemsetAsync(scr, 0, bytes, ctx->stream));
    dim3 grid((stride + 255) / 256, n);
    scatter_rows<uint32_t><<<grid, 256, 0, ctx->stream>>>(ctx->d_hist, d_off, d_len, n, stride, 1,
                                                          (const uint32_t *)scr);
    EA_CUDA(cudaGetLastError());
    EA_CUDA(cudaStreamSynchronize(ctx->stream));
    return EA_OK;
}

extern "C" int muca_set_eg(ea_ctx *ctx, int chain0, int n, const int32_t *e_g) {
    int rc = ctx_check_range(ctx, chain0, n);
    if (rc || n == 0) return rc;
    void *scr;
    int32_t *d_slot, *d_len;
    uint64_t *d_off;
    if ((rc = ctx_range_meta(ctx, chain0, n, (size_t)n * sizeof(int32_t), &scr, &d_slot, &d_off, &d_len)))
        return rc;
    int32_t *d_eg = nullptr;
    if (e_g) {
        d_eg = (int32_t *)scr;
        EA_CUDA(cudaMemcpyAsync(d_eg, e_g, (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
    }
    set_eg_kernel<<<(n + 127) / 128, 128, 0, ctx->stream>>>(ctx->d_tiles, ctx->d_slots, d_slot, n, d_eg);
    EA_CUDA(cudaGetLastError());
    EA_CUDA(cudaStreamSynchronize(ctx->stream));
    return EA_OK;
}

// The colour order runs in the checkerboard kernels (one lane per chain in the tiles of the
// lexicographic kernel; three colour passes for odd L, a kernel of their own); the shared memory
// for the context's tiles and which kernel-form classes occur (bit 0 even, bit 1 odd L, bit 2 the
// small even sizes' narrow tiles).
static int colour_launch(ea_ctx *ctx, size_t *ck_smem_out, int *parities) {
    int optin = 0;
    EA_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
    size_t ck = 0;
    int par = 0;
    for (const TileDesc &td : ctx->tiles) {
        ck = std::max(ck, checker_smem_bytes(td.dim, td.L, td.width));
        par |= checker_parity_class(td.dim, td.L, td.width);
    }
    if (ck > (size_t)optin) return fail(EA_EINVAL, "the colour-order sweep does not fit in shared memory");
    *ck_smem_out = ck;
    *parities = par;
    return EA_OK;
}

// the context's sweeps in its order and launch configuration, queued on its stream (also the
// serving loop's tick in the colour order)
int ctx_enqueue_sweeps(ea_ctx *ctx, uint64_t n_sweeps, int count_roundtrips) {
    const int nt = (int)ctx->tiles.size();
    const uint64_t chunk = ctx->sweeps_per_launch ? ctx->sweeps_per_launch : n_sweeps;
    if (ctx->order == 1) {
        int rc, parities = 0;
        size_t ck_smem = 0;
        if ((rc = colour_launch(ctx, &ck_smem, &parities))) return rc;
        unsigned *diag = reinterpret_cast<unsigned *>(ctx->d_queue + 1);
        for (uint64_t done = 0; done < n_sweeps && ck_smem > 0; done += chunk) {
            const uint64_t now = std::min(chunk, n_sweeps - done);
            EA_CUDA(launch_sweeps_checker(ctx->d_tiles, nt, ctx->dim, ck_smem, ctx->d_slots, ctx->d_spins,
                                          ctx->d_bonds, ctx->d_thr, ctx->d_hist, now, ctx->key, count_roundtrips,
                                          diag, ctx->stream, parities));
        }
        return EA_OK;
    }
    for (const TileDesc &td : ctx->tiles)
        if (!sweep_width_supported(td.dim, td.L, td.width))
            return fail(EA_EINVAL, "tiles of %d chains at L=%d run only in the colour order", td.width, td.L);
    for (uint64_t done = 0; done < n_sweeps; done += chunk) {
        const uint64_t now = std::min(chunk, n_sweeps - done);
        if (ctx->persistent) {
            int per_sm = sweep_blocks_per_sm(ctx->dim, ctx->sweep_smem);
            if (ctx->blocks_per_sm > 0) per_sm = std::min(per_sm, ctx->blocks_per_sm);
            const int grid = std::min(nt, per_sm * std::max(ctx->n_sm, 1));
            EA_CUDA(launch_sweeps(ctx->d_tiles, ctx->d_order, grid, nt, ctx->d_queue, ctx->dim, ctx->sweep_smem,
                                  ctx->d_slots, ctx->d_spins, ctx->d_bonds, ctx->d_thr, ctx->d_hist, now, ctx->key,
                                  count_roundtrips, reinterpret_cast<unsigned *>(ctx->d_queue + 1), ctx->stream));
        } else {
            EA_CUDA(launch_sweeps(ctx->d_tiles, nullptr, nt, nt, nullptr, ctx->dim, ctx->sweep_smem, ctx->d_slots,
                                  ctx->d_spins, ctx->d_bonds, ctx->d_thr, ctx->d_hist, now, ctx->key,
                                  count_roundtrips, reinterpret_cast<unsigned *>(ctx->d_queue + 1), ctx->stream));
        }
    }
    return EA_OK;
}

extern "C" int muca_run_sweeps(ea_ctx *ctx, uint64_t n_sweeps, int count_roundtrips) {
    if (!ctx) return fail(EA_EINVAL, "null context");
    if (ctx->tiles.empty()) return fail(EA_ESTATE, "no chains: call ea_init_disorder first");
    uint64_t mul = 1;
    for (const TileDesc &td : ctx->tiles) mul = std::max<uint64_t>(mul, (uint64_t)td.sweep_mul);
    if (n_sweeps > (1ull << 32) || ctx->max_t_host + n_sweeps * mul > (1ull << 32))
        return fail(EA_EINVAL, "sweep counter would exceed 2^32");
    int rc = ctx_enqueue_sweeps(ctx, n_sweeps, count_roundtrips);
    if (rc) return rc;
    ctx->max_t_host += n_sweeps * mul;
    return EA_OK;
}

extern "C" int muca_set_sweep_multiplier(ea_ctx *ctx, int L, int multiplier) {
    if (!ctx) return fail(EA_EINVAL, "null context");
    if (multiplier < 1 || multiplier > 4096) return fail(EA_EINVAL, "multiplier must be in [1, 4096]");
    bool any = false;
    for (size_t t = 0; t < ctx->tiles.size(); ++t)
        if (ctx->tiles[t].L == L) {
            ctx->tiles[t].sweep_mul = multiplier;
            EA_CUDA(cudaMemcpyAsync(&ctx->d_tiles[t].sweep_mul, &ctx->tiles[t].sweep_mul, sizeof(int32_t),
                                    cudaMemcpyHostToDevice, ctx->stream));
            any = true;
        }
    if (!any) return fail(EA_EINVAL, "no tile of L=%d", L);
    EA_CUDA(cudaStreamSynchronize(ctx->stream));
    return EA_OK;
}

extern "C" int muca_set_sweep_order(ea_ctx *ctx, int order, int chains_per_cta) {
    if (!ctx) return fail(EA_EINVAL, "null context");
    if (order != EA_ORDER_LEX && order != EA_ORDER_COLOUR) return fail(EA_EINVAL, "unknown sweep order %d", order);
    if (chains_per_cta != 0 && (chains_per_cta < 1 || chains_per_cta > 8 || (32 % chains_per_cta) != 0))
        return fail(EA_EINVAL, "chains_per_cta must be 0 or one of 1, 2, 4, 8");
    ctx->order = order;
    (void)chains_per_cta;  // no effect: the colour order runs one lane per chain at every L
    return EA_OK;
}

extern "C" int muca_set_tile_width(ea_ctx *ctx, int L, int width) {
    if (!ctx) return fail(EA_EINVAL, "null context");
    if (L < 3 || L > 12) return fail(EA_EINVAL, "L must be in [3, 12] (got %d)", L);
    const int dim = ctx->dim ? ctx->dim : 3;
    if (!sweep_width_supported(dim, L, width) && checker_smem_bytes(dim, L, width) == 0)
        return fail(EA_EINVAL, "tile width %d is not available for dim=%d, L=%d (32 always; in 3D 16 for "
                               "L=7,8, and in the colour order 8 for L=9,10 and 4 for L=11,12)", width, dim, L);
    ctx->tile_width[L] = width;
    return EA_OK;
}

extern "C" int muca_get_tile_width(int dim, int L, int width, size_t *smem_bytes, int *thresholds_in_smem) {
    if (!sweep_width_supported(dim, L, width)) return fail(EA_EINVAL, "tile width %d unavailable", width);
    if (smem_bytes) *smem_bytes = sweep_smem_bytes(dim, L, width);
    if (thresholds_in_smem) *thresholds_in_smem = sweep_thresholds_in_smem(dim, L, width) ? 1 : 0;
    return EA_OK;
}

extern "C" int muca_get_tile_width_colour(int dim, int L, int width, size_t *smem_bytes, int *thresholds_in_smem) {
    const size_t b = checker_smem_bytes(dim, L, width);
    if (b == 0) return fail(EA_EINVAL, "tile width %d unavailable in the colour order", width);
    if (smem_bytes) *smem_bytes = b;
    if (thresholds_in_smem) *thresholds_in_smem = checker_thresholds_in_smem(dim, L, width) ? 1 : 0;
    return EA_OK;
}

extern "C" int muca_set_launch(ea_ctx *ctx, int persistent, uint64_t sweeps_per_launch, int blocks_per_sm) {
    if (!ctx) return fail(EA_EINVAL, "null context");
    if (blocks_per_sm < 0) return fail(EA_EINVAL, "blocks_per_sm must be >= 0");
    ctx->persistent = persistent ? 1 : 0;
    ctx->sweeps_per_launch = sweeps_per_launch;
    ctx->blocks_per_sm = blocks_per_sm;
    return EA_OK;
}

extern "C" int ea_graph_capture(ea_ctx *ctx, int n_iter, uint64_t sweeps_per_iter, int count_roundtrips,
                                int update_weights) {
    if (!ctx) return fail(EA_EINVAL, "null context");
    if (ctx->tiles.empty()) return fail(EA_ESTATE, "no chains: call ea_init_disorder first");
    if (!ctx->stream) return fail(EA_EINVAL, "graph capture needs a non-default stream");
    if (n_iter <= 0 || sweeps_per_iter == 0) return fail(EA_EINVAL, "empty iteration graph");
    if (ctx->graph_exec) { cudaGraphExecDestroy(ctx->graph_exec); ctx->graph_exec = nullptr; }
    if (ctx->graph) { cudaGraphDestroy(ctx->graph); ctx->graph = nullptr; }
    EA_CUDA(cudaStreamSynchronize(ctx->stream));
    // attributes are set outside the capture (they are not stream work)
    EA_CUDA(prepare_sweeps(ctx->dim, ctx->sweep_smem));
    EA_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    int rc = EA_OK;
    const int nt = (int)ctx->tiles.size();
    for (int it = 0; it < n_iter && rc == EA_OK; ++it) {
        rc = ctx_enqueue_sweeps(ctx, sweeps_per_iter, count_roundtrips);
        if (rc == EA_OK && update_weights) {
            cudaError_t e = launch_update_weights(ctx->d_tiles, nt, ctx->d_slots, ctx->d_lnW, ctx->d_hist, ctx->d_acc, ctx->stream);
            if (e == cudaSuccess) e = launch_quantize(ctx->d_tiles, nt, ctx->d_slots, ctx->d_lnW, ctx->d_thr, ctx->stream);
            if (e != cudaSuccess) rc = cuda_fail(e, "update in capture");
        }
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&ctx->graph_exec, g, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(e, "cudaGraphInstantiate"); }
    ctx->graph = g;
    uint64_t mul = 1;
    for (const TileDesc &td : ctx->tiles) mul = std::max<uint64_t>(mul, (uint64_t)td.sweep_mul);
    ctx->graph_sweeps = (uint64_t)n_iter * sweeps_per_iter * mul;
    return EA_OK;
}

extern "C" int ea_graph_launch(ea_ctx *ctx, int replays) {
    if (!ctx) return fail(EA_EINVAL, "null context");
    if (!ctx->graph_exec) return fail(EA_ESTATE, "no captured graph: call ea_graph_capture first");
    if (replays < 0) return fail(EA_EINVAL, "negative replay count");
    if (ctx->max_t_host + (uint64_t)replays * ctx->graph_sweeps > (1ull << 32))
        return fail(EA_EINVAL, "sweep counter would exceed 2^32");
    for (int r = 0; r < replays; ++r) EA_CUDA(cudaGraphLaunch(ctx->graph_exec, ctx->stream));
    ctx->max_t_host += (uint64_t)replays * ctx->graph_sweeps;
    return EA_OK;
}

extern "C" int ea_graph_release(ea_ctx *ctx) {
    if (!ctx) return fail(EA_EINVAL, "null context");
    EA_CUDA(cudaStreamSynchronize(ctx->stream));
    if (ctx->graph_exec) { cudaGraphExecDestroy(ctx->graph_exec); ctx->graph_exec = nullptr; }
    if (ctx->graph) { cudaGraphDestroy(ctx->graph); ctx->graph = nullptr; }
    ctx->graph_sweeps = 0;
    return EA_OK;
}

extern "C" int muca_update_weights(ea_ctx *ctx) {
    if (!ctx) return fail(EA_EINVAL, "null context");
    if (ctx->tiles.empty()) return fail(EA_ESTATE, "no chains");
    const int nt = (int)ctx->tiles.size();
    EA_CUDA(launch_update_weights(ctx->d_tiles, nt, ctx->d_slots, ctx->d_lnW, ctx->d_hist, ctx->d_acc, ctx->stream));
    EA_CUDA(launch_quantize(ctx->d_tiles, nt, ctx->d_slots, ctx->d_lnW, ctx->d_thr, ctx->stream));
    return EA_OK;
}

static int select_range(ea_ctx *ctx, int chain0, int n, uint8_t **d_sel) {
    const size_t ns = ctx->tiles.size() * kTile;
    std::vector<uint8_t> sel(ns, 0);
    for (int k = 0; k < n; ++k) sel[ctx->chain_slot[chain0 + k]] = 1;
    void *scr;
    int rc = ctx_scratch(ctx, ns + 64, &scr);
    if (rc) return rc;
    EA_CUDA(cudaMemcpyAsync(scr, sel.data(), ns, cudaMemcpyHostToDevice, ctx->stream));
    EA_CUDA(cudaStreamSynchronize(ctx->stream));
    *d_sel = (uint8_t *)scr;
    return EA_OK;
}

extern "C" int muca_build_ensemble(ea_ctx *ctx, int chain0, int n, int kind, double alpha,
                                   double pole_dE, double beta) {
    int rc = ctx_check_range(ctx, chain0, n);
    if (rc || n == 0) return rc;
    if (kind < EA_FLAT || kind > EA_CANON) return fail(EA_EINVAL, "unknown ensemble kind %d", kind);
    uint8_t *d_sel;
    if ((rc = select_range(ctx, chain0, n, &d_sel))) return rc;
    const int nt = (int)ctx->tiles.size();
    EA_CUDA(launch_build_ensemble(ctx->d_tiles, nt, ctx->d_slots, d_sel, kind, alpha, pole_dE, beta,
                                  ctx->d_lnW, ctx->stream));
    EA_CUDA(launch_quantize(ctx->d_tiles, nt, ctx->d_slots, ctx->d_lnW, ctx->d_thr, ctx->stream));
    EA_CUDA(cudaStreamSynchronize(ctx->stream));
    return EA_OK;
}

// chain list -> device slot list (after `extra` bytes of scratch)
static int upload_slots(ea_ctx *ctx, const int32_t *chains, int n, size_t extra, void **scr, int32_t **d_slot) {
    std::vector<int32_t> hs(n);
    for (int k = 0; k < n; ++k) {
        if (chains[k] < 0 || chains[k] >= (int)ctx->chain_slot.size())
            return fail(EA_EINVAL, "chain %d outside [0, %zu)", chains[k], ctx->chain_slot.size());
        hs[k] = ctx->chain_slot[chains[k]];
    }
    const size_t a = (extra + 255) & ~(size_t)255;
    int rc = ctx_scratch(ctx, a + (size_t)n * sizeof(int32_t) + 256, scr);
    if (rc) return rc;
    *d_slot = (int32_t *)((char *)*scr + a);
    EA_CUDA(cudaMemcpyAsync(*d_slot, hs.data(), (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
    return EA_OK;
}

extern "C" int ea_reset_chains(ea_ctx *ctx, const int32_t *chains, int n, const uint32_t *rids,
                               const uint32_t *streams) {
    if (!ctx) return fail(EA_EINVAL, "null context");
    if (n < 0 || (n > 0 && (!chains || !rids || !streams))) return fail(EA_EINVAL, "bad chain list");
    if (n == 0) return EA_OK;
    for (int k = 0; k < n; ++k)
        if (streams[k] >= (1u << 24)) return fail(EA_EINVAL, "stream must be < 2^24");
    void *scr;
    int32_t *d_slot;
    const size_t bytes = (size_t)n * 2 * sizeof(uint32_t);
    int rc = upload_slots(ctx, chains, n, bytes, &scr, &d_slot);
    if (rc) return rc;
    uint32_t *d_rid = (uint32_t *)scr, *d_stream = d_rid + n;
    EA_CUDA(cudaMemcpyAsync(d_rid, rids, n * sizeof(uint32_t), cudaMemcpyHostToDevice, ctx->stream));
    EA_CUDA(cudaMemcpyAsync(d_stream, streams, n * sizeof(uint32_t), cudaMemcpyHostToDevice, ctx->stream));
    EA_CUDA(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
    EA_CUDA(launch_reset_lanes(ctx->d_tiles, ctx->dim, ctx->d_slots, ctx->d_spins, ctx->d_bonds, ctx->d_lnW,
                               ctx->d_hist, d_slot, d_rid, d_stream, n, ctx->key, ctx->d_err, ctx->stream));
    EA_CUDA(launch_quantize(ctx->d_tiles, (int)ctx->tiles.size(), ctx->d_slots, ctx->d_lnW, ctx->d_thr,
                            ctx->stream));
    int herr = 0;
    EA_CUDA(cudaMemcpyAsync(&herr, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    EA_CUDA(cudaStreamSynchronize(ctx->stream));
    if ((rc = ctx_refresh_chains(ctx))) return rc;
    if (herr) return fail(EA_ESTATE, "descent to E_top got stuck for a reset chain (left inactive)");
    return EA_OK;
}

extern "C" int muca_update_weights_subset(ea_ctx *ctx, const int32_t *chains, int n) {
    if (!ctx) return fail(EA_EINVAL, "null context");
    if (n < 0 || (n > 0 && !chains)) return fail(EA_EINVAL, "bad chain list");
    if (n == 0) return EA_OK;
    void *scr;
    int32_t *d_slot;
    int rc = upload_slots(ctx, chains, n, 0, &scr, &d_slot);
    if (rc) return rc;
    EA_CUDA(launch_update_weights_sel(ctx->d_tiles, ctx->d_slots, ctx->d_lnW, ctx->d_hist, ctx->d_acc, d_slot, n, ctx->stream));
    EA_CUDA(launch_quantize(ctx->d_tiles, (int)ctx->tiles.size(), ctx->d_slots, ctx->d_lnW, ctx->d_thr,
                            ctx->stream));
    EA_CUDA(cudaStreamSynchronize(ctx->stream));
    return EA_OK;
}

// dst chain k takes src chain k's ln W row, ensemble (kind and parameters) and E_g
__global__ void copy_weights_kernel(SlotState *__restrict__ slots, double *__restrict__ lnW,
                                    const int32_t *__restrict__ meta, const uint64_t *__restrict__ off, int n) {
    const int k = blockIdx.x;
    if (k >= n) return;
    const int ss_src = meta[4 * k + 0], ss_dst = meta[4 * k + 1], len = meta[4 * k + 2];
    const double *w_src = lnW + off[2 * k + 0];
    double *w_dst = lnW + off[2 * k + 1];
    for (int b = threadIdx.x; b < len; b += blockDim.x) w_dst[b] = w_src[b];
    if (threadIdx.x == 0) {
        const SlotState a = slots[ss_src];
        SlotState &d = slots[ss_dst];
        d.kind = a.kind;
        d.alpha = a.alpha;
        d.pole = a.pole;
        d.beta = a.beta;
        d.e_g = a.e_g;
        d.b_g = a.b_g;
    }
}

extern "C" int muca_copy_weights(ea_ctx *ctx, const int32_t *src, const int32_t *dst, int n) {
    if (!ctx) return fail(EA_EINVAL, "null context");
    if (n < 0 || (n > 0 && (!src || !dst))) return fail(EA_EINVAL, "bad chain lists");
    if (n == 0) return EA_OK;
    const int nc = (int)ctx->chain_slot.size();
    std::vector<int32_t> meta(4 * (size_t)n);
    std::vector<uint64_t> off(2 * (size_t)n);
    std::vector<char> seen(nc, 0);
    for (int k = 0; k < n; ++k) {
        const int a = src[k], b = dst[k];
        if (a < 0 || a >= nc || b < 0 || b >= nc) return fail(EA_EINVAL, "chain index out of range");
        if (seen[b]) return fail(EA_EINVAL, "chain %d is a destination twice", b);
        seen[b] = 1;
        const TileDesc &ta = ctx->tiles[ctx->chain_slot[a] / kTile], &tb = ctx->tiles[ctx->chain_slot[b] / kTile];
        if (ta.L != tb.L || ctx->chain_btop[a] != ctx->chain_btop[b])
            return fail(EA_EINVAL, "chains %d and %d differ in L or in their energy range", a, b);
        meta[4 * k + 0] = ctx->chain_slot[a];
        meta[4 * k + 1] = ctx->chain_slot[b];
        meta[4 * k + 2] = ctx->chain_btop[a] + 1;
        off[2 * k + 0] = ctx->chain_woff[a];
        off[2 * k + 1] = ctx->chain_woff[b];
    }
    for (int k = 0; k < n; ++k)
        if (seen[src[k]]) return fail(EA_EINVAL, "chain %d is both a source and a destination", src[k]);
    void *scr;
    int rc = ctx_scratch(ctx, meta.size() * 4 + off.size() * 8 + 512, &scr);
    if (rc) return rc;
    uint64_t *d_off = (uint64_t *)scr;
    int32_t *d_meta = (int32_t *)((char *)scr + ((off.size() * 8 + 255) & ~(size_t)255));
    EA_CUDA(cudaMemcpyAsync(d_off, off.data(), off.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
    EA_CUDA(cudaMemcpyAsync(d_meta, meta.data(), meta.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    copy_weights_kernel<<<n, 128, 0, ctx->stream>>>(ctx->d_slots, ctx->d_lnW, d_meta, d_off, n);
    EA_CUDA(cudaGetLastError());
    EA_CUDA(launch_quantize(ctx->d_tiles, (int)ctx->tiles.size(), ctx->d_slots, ctx->d_lnW, ctx->d_thr,
                            ctx->stream));
    EA_CUDA(cudaStreamSynchronize(ctx->stream));
    return EA_OK;
}

extern "C" int get_roundtrips(ea_ctx *ctx, int chain0, int n, ea_rt_stats *out, int reset) {
    int rc = ctx_check_range(ctx, chain0, n);
    if (rc || n == 0) return rc;
    if (!out) return fail(EA_EINVAL, "null output");
    void *scr;
    int32_t *d_slot, *d_len;
    uint64_t *d_off;
    if ((rc = ctx_range_meta(ctx, chain0, n, (size_t)n * sizeof(ea_rt_stats), &scr, &d_slot, &d_off, &d_len)))
        return rc;
    ea_rt_stats *d_out = (ea_rt_stats *)scr;
    rt_out_kernel<<<(n + 127) / 128, 128, 0, ctx->stream>>>(ctx->d_tiles, ctx->d_slots, d_slot, n, d_out,
                                                            nullptr);
    EA_CUDA(cudaGetLastError());
    EA_CUDA(cudaMemcpyAsync(out, d_out, (size_t)n * sizeof(ea_rt_stats), cudaMemcpyDeviceToHost, ctx->stream));
    EA_CUDA(cudaStreamSynchronize(ctx->stream));
    if (reset) {
        uint8_t *d_sel;
        if ((rc = select_range(ctx, chain0, n, &d_sel))) return rc;
        EA_CUDA(launch_reset_rt(ctx->d_tiles, (int)ctx->tiles.size(), ctx->d_slots, d_sel, ctx->stream));
        EA_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    return EA_OK;
}

extern "C" int get_state(ea_ctx *ctx, int chain0, int n, int8_t *spins, int stride, int32_t *E,
                         uint64_t *t) {
    int rc = ctx_check_range(ctx, chain0, n);
    if (rc || n == 0) return rc;
    int maxV = 0;
    for (int k = 0; k < n; ++k) {
        const int slot = ctx->chain_slot[chain0 + k];
        maxV = std::max(maxV, ctx->tiles[slot / kTile].V);
    }
    if (spins && stride < maxV) return fail(EA_EINVAL, "spin stride %d < V = %d", stride, maxV);
    const size_t sbytes = spins ? (size_t)n * stride : 0;
    const size_t dbytes = (size_t)n * sizeof(ea_chain_desc);
    void *scr;
    int32_t *d_slot, *d_len;
    uint64_t *d_off;
    if ((rc = ctx_range_meta(ctx, chain0, n, ((sbytes + 255) & ~(size_t)255) + dbytes, &scr, &d_slot, &d_off,
                             &d_len)))
        return rc;
    int8_t *d_sp = (int8_t *)scr;
    ea_chain_desc *d_desc = (ea_chain_desc *)((char *)scr + ((sbytes + 255) & ~(size_t)255));
    if (spins) {
        dim3 grid((stride + 255) / 256, n);
        unpack_spins<<<grid, 256, 0, ctx->stream>>>(ctx->d_tiles, d_slot, n, stride, ctx->d_spins, d_sp);
        EA_CUDA(cudaGetLastError());
        EA_CUDA(cudaMemcpyAsync(spins, d_sp, sbytes, cudaMemcpyDeviceToHost, ctx->stream));
    }
    rt_out_kernel<<<(n + 127) / 128, 128, 0, ctx->stream>>>(ctx->d_tiles, ctx->d_slots, d_slot, n, nullptr,
                                                            d_desc);
    EA_CUDA(cudaGetLastError());
    std::vector<ea_chain_desc> h(n);
    EA_CUDA(cudaMemcpyAsync(h.data(), d_desc, dbytes, cudaMemcpyDeviceToHost, ctx->stream));
    EA_CUDA(cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < n; ++k) {
        if (E) E[k] = h[k].E;
        if (t) t[k] = h[k].t;
    }
    return EA_OK;
}

extern "C" int ea_check(ea_ctx *ctx) {
    if (!ctx) return fail(EA_EINVAL, "null context");
    unsigned flags = 0u;
    EA_CUDA(cudaMemcpyAsync(&flags, ctx->d_queue + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
    EA_CUDA(cudaMemsetAsync(ctx->d_queue + 1, 0, sizeof(unsigned), ctx->stream));
    EA_CUDA(cudaStreamSynchronize(ctx->stream));
    if (flags & 1u) return fail(EA_ESTATE, "a chain left its energy range [0, b_top] during a sweep");
    return EA_OK;
}

extern "C" int ea_synchronize(ea_ctx *ctx) {
    if (!ctx) return fail(EA_EINVAL, "null context");
    EA_CUDA(cudaStreamSynchronize(ctx->stream));
    EA_CUDA(cudaGetLastError());
    return EA_OK;
}

// ------------------------------------------------------------------------------ snapshots
namespace {
constexpr uint64_t kSnapMagic = 0x45414d43534e4150ull;  // "EAMCSNAP"
constexpr uint32_t kSnapVersion = 3;

struct SnapHeader {
    uint64_t magic;
    uint32_t version, dim;
    uint64_t seed, n_tiles, n_chains, spin_used, bond_used, w_used, max_t_host;
    int32_t max_V, has_acc;  // has_acc: the Berg accumulators follow the thresholds
    uint64_t sweep_smem;
};

template <class T>
size_t put_vec(char *dst, const std::vector<T> &v) {
    if (dst) std::memcpy(dst, v.data(), v.size() * sizeof(T));
    return v.size() * sizeof(T);
}
}  // namespace

static size_t snapshot_bytes(const ea_ctx *ctx) {
    const size_t nt = ctx->tiles.size(), nc = ctx->chain_slot.size();
    return sizeof(SnapHeader) + nt * sizeof(TileDesc) + nc * (sizeof(int32_t) * 2 + sizeof(uint64_t)) +
           nt * kTile * sizeof(SlotState) + (ctx->spin_used + ctx->bond_used) * sizeof(uint32_t) +
           ctx->w_used * (sizeof(double) + sizeof(uint32_t) + 8 * sizeof(uint32_t)) +
           (ctx->d_acc ? ctx->w_used * sizeof(double2) : 0);
}

extern "C" int ea_snapshot_size(ea_ctx *ctx, size_t *bytes) {
    if (!ctx || !bytes) return fail(EA_EINVAL, "null argument");
    *bytes = snapshot_bytes(ctx);
    return EA_OK;
}

extern "C" int ea_snapshot_save(ea_ctx *ctx, void *buf, size_t cap) {
    if (!ctx || !buf) return fail(EA_EINVAL, "null argument");
    const size_t need = snapshot_bytes(ctx);
    if (cap < need) return fail(EA_EINVAL, "snapshot needs %zu bytes, buffer has %zu", need, cap);
    EA_CUDA(cudaStreamSynchronize(ctx->stream));
    char *p = (char *)buf;
    SnapHeader h;
    std::memset(&h, 0, sizeof h);
    h.magic = kSnapMagic;
    h.version = kSnapVersion;
    h.dim = (uint32_t)ctx->dim;
    h.seed = ctx->seed;
    h.n_tiles = ctx->tiles.size();
    h.n_chains = ctx->chain_slot.size();
    h.spin_used = ctx->spin_used;
    h.bond_used = ctx->bond_used;
    h.w_used = ctx->w_used;
    h.max_t_host = ctx->max_t_host;
    h.max_V = ctx->max_V;
    h.has_acc = ctx->d_acc ? 1 : 0;
    h.sweep_smem = ctx->sweep_smem;
    std::memcpy(p, &h, sizeof h);
    p += sizeof h;
    p += put_vec(p, ctx->tiles);  // host mirror (sweep multipliers included)
    p += put_vec(p, ctx->chain_slot);
    p += put_vec(p, ctx->chain_woff);
    p += put_vec(p, ctx->chain_btop);
    auto dev = [&](const void *src, size_t bytes) -> int {
        if (bytes) EA_CUDA(cudaMemcpy(p, src, bytes, cudaMemcpyDeviceToHost));
        p += bytes;
        return EA_OK;
    };
    int rc;
    if ((rc = dev(ctx->d_slots, h.n_tiles * kTile * sizeof(SlotState))) ||
        (rc = dev(ctx->d_spins, h.spin_used * 4)) || (rc = dev(ctx->d_bonds, h.bond_used * 4)) ||
        (rc = dev(ctx->d_lnW, h.w_used * 8)) || (rc = dev(ctx->d_hist, h.w_used * 4)) ||
        (rc = dev(ctx->d_thr, h.w_used * 8 * 4)) || (h.has_acc && (rc = dev(ctx->d_acc, h.w_used * 16))))
        return rc;
    return EA_OK;
}

extern "C" int ea_snapshot_load(ea_ctx *ctx, const void *buf, size_t size) {
    if (!ctx || !buf) return fail(EA_EINVAL, "null argument");
    if (!ctx->tiles.empty()) return fail(EA_ESTATE, "a snapshot loads into a context without chains");
    ctx_drop_graph(ctx);
    if (size < sizeof(SnapHeader)) return fail(EA_EINVAL, "snapshot too short");
    SnapHeader h;
    std::memcpy(&h, buf, sizeof h);
    if (h.magic != kSnapMagic || h.version != kSnapVersion) return fail(EA_EINVAL, "not an eamc snapshot");
    const char *p = (const char *)buf + sizeof h;
    std::vector<TileDesc> tiles(h.n_tiles);
    std::vector<int32_t> cslot(h.n_chains), cbtop(h.n_chains);
    std::vector<uint64_t> cwoff(h.n_chains);
    const size_t need = sizeof h + h.n_tiles * sizeof(TileDesc) + h.n_chains * 16 + h.n_tiles * kTile * sizeof(SlotState) +
                        (h.spin_used + h.bond_used) * 4 + h.w_used * (8 + 4 + 32) + (h.has_acc ? h.w_used * 16 : 0);
    if (size < need) return fail(EA_EINVAL, "snapshot truncated (%zu of %zu bytes)", size, need);
    std::memcpy(tiles.data(), p, h.n_tiles * sizeof(TileDesc)); p += h.n_tiles * sizeof(TileDesc);
    std::memcpy(cslot.data(), p, h.n_chains * 4); p += h.n_chains * 4;
    std::memcpy(cwoff.data(), p, h.n_chains * 8); p += h.n_chains * 8;
    std::memcpy(cbtop.data(), p, h.n_chains * 4); p += h.n_chains * 4;
    int rc;
    if ((rc = grow(&ctx->d_tiles, &ctx->tiles_cap, 0, h.n_tiles, ctx->stream)) ||
        (rc = grow(&ctx->d_slots, &ctx->slots_cap, 0, h.n_tiles * kTile, ctx->stream)) ||
        (rc = grow(&ctx->d_spins, &ctx->spins_cap, 0, h.spin_used, ctx->stream)) ||
        (rc = grow(&ctx->d_bonds, &ctx->bonds_cap, 0, h.bond_used, ctx->stream)) ||
        (rc = grow(&ctx->d_lnW, &ctx->lnW_cap, 0, h.w_used, ctx->stream)) ||
        (rc = grow(&ctx->d_hist, &ctx->hist_cap, 0, h.w_used, ctx->stream)) ||
        (rc = grow_thr(ctx, h.w_used * 8)) ||
        (h.has_acc && (rc = grow(&ctx->d_acc, &ctx->acc_cap, 0, h.w_used, ctx->stream))))
        return rc;
    EA_CUDA(cudaStreamSynchronize(ctx->stream));
    auto dev = [&](void *dst, size_t bytes) -> int {
        if (bytes) EA_CUDA(cudaMemcpy(dst, p, bytes, cudaMemcpyHostToDevice));
        p += bytes;
        return EA_OK;
    };
    EA_CUDA(cudaMemcpy(ctx->d_tiles, tiles.data(), h.n_tiles * sizeof(TileDesc), cudaMemcpyHostToDevice));
    if ((rc = dev(ctx->d_slots, h.n_tiles * kTile * sizeof(SlotState))) || (rc = dev(ctx->d_spins, h.spin_used * 4)) ||
        (rc = dev(ctx->d_bonds, h.bond_used * 4)) || (rc = dev(ctx->d_lnW, h.w_used * 8)) ||
        (rc = dev(ctx->d_hist, h.w_used * 4)) || (rc = dev(ctx->d_thr, h.w_used * 8 * 4)) ||
        (h.has_acc && (rc = dev(ctx->d_acc, h.w_used * 16))))
        return rc;
    ctx->dim = (int)h.dim;
    ctx->seed = h.seed;
    ctx->key = PhiloxKey{(uint32_t)h.seed, (uint32_t)(h.seed >> 32)};
    ctx->tiles = tiles;
    ctx->chain_slot = cslot;
    ctx->chain_woff = cwoff;
    ctx->chain_btop = cbtop;
    ctx->spin_used = h.spin_used;
    ctx->bond_used = h.bond_used;
    ctx->w_used = h.w_used;
    ctx->max_t_host = h.max_t_host;
    ctx->max_V = h.max_V;
    ctx->sweep_smem = h.sweep_smem;
    return ctx_rebuild_order(ctx);
}
