// eamc_ctx.cuh -- the opaque ea_ctx behind the C ABI (host side).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "eamc_internal.cuh"

struct PtState;  // parallel tempering state (pt_kernels.cu)

struct ea_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    uint64_t seed = 0;
    eamc::PhiloxKey key{0, 0};
    int dim = 0;
    int max_V = 0;
    size_t sweep_smem = 0;    // dynamic shared memory of the sweep launch (largest tile)
    uint64_t max_t_host = 0;  // upper bound of every chain's sweep counter

    // host mirrors
    std::vector<eamc::TileDesc> tiles;
    std::vector<int32_t> chain_slot;   // chain -> tile*32 + lane
    std::vector<uint64_t> chain_woff;  // chain -> row offset of lnW / hist (thr: x8)
    std::vector<int32_t> chain_btop;   // chain -> b_top

    // device arenas (library-owned)
    eamc::TileDesc *d_tiles = nullptr;
    eamc::SlotState *d_slots = nullptr;
    uint32_t *d_spins = nullptr, *d_bonds = nullptr, *d_hist = nullptr, *d_thr = nullptr;
    double *d_lnW = nullptr;
    size_t tiles_cap = 0, slots_cap = 0, spins_cap = 0, bonds_cap = 0, lnW_cap = 0, hist_cap = 0,
           thr_cap = 0;
    size_t spin_used = 0, bond_used = 0, w_used = 0;
    double2 *d_acc = nullptr;         // f1: Berg accumulators {D, G} per bin (allocated on first use)
    size_t acc_cap = 0;

    // staging / scratch for marshalling (grown on demand)
    void *d_scratch = nullptr;
    size_t scratch_cap = 0;
    int *d_err = nullptr;
    int8_t *d_Jin = nullptr;

    // a8: launch configuration of the sweep kernel and the captured iteration graph
    int persistent = 0;               // 1: resident grid pulling tiles from a queue
    uint64_t sweeps_per_launch = 0;   // 0: all requested sweeps in one launch
    int blocks_per_sm = 0;            // persistent grid: resident blocks per SM (0: occupancy limit)
    int tile_width[13] = {32, 32, 32, 32, 32, 32, 32, 32, 32, 32, 32, 32, 32};  // chains per tile by L
    int order = 0;                    // sweep order: 0 lexicographic, 1 colour class by colour class
    int n_sm = 0;
    int32_t *d_order = nullptr;       // tile ids, longest tiles first
    size_t order_cap = 0;
    int *d_queue = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    uint64_t graph_sweeps = 0;        // sweeps one replay adds to every chain

    PtState *pt = nullptr;
};

namespace eamc {
int fail(int code, const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);
int ctx_scratch(ea_ctx *ctx, size_t bytes, void **out);
int ctx_check_range(ea_ctx *ctx, int chain0, int n);
int ctx_range_meta(ea_ctx *ctx, int chain0, int n, size_t extra, void **scratch, int32_t **d_slot,
                   uint64_t **d_off, int32_t **d_len);
int ctx_refresh_chains(ea_ctx *ctx);
int ctx_rebuild_order(ea_ctx *ctx);
void ctx_drop_graph(ea_ctx *ctx);
}  // namespace eamc
int ctx_enqueue_sweeps(ea_ctx *ctx, uint64_t n_sweeps, int count_roundtrips);

void pt_release(ea_ctx *ctx);
