// eamc_internal.cuh -- device data layout shared by the kernels and the C-ABI layer.
//
// Chains are packed up to 32 to a tile (one warp; the tile's width, 32 by default): bit
// `lane` of every spin / bond word of a tile belongs to the tile's chain `lane`.  All chains
// of a tile have the same dim and L.  Every tile has 32 slots and 32 table rows per array
// whatever its width; the slots beyond the width stay inactive.
//
//   spins  u32[spin_off + i]          site i, bit lane = spin of chain lane is -1
//   bonds  u32[bond_off + i*dim + d]  bond (i, d), bit lane = coupling of chain lane is -1
//   lnW    f64[w_base + lane*B + b]   ln W(b), b = 0..b_top(chain)
//   hist   u32[w_base + lane*B + b]   H(b)
//   thr    u32[(w_base + lane*B + b)*8 + n]  acceptance threshold from bin b, n unsatisfied
//   slots  SlotState[tile*32 + lane]  per-chain scalars
#pragma once
#include <cstdint>

#include "philox.cuh"

namespace eamc {

constexpr uint32_t kAlways = 0xFFFFFFFFu;
constexpr int kTile = 32;
constexpr int kNoBottom = -1;  // b_g when no E_g is known yet: never reached

struct TileDesc {
    int32_t dim, L, V, B;  // B = table rows per chain = largest b_top + 1 for this (dim, L)
    int32_t n_active, sweep_mul;  // sweep_mul: this tile runs n_sweeps * sweep_mul sweeps
    int32_t width, pad;    // chains the tile holds (32, 16 or 8; lanes 0..width-1 of each word)
    uint64_t w_base;       // element offset of lane 0's lnW / hist rows
    uint64_t spin_off;     // word offset of the tile's V spin words
    uint64_t bond_off;     // word offset of the tile's dim*V bond words
};

struct SlotState {
    int32_t b, parity, b_top, b_min;  // current bin, parity of u, top bin, lowest bin seen
    int32_t b_g, e_g;                 // bottom of a round trip (bin, energy)
    int32_t phase, n_rt;              // round-trip state machine
    int64_t t_first, t_last;
    uint64_t t;                       // sweeps done
    uint32_t rid, stream;
    int32_t kind, active;
    int32_t requeue, recursion;       // recursion: 0 plain weight step, 1 Berg's accumulated one
    double alpha, pole, beta;         // ensemble parameters
};

// a9 serving: the job a slot runs, controlled on the device between sweep launches
struct JobCtl {
    uint64_t job;                      // job id (0: none)
    int32_t phase;                     // kJobIdle, kJobIterate, kJobProduce, kJobFinished
    int32_t sweeps_per_tick;           // this job's sweeps per tick (its tile's multiplier x base)
    int32_t ticks, steps_done, iter_steps, ticks_per_step;
    int32_t prod_ticks, max_prod_ticks, requeues, max_requeues;
    int32_t rt_target, pad;
};
constexpr int kJobIdle = 0, kJobIterate = 1, kJobProduce = 2, kJobFinished = 3;
constexpr int kJobDone = 1, kJobCensored = 2, kJobFailed = 3;  // finish status
// per-slot flag of the tick: kFlagUpdate = weight step (then thresholds), kFlagQuantize =
// thresholds only; kFlagResetRt is or'ed in when the round-trip record restarts after the step
constexpr int kFlagUpdate = 1, kFlagQuantize = 2, kFlagResetRt = 4;

// completion record written by the device when a job finishes (one ring slot)
struct SrvRecord {
    uint64_t job;
    int32_t status, slot;
    int32_t n_rt, requeues;
    int64_t t_first, t_last;
    int32_t e_g, e_min;
    uint64_t sweeps;
    uint64_t tick;                     // tick after which the job finished
};

// parameters of one admitted job (host -> device at admission)
struct SrvStart {
    uint64_t job;
    int32_t slot, kind, recursion, iter_steps, ticks_per_step, max_prod_ticks, max_requeues, rt_target;
    int32_t sweeps_per_tick, pad;
    double alpha, pole;
};

__host__ __device__ inline int volume_of(int dim, int L) { return dim == 2 ? L * L : L * L * L; }
__host__ __device__ inline int rows_of(int dim, int L) {
    return ((dim * volume_of(dim, L)) / 2 >> 1) + 1;
}
__host__ __device__ inline int energy_of_bin(int nb, int parity, int b) {
    return 2 * (2 * b + parity) - nb;
}
__host__ __device__ inline int bin_of_energy(int nb, int E) { return ((E + nb) / 2) >> 1; }
__host__ __device__ inline int top_bin(int nb, int parity) {
    const int uhalf = nb / 2;
    const int utop = ((uhalf & 1) == parity) ? uhalf : uhalf - 1;
    return utop >> 1;
}

// kernel launchers (muca_kernels.cu)
cudaError_t launch_init(const TileDesc *d_tiles, int tile0, int n_tiles, int dim,
                        SlotState *d_slots, uint32_t *d_spins, uint32_t *d_bonds,
                        const int8_t *d_J, const int8_t *d_S, int in_row0, PhiloxKey key,
                        int *d_err, cudaStream_t st);
// dynamic shared memory of a sweep block over a tile of this (dim, L, width); 0 if that width
// is not compiled for this size
size_t sweep_smem_bytes(int dim, int L, int width);
bool sweep_width_supported(int dim, int L, int width);
bool sweep_thresholds_in_smem(int dim, int L, int width);
cudaError_t launch_sweeps(const TileDesc *d_tiles, const int32_t *d_tile_list, int n_blocks, int n_work,
                          int *d_queue, int dim, size_t smem, SlotState *d_slots, uint32_t *d_spins,
                          const uint32_t *d_bonds, const uint32_t *d_thr, uint32_t *d_hist, uint64_t n_sweeps,
                          PhiloxKey key, int count_rt, unsigned *d_diag, cudaStream_t st);
int sweep_blocks_per_sm(int dim, size_t smem);
// the colour-order sweep (muca_checker.cu): one lane per chain, every L; widths 32 and (3D) 16 at
// L = 7, 8, 8 at L = 9, 10, 4 at L = 11, 12 (0 bytes: not available)
size_t checker_smem_bytes(int dim, int L, int width);
bool checker_thresholds_in_smem(int dim, int L, int width);
// the kernel-form class of a tile in the colour order: 1 even L, 2 odd L, 4 the narrow tiles of the
// small even sizes (3D, L <= 6), which run in forms of their own
int checker_parity_class(int dim, int L, int width);
cudaError_t launch_sweeps_checker(const TileDesc *d_tiles, int n_tiles, int dim, size_t smem, SlotState *d_slots,
                                  uint32_t *d_spins, const uint32_t *d_bonds, const uint32_t *d_thr,
                                  uint32_t *d_hist, uint64_t n_sweeps, PhiloxKey key, int count_rt,
                                  unsigned *d_diag, cudaStream_t st, int parities);  // bit 0 even L, bit 1 odd L
cudaError_t prepare_sweeps(int dim, size_t smem);  // resident sweep blocks per SM at this smem
cudaError_t launch_quantize(const TileDesc *d_tiles, int n_tiles, const SlotState *d_slots,
                            const double *d_lnW, uint32_t *d_thr, cudaStream_t st);
cudaError_t launch_enforce_walls(const TileDesc *d_tiles, int n_tiles, const SlotState *d_slots,
                                 uint32_t *d_thr, cudaStream_t st);
cudaError_t launch_update_weights(const TileDesc *d_tiles, int n_tiles, SlotState *d_slots,
                                  double *d_lnW, uint32_t *d_hist, double2 *d_acc, cudaStream_t st);
cudaError_t launch_build_ensemble(const TileDesc *d_tiles, int n_tiles, SlotState *d_slots,
                                  const uint8_t *d_sel, int kind, double alpha, double pole,
                                  double beta, double *d_lnW, cudaStream_t st);
cudaError_t launch_reset_lanes(const TileDesc *d_tiles, int dim, SlotState *d_slots, uint32_t *d_spins,
                               uint32_t *d_bonds, double *d_lnW, uint32_t *d_hist, const int32_t *d_slot_of,
                               const uint32_t *d_rids, const uint32_t *d_streams, int n, PhiloxKey key,
                               int *d_err, cudaStream_t st);
cudaError_t launch_update_weights_sel(const TileDesc *d_tiles, SlotState *d_slots, double *d_lnW,
                                      uint32_t *d_hist, double2 *d_acc, const int32_t *d_slot_of, int n,
                                      cudaStream_t st);
cudaError_t launch_reset_rt(const TileDesc *d_tiles, int n_tiles, SlotState *d_slots,
                            const uint8_t *d_sel, cudaStream_t st);
// a9 serving (muca_kernels.cu): per-tick job control, flagged weight steps / quantisation,
// job start and cancellation
cudaError_t launch_srv_control(const TileDesc *d_tiles, int n_slots, SlotState *d_slots, JobCtl *d_ctl,
                               int32_t *d_flag, SrvRecord *d_ring, uint32_t *d_head, uint32_t ring_cap,
                               unsigned long long *d_attempts, uint64_t tick, cudaStream_t st);
cudaError_t launch_srv_update(const TileDesc *d_tiles, int n_slots, SlotState *d_slots, double *d_lnW,
                              uint32_t *d_hist, double2 *d_acc, const int32_t *d_flag, cudaStream_t st);
cudaError_t launch_quantize_flagged(const TileDesc *d_tiles, int n_slots, const SlotState *d_slots,
                                    const double *d_lnW, uint32_t *d_thr, const int32_t *d_flag, cudaStream_t st);
cudaError_t launch_srv_start(const TileDesc *d_tiles, SlotState *d_slots, JobCtl *d_ctl, int32_t *d_flag,
                             double2 *d_acc, const SrvStart *d_start, int n, cudaStream_t st);
cudaError_t launch_srv_cancel(SlotState *d_slots, JobCtl *d_ctl, const int32_t *d_slot_of, int n, cudaStream_t st);

}  // namespace eamc
