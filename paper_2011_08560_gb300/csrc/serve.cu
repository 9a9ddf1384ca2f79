// serve.cu -- a9: the serving loop behind ea_srv_* (continuous batching of realization jobs).
//
// A job is one disorder realization simulated with a MUCA ensemble (Sec. II): a number of
// weight-iteration steps, then production until it has completed its target number of round
// trips (Sec. III), with the paper's requeue when a lower energy turns up.  All state stays on
// the device in one context whose tiles act as a pool of lanes per lattice size; one tick is
//   sweep launch over every tile -> job control (one thread per slot: tick counts, weight-step
//   and phase decisions, requeue, completion records) -> weight steps of the flagged slots ->
//   thresholds of the flagged slots,
// all queued on the server's stream with no host synchronisation.  The host side only
//   * admits waiting jobs into free lanes (reset of the lane in place + job start, from a
//     pinned staging buffer), growing the pool of an L while the memory budget allows;
//   * starts, every poll_ticks ticks, an asynchronous copy of the completion ring into one of
//     two pinned buffers and reads the previous one once its event has completed;
//   * keeps at most max_ahead ticks queued beyond the last completed read-back.
// A job's schedule is counted in its own ticks and its random numbers are keyed by its own
// sweep counter, so its result does not depend on the jobs it shares the device with.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <unordered_map>
#include <vector>

#include "eamc.h"
#include "eamc_ctx.cuh"
#include "eamc_internal.cuh"

using namespace eamc;

namespace {

constexpr uint32_t kRingCap = 1u << 14;
constexpr int kStageBufs = 4;
constexpr int kMaxStage = 4096;  // jobs admitted per staging buffer

struct HostJob {
    uint64_t id;
    ea_job job;
    int32_t slot = -1;
    double t_submit = 0, t_admit = 0;
};

struct StageBuf {
    SrvStart *start = nullptr;   // pinned
    int32_t *slots = nullptr;    // pinned
    uint32_t *rids = nullptr, *streams = nullptr;
    cudaEvent_t done = nullptr;
    bool used = false;
};

struct ReadBack {
    SrvRecord *ring = nullptr;   // pinned copy of the device ring
    uint32_t *head = nullptr;    // pinned
    unsigned long long *attempts = nullptr;
    cudaEvent_t done = nullptr;
    bool pending = false;
    uint64_t ticks = 0;          // ticks queued when the copy was issued
};

double now_s(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct ea_srv {
    ea_ctx *ctx = nullptr;
    cudaStream_t st = nullptr;
    int device = 0, dim = 3;
    std::vector<int> Ls;
    size_t mem_budget = 0, mem_used = 0;
    int base_sweeps = 16, poll_ticks = 8, max_ahead = 64, lmax = 0;
    std::chrono::steady_clock::time_point t0;

    // device arrays (per slot), grown with the context
    JobCtl *d_ctl = nullptr;
    int32_t *d_flag = nullptr;
    size_t slot_cap = 0;
    SrvRecord *d_ring = nullptr;
    uint32_t *d_head = nullptr;
    unsigned long long *d_attempts = nullptr;
    SrvStart *d_start = nullptr;
    int32_t *d_slots_io = nullptr;
    uint32_t *d_rids = nullptr, *d_streams = nullptr;

    StageBuf stage[kStageBufs];
    int stage_next = 0;
    ReadBack rb[2];
    int rb_next = 0;
    uint32_t read_cursor = 0;
    unsigned long long attempts = 0;

    // host bookkeeping
    uint64_t next_id = 1, ticks = 0, ticks_read = 0;
    std::deque<HostJob> queue;
    std::unordered_map<uint64_t, HostJob> running;  // by job id
    std::vector<uint64_t> slot_job;                 // slot -> job id (0: free)
    std::vector<std::vector<int32_t>> free_slots;   // per L: free slots
    std::vector<int> lanes;                          // per L: lanes in the pool
    std::vector<ea_srv_result> results;              // finished, not yet polled
    uint64_t n_done = 0, n_censored = 0, n_failed = 0, n_cancelled = 0, n_rt_total = 0;
    uint32_t placeholder = 0x80000000u;
};

namespace {

int idx_of_L(const ea_srv *s, int L) {
    for (size_t k = 0; k < s->Ls.size(); ++k)
        if (s->Ls[k] == L) return (int)k;
    return -1;
}

int sweeps_per_tick(const ea_srv *s, int L) {
    // small lattices get proportionally more sweeps: about equal attempts per tick for every L
    const double r = (double)s->lmax / (double)L;
    const int mul = std::max(1, (int)(r * r * r + 0.5));
    return s->base_sweeps * mul;
}

size_t tile_bytes(int dim, int L) {
    const int V = volume_of(dim, L), B = rows_of(dim, L);
    return (size_t)kTile * B * (8 + 4 + 32 + 16) + 4 * (size_t)(V + dim * V) + kTile * sizeof(SlotState) +
           kTile * (sizeof(JobCtl) + 4);
}

template <class T>
int dev_grow(T **p, size_t old_n, size_t new_n, cudaStream_t st) {
    T *np = nullptr;
    if (cudaMalloc(&np, new_n * sizeof(T)) != cudaSuccess) return fail(EA_ENOMEM, "server allocation failed");
    cudaMemsetAsync(np, 0, new_n * sizeof(T), st);
    if (*p && old_n) cudaMemcpyAsync(np, *p, old_n * sizeof(T), cudaMemcpyDeviceToDevice, st);
    cudaStreamSynchronize(st);
    if (*p) cudaFree(*p);
    *p = np;
    return EA_OK;
}

// adds one tile of lattice size L to the pool (an allocation: only when no lane is free)
int grow_pool(ea_srv *s, int li) {
    const int L = s->Ls[li];
    const size_t need = tile_bytes(s->dim, L);
    if (s->mem_used + need > s->mem_budget) return EA_ENOMEM;
    int first = -1, rc;
    const int W = kTile;
    if ((rc = ea_init_disorder(s->ctx, s->dim, L, W, s->placeholder, 0, nullptr, nullptr, &first))) return rc;
    s->placeholder += W;
    if ((rc = muca_set_sweep_multiplier(s->ctx, L, sweeps_per_tick(s, L) / s->base_sweeps))) return rc;
    if (!s->ctx->d_acc && (rc = muca_set_recursion(s->ctx, first, W, EA_REC_BERG))) return rc;
    const size_t ns = s->ctx->tiles.size() * kTile;
    if (ns > s->slot_cap) {
        const size_t cap = std::max(ns, 2 * s->slot_cap);
        if ((rc = dev_grow(&s->d_ctl, s->slot_cap, cap, s->st)) || (rc = dev_grow(&s->d_flag, s->slot_cap, cap, s->st)))
            return rc;
        s->slot_cap = cap;
        s->slot_job.resize(cap, 0);
    }
    // the new lanes idle until a job is admitted
    std::vector<int32_t> idle;
    for (int k = 0; k < W; ++k) idle.push_back(s->ctx->chain_slot[first + k]);
    if (cudaMemcpyAsync(s->d_slots_io, idle.data(), idle.size() * 4, cudaMemcpyHostToDevice, s->st) != cudaSuccess)
        return fail(EA_ECUDA, "idle upload failed");
    cudaError_t e = launch_srv_cancel(s->ctx->d_slots, s->d_ctl, s->d_slots_io, (int)idle.size(), s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    if (e != cudaSuccess) return cuda_fail(e, "pool growth");
    for (int k = W - 1; k >= 0; --k) s->free_slots[li].push_back(idle[k]);
    s->lanes[li] += W;
    s->mem_used += need;
    return EA_OK;
}

// reads a completed read-back: records from read_cursor to the copied head
int consume(ea_srv *s, ReadBack &r) {
    const double t = now_s(s->t0);
    const uint32_t head = *r.head;
    if (head - s->read_cursor > kRingCap)
        return fail(EA_ESTATE, "completion ring overflow: more than %u jobs finished between two read-backs", kRingCap);
    s->attempts = *r.attempts;
    s->ticks_read = std::max(s->ticks_read, r.ticks);
    for (; s->read_cursor != head; ++s->read_cursor) {
        const SrvRecord &rec = r.ring[s->read_cursor % kRingCap];
        auto it = s->running.find(rec.job);
        if (it == s->running.end()) continue;  // cancelled meanwhile
        HostJob &hj = it->second;
        ea_srv_result out;
        std::memset(&out, 0, sizeof out);
        out.job_id = rec.job;
        out.status = rec.status == kJobDone ? EA_JOB_DONE : rec.status == kJobCensored ? EA_JOB_CENSORED : EA_JOB_FAILED;
        out.L = hj.job.L;
        out.rid = hj.job.rid;
        out.rt_target = hj.job.rt_target;
        out.n_rt = rec.n_rt;
        out.requeues = rec.requeues;
        out.t_first = rec.t_first;
        out.t_last = rec.t_last;
        out.e_g = rec.e_g;
        out.e_min = rec.e_min;
        out.sweeps = rec.sweeps;
        out.t_submit = hj.t_submit;
        out.t_admit = hj.t_admit;
        out.t_done = t;
        s->results.push_back(out);
        if (out.status == EA_JOB_DONE) ++s->n_done;
        else if (out.status == EA_JOB_CENSORED) ++s->n_censored;
        else ++s->n_failed;
        s->n_rt_total += (uint64_t)std::max(0, rec.n_rt);
        const int li = idx_of_L(s, hj.job.L);
        s->slot_job[rec.slot] = 0;
        s->free_slots[li].push_back(rec.slot);
        s->running.erase(it);
    }
    return EA_OK;
}

int poll_readbacks(ea_srv *s, bool wait) {
    for (int k = 0; k < 2; ++k) {
        ReadBack &r = s->rb[(s->rb_next + k) % 2];  // the older one first
        if (!r.pending) continue;
        cudaError_t e = wait ? cudaEventSynchronize(r.done) : cudaEventQuery(r.done);
        if (e == cudaErrorNotReady) continue;
        if (e != cudaSuccess) return cuda_fail(e, "completion read-back");
        r.pending = false;
        const int rc = consume(s, r);
        if (rc) return rc;
    }
    return EA_OK;
}

int issue_readback(ea_srv *s) {
    ReadBack &r = s->rb[s->rb_next];
    if (r.pending) {  // both buffers in flight: wait for this (the older) one
        cudaError_t e = cudaEventSynchronize(r.done);
        if (e != cudaSuccess) return cuda_fail(e, "completion read-back");
        r.pending = false;
        const int rc = consume(s, r);
        if (rc) return rc;
    }
    cudaError_t e = cudaMemcpyAsync(r.head, s->d_head, sizeof(uint32_t), cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r.attempts, s->d_attempts, sizeof(unsigned long long),
                                              cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r.ring, s->d_ring, kRingCap * sizeof(SrvRecord),
                                              cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaEventRecord(r.done, s->st);
    if (e != cudaSuccess) return cuda_fail(e, "completion read-back");
    r.pending = true;
    r.ticks = s->ticks;
    s->rb_next ^= 1;
    return EA_OK;
}

int admit(ea_srv *s) {
    if (s->queue.empty()) return EA_OK;
    StageBuf &sb = s->stage[s->stage_next];
    if (sb.used) {
        cudaError_t e = cudaEventSynchronize(sb.done);  // its uploads are done before reuse
        if (e != cudaSuccess) return cuda_fail(e, "staging buffer");
    }
    std::deque<HostJob> waiting;
    int n = 0;
    const double t = now_s(s->t0);
    while (!s->queue.empty() && n < kMaxStage) {
        HostJob hj = s->queue.front();
        s->queue.pop_front();
        const int li = idx_of_L(s, hj.job.L);
        if (s->free_slots[li].empty()) {
            const int rc = grow_pool(s, li);
            if (rc == EA_ENOMEM) { waiting.push_back(hj); continue; }  // backpressure
            if (rc) return rc;
        }
        const int slot = s->free_slots[li].back();
        s->free_slots[li].pop_back();
        hj.slot = slot;
        hj.t_admit = t;
        SrvStart &st = sb.start[n];
        std::memset(&st, 0, sizeof st);
        st.job = hj.id;
        st.slot = slot;
        st.kind = hj.job.kind;
        st.recursion = hj.job.recursion;
        st.iter_steps = hj.job.iter_steps;
        st.ticks_per_step = hj.job.ticks_per_step;
        st.max_prod_ticks = hj.job.max_prod_ticks;
        st.max_requeues = hj.job.max_requeues;
        st.rt_target = hj.job.rt_target;
        st.sweeps_per_tick = sweeps_per_tick(s, hj.job.L);
        st.alpha = hj.job.alpha;
        st.pole = hj.job.pole;
        sb.slots[n] = slot;
        sb.rids[n] = hj.job.rid;
        sb.streams[n] = hj.job.stream;
        s->slot_job[slot] = hj.id;
        s->running[hj.id] = hj;
        ++n;
    }
    for (auto &w : waiting) s->queue.push_back(w);
    if (n == 0) return EA_OK;
    cudaError_t e = cudaMemcpyAsync(s->d_start, sb.start, n * sizeof(SrvStart), cudaMemcpyHostToDevice, s->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_slots_io, sb.slots, n * 4, cudaMemcpyHostToDevice, s->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_rids, sb.rids, n * 4, cudaMemcpyHostToDevice, s->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_streams, sb.streams, n * 4, cudaMemcpyHostToDevice, s->st);
    ea_ctx *c = s->ctx;
    if (e == cudaSuccess)
        e = launch_reset_lanes(c->d_tiles, c->dim, c->d_slots, c->d_spins, c->d_bonds, c->d_lnW, c->d_hist,
                               s->d_slots_io, s->d_rids, s->d_streams, n, c->key, c->d_err, s->st);
    if (e == cudaSuccess)
        e = launch_srv_start(c->d_tiles, c->d_slots, s->d_ctl, s->d_flag, c->d_acc, s->d_start, n, s->st);
    if (e == cudaSuccess)
        e = launch_quantize_flagged(c->d_tiles, (int)(c->tiles.size() * kTile), c->d_slots, c->d_lnW, c->d_thr,
                                    s->d_flag, s->st);
    if (e == cudaSuccess) e = cudaEventRecord(sb.done, s->st);
    if (e != cudaSuccess) return cuda_fail(e, "admission");
    sb.used = true;
    s->stage_next = (s->stage_next + 1) % kStageBufs;
    return EA_OK;
}

int enqueue_tick(ea_srv *s) {
    ea_ctx *c = s->ctx;
    const int nt = (int)c->tiles.size(), ns = nt * kTile;
    cudaError_t e = cudaSuccess;
    if (c->order == EA_ORDER_COLOUR) {  // the context's colour-order kernels (both parities)
        const int rc = ctx_enqueue_sweeps(c, (uint64_t)s->base_sweeps, 1);
        if (rc) return rc;
    } else {
        e = launch_sweeps(c->d_tiles, nullptr, nt, nt, nullptr, c->dim, c->sweep_smem, c->d_slots, c->d_spins,
                          c->d_bonds, c->d_thr, c->d_hist, (uint64_t)s->base_sweeps, c->key, 1,
                          reinterpret_cast<unsigned *>(c->d_queue + 1), s->st);
    }
    if (e == cudaSuccess)
        e = launch_srv_control(c->d_tiles, ns, c->d_slots, s->d_ctl, s->d_flag, s->d_ring, s->d_head, kRingCap,
                               s->d_attempts, s->ticks + 1, s->st);
    if (e == cudaSuccess) e = launch_srv_update(c->d_tiles, ns, c->d_slots, c->d_lnW, c->d_hist, c->d_acc, s->d_flag, s->st);
    if (e == cudaSuccess)
        e = launch_quantize_flagged(c->d_tiles, ns, c->d_slots, c->d_lnW, c->d_thr, s->d_flag, s->st);
    if (e != cudaSuccess) return cuda_fail(e, "tick");
    ++s->ticks;
    return EA_OK;
}

}  // namespace

extern "C" int ea_srv_create(ea_srv **out, int device, void *cuda_stream, uint64_t seed, const ea_srv_config *cfg) {
    if (!out || !cfg) return fail(EA_EINVAL, "null argument");
    if (cfg->dim != 3 && cfg->dim != 2) return fail(EA_EINVAL, "dim must be 2 or 3");
    if (cfg->n_L <= 0 || cfg->n_L > 16) return fail(EA_EINVAL, "n_L must be in [1, 16]");
    if (cfg->base_sweeps <= 0 || cfg->poll_ticks <= 0 || cfg->max_ahead < cfg->poll_ticks)
        return fail(EA_EINVAL, "need base_sweeps > 0, poll_ticks > 0, max_ahead >= poll_ticks");
    if (cfg->sweep_order != EA_ORDER_LEX && cfg->sweep_order != EA_ORDER_COLOUR)
        return fail(EA_EINVAL, "unknown sweep order %d", cfg->sweep_order);
    ea_srv *s = new ea_srv();
    s->device = device;
    s->dim = cfg->dim;
    s->mem_budget = cfg->mem_budget;
    s->base_sweeps = cfg->base_sweeps;
    s->poll_ticks = cfg->poll_ticks;
    s->max_ahead = cfg->max_ahead;
    for (int k = 0; k < cfg->n_L; ++k) {
        const int L = cfg->Ls[k];
        if (L < 3 || L > 12) { delete s; return fail(EA_EINVAL, "L must be in [3, 12]"); }
        s->Ls.push_back(L);
        s->lmax = std::max(s->lmax, L);
    }
    s->free_slots.resize(s->Ls.size());
    s->lanes.assign(s->Ls.size(), 0);
    s->st = (cudaStream_t)cuda_stream;
    s->t0 = std::chrono::steady_clock::now();
    int rc = ea_create(&s->ctx, device, cuda_stream, seed);
    if (rc) { delete s; return rc; }
    if ((rc = muca_set_sweep_order(s->ctx, cfg->sweep_order, 0))) { ea_destroy(s->ctx); delete s; return rc; }
    if (cfg->sweep_order == EA_ORDER_COLOUR) {
        // the narrowest tiles whose thresholds fit in shared memory: each served chain runs as
        // fast as it can (jobs are few per lattice size), the pool holds fewer lanes per tile
        for (int L : s->Ls)
            for (int w : {4, 8, 16})
                if (muca_set_tile_width(s->ctx, L, w) == EA_OK) break;
    }
    bool ok = cudaMalloc(&s->d_ring, kRingCap * sizeof(SrvRecord)) == cudaSuccess &&
              cudaMalloc(&s->d_head, sizeof(uint32_t)) == cudaSuccess &&
              cudaMalloc(&s->d_attempts, sizeof(unsigned long long)) == cudaSuccess &&
              cudaMalloc(&s->d_start, kMaxStage * sizeof(SrvStart)) == cudaSuccess &&
              cudaMalloc(&s->d_slots_io, kMaxStage * 4) == cudaSuccess &&
              cudaMalloc(&s->d_rids, kMaxStage * 4) == cudaSuccess &&
              cudaMalloc(&s->d_streams, kMaxStage * 4) == cudaSuccess;
    for (int k = 0; ok && k < kStageBufs; ++k) {
        StageBuf &b = s->stage[k];
        ok = cudaMallocHost(&b.start, kMaxStage * sizeof(SrvStart)) == cudaSuccess &&
             cudaMallocHost(&b.slots, kMaxStage * 4) == cudaSuccess &&
             cudaMallocHost(&b.rids, kMaxStage * 4) == cudaSuccess &&
             cudaMallocHost(&b.streams, kMaxStage * 4) == cudaSuccess &&
             cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming) == cudaSuccess;
    }
    for (int k = 0; ok && k < 2; ++k) {
        ReadBack &r = s->rb[k];
        ok = cudaMallocHost(&r.ring, kRingCap * sizeof(SrvRecord)) == cudaSuccess &&
             cudaMallocHost(&r.head, sizeof(uint32_t)) == cudaSuccess &&
             cudaMallocHost(&r.attempts, sizeof(unsigned long long)) == cudaSuccess &&
             cudaEventCreateWithFlags(&r.done, cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) { ea_srv_destroy(s); return fail(EA_ENOMEM, "server allocation failed"); }
    cudaMemsetAsync(s->d_head, 0, sizeof(uint32_t), s->st);
    cudaMemsetAsync(s->d_attempts, 0, sizeof(unsigned long long), s->st);
    cudaStreamSynchronize(s->st);
    *out = s;
    return EA_OK;
}

extern "C" void ea_srv_destroy(ea_srv *s) {
    if (!s) return;
    if (s->ctx) {
        cudaSetDevice(s->device);
        cudaStreamSynchronize(s->st);
    }
    void *dev[] = {s->d_ctl, s->d_flag, s->d_ring, s->d_head, s->d_attempts, s->d_start, s->d_slots_io, s->d_rids,
                   s->d_streams};
    for (void *p : dev)
        if (p) cudaFree(p);
    for (StageBuf &b : s->stage) {
        void *h[] = {b.start, b.slots, b.rids, b.streams};
        for (void *p : h)
            if (p) cudaFreeHost(p);
        if (b.done) cudaEventDestroy(b.done);
    }
    for (ReadBack &r : s->rb) {
        void *h[] = {r.ring, r.head, r.attempts};
        for (void *p : h)
            if (p) cudaFreeHost(p);
        if (r.done) cudaEventDestroy(r.done);
    }
    if (s->ctx) ea_destroy(s->ctx);
    delete s;
}

extern "C" int ea_srv_submit(ea_srv *s, const ea_job *job, uint64_t *job_id) {
    if (!s || !job) return fail(EA_EINVAL, "null argument");
    if (idx_of_L(s, job->L) < 0) return fail(EA_EINVAL, "L=%d is not served", job->L);
    if (job->kind != EA_FLAT && job->kind != EA_POWERLAW) return fail(EA_EINVAL, "kind must be EA_FLAT or EA_POWERLAW");
    if (job->kind == EA_POWERLAW && !(job->pole > 0.0)) return fail(EA_EINVAL, "pole must be > 0");
    if (job->recursion != EA_REC_PLAIN && job->recursion != EA_REC_BERG) return fail(EA_EINVAL, "unknown recursion");
    if (job->rt_target < 1 || job->iter_steps < 1 || job->ticks_per_step < 1 || job->max_prod_ticks < 1 ||
        job->max_requeues < 0)
        return fail(EA_EINVAL, "rt_target, iter_steps, ticks_per_step, max_prod_ticks must be >= 1");
    if (job->stream >= (1u << 24)) return fail(EA_EINVAL, "stream must be < 2^24");
    // a job's sweep counter must stay below 2^32
    const uint64_t ticks_max = (uint64_t)job->iter_steps * job->ticks_per_step +
                               (uint64_t)(job->max_requeues + 1) * job->max_prod_ticks;
    if (ticks_max * (uint64_t)sweeps_per_tick(s, job->L) >= (1ull << 32))
        return fail(EA_EINVAL, "the job's schedule would exceed 2^32 sweeps");
    HostJob hj;
    hj.id = s->next_id++;
    hj.job = *job;
    hj.t_submit = now_s(s->t0);
    s->queue.push_back(hj);
    if (job_id) *job_id = hj.id;
    return EA_OK;
}

extern "C" int ea_srv_cancel(ea_srv *s, uint64_t job_id) {
    if (!s) return fail(EA_EINVAL, "null server");
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
        if (it->id == job_id) {
            s->queue.erase(it);
            ++s->n_cancelled;
            return EA_OK;
        }
    auto it = s->running.find(job_id);
    if (it == s->running.end()) return fail(EA_ESTATE, "job %llu is not waiting or running", (unsigned long long)job_id);
    // stream-ordered: the lane stops before any later tick, and a job admitted into it later is
    // reset after that
    const int32_t slot = it->second.slot;
    StageBuf &sb = s->stage[s->stage_next];
    if (sb.used) {
        cudaError_t e = cudaEventSynchronize(sb.done);
        if (e != cudaSuccess) return cuda_fail(e, "staging buffer");
    }
    sb.slots[0] = slot;
    cudaError_t e = cudaMemcpyAsync(s->d_slots_io, sb.slots, 4, cudaMemcpyHostToDevice, s->st);
    if (e == cudaSuccess) e = launch_srv_cancel(s->ctx->d_slots, s->d_ctl, s->d_slots_io, 1, s->st);
    if (e == cudaSuccess) e = cudaEventRecord(sb.done, s->st);
    if (e != cudaSuccess) return cuda_fail(e, "cancel");
    sb.used = true;
    s->stage_next = (s->stage_next + 1) % kStageBufs;
    const int li = idx_of_L(s, it->second.job.L);
    s->slot_job[slot] = 0;
    s->free_slots[li].push_back(slot);
    s->running.erase(it);
    ++s->n_cancelled;
    return EA_OK;
}

extern "C" int ea_srv_step(ea_srv *s, int ticks) {
    if (!s) return fail(EA_EINVAL, "null server");
    if (ticks < 0) return fail(EA_EINVAL, "negative tick count");
    int rc;
    if ((rc = cudaSetDevice(s->device) == cudaSuccess ? EA_OK : fail(EA_ECUDA, "cudaSetDevice"))) return rc;
    if ((rc = poll_readbacks(s, false))) return rc;
    if ((rc = admit(s))) return rc;
    for (int k = 0; k < ticks; ++k) {
        if (s->running.empty()) break;  // nothing to advance
        // flow control: at most max_ahead ticks beyond the last read-back the host has seen
        while (s->ticks >= s->ticks_read + (uint64_t)s->max_ahead) {
            bool any = s->rb[0].pending || s->rb[1].pending;
            if (!any && (rc = issue_readback(s))) return rc;
            if ((rc = poll_readbacks(s, true))) return rc;
        }
        if ((rc = enqueue_tick(s))) return rc;
        if (s->ticks % (uint64_t)s->poll_ticks == 0 && (rc = issue_readback(s))) return rc;
    }
    return EA_OK;
}

extern "C" int ea_srv_poll(ea_srv *s, ea_srv_result *out, int cap, int *n_out, int wait) {
    if (!s || !n_out || (cap > 0 && !out)) return fail(EA_EINVAL, "null argument");
    int rc;
    if (wait) {  // everything queued so far is read back
        if ((rc = issue_readback(s)) || (rc = poll_readbacks(s, true)) || (rc = poll_readbacks(s, true))) return rc;
    } else if ((rc = poll_readbacks(s, false))) {
        return rc;
    }
    const int n = std::min<int>(cap, (int)s->results.size());
    for (int k = 0; k < n; ++k) out[k] = s->results[k];
    s->results.erase(s->results.begin(), s->results.begin() + n);
    *n_out = n;
    return EA_OK;
}

extern "C" int ea_srv_stats(ea_srv *s, ea_srv_counters *out) {
    if (!s || !out) return fail(EA_EINVAL, "null argument");
    std::memset(out, 0, sizeof *out);
    out->ticks = s->ticks;
    out->ticks_read = s->ticks_read;
    out->attempts = s->attempts;
    out->queued = (int32_t)s->queue.size();
    out->running = (int32_t)s->running.size();
    out->done = s->n_done;
    out->censored = s->n_censored;
    out->failed = s->n_failed;
    out->cancelled = s->n_cancelled;
    out->round_trips = s->n_rt_total;
    out->mem_used = s->mem_used;
    int lanes = 0;
    for (int l : s->lanes) lanes += l;
    out->lanes = lanes;
    out->seconds = now_s(s->t0);
    return EA_OK;
}

extern "C" size_t ea_srv_tile_bytes(int dim, int L) {
    if ((dim != 2 && dim != 3) || L < 3 || L > 12) return 0;
    return tile_bytes(dim, L);
}

extern "C" int ea_srv_context(ea_srv *s, ea_ctx **ctx) {
    if (!s || !ctx) return fail(EA_EINVAL, "null argument");
    *ctx = s->ctx;
    return EA_OK;
}
