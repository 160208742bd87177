// iod_batch.cu -- host side of the batch / serving interface (include/iod.h).
//
// Residency and memory: each admitted request gets one device allocation (through the
// allocator hook) holding its observation table, constants, swarm, block winners,
// trace and, for IOD_MIXED, the chief's stage tables; admission stops at the memory
// budget or the slot limit (first come, first served).  Rounds: a plan kernel picks
// every resident problem's next action from its device state, then per size class one
// FP32 and one FP64 round kernel pull that class's tiles from atomic queues.  The rounds
// of a step are captured once as a CUDA graph and replayed until residency changes.
#include "iod.h"
#include "iod_internal.h"

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <vector>

using namespace iod;

namespace {

enum ReqState { kQueued = 0, kResident = 1, kDone = 2, kCancelled = 3, kFailed = 4 };

struct Req {
    double mu = 0;
    double chief[6] = {};
    std::vector<double> t, ang;
    double sigma[2] = {}, bounds[12] = {};
    int m = 0, iters = 0;
    double w = 0, c1 = 0, c2 = 0;
    uint64_t seed = 0;
    int state = kQueued, slot = -1;
    double t_submit = -1, t_admit = -1, t_done = -1;
    GBest gb{};
    std::vector<double> trace_J;
    std::vector<int> trace_idx;
};

struct SlotH {
    long long ticket = -1;
    DevBuf buf;
    int cls = 0, n_tiles = 0, trace_cap = 0;
    long long steps_bound = 0;
    size_t bytes = 0, smem_mix = 0, smem_fp64 = 0;
    double cost = 0;
};

// per-slot allocation layout (every region 256-byte aligned)
struct Layout {
    size_t obs, misc, swarm, blk, trace, mix, cs, od, ct, lm, total;
};

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

Layout layout(int K, int m, int n_tiles, int trace_cap, long long steps_bound, bool mixed, bool refine)
{
    Layout L{};
    size_t o = 0;
    L.obs = o;
    o = up256(o + (8 * sizeof(double) + sizeof(int)) * (size_t)K);
    L.misc = o;
    o = up256(o + kMiscBytes);
    L.swarm = o;
    o = up256(o + 20 * sizeof(double) * (size_t)m);
    L.blk = o;
    o = up256(o + sizeof(BlockBest) * (size_t)n_tiles);
    L.trace = o;
    o = up256(o + (sizeof(double) + sizeof(int)) * (size_t)trace_cap);
    if (mixed) {
        const long long ch = mixed_chunk_steps();
        L.mix = o;
        o = up256(o + sizeof(mix::Step) * (size_t)steps_bound);
        L.cs = o;
        o = up256(o + 6 * sizeof(double) * (size_t)(steps_bound + 1));
        L.od = o;
        o = up256(o + sizeof(mix::ObsDir) * (size_t)K);
        L.ct = o;
        o = up256(o + sizeof(float) * (size_t)((steps_bound + ch - 1) / ch + 1));
    }
    if (refine) {
        // Levenberg-Marquardt scratch: kLmVecs residual vectors of at most 2K entries and the
        // carried state
        L.lm = o;
        o = up256(o + sizeof(double) * (kLmVecs * 2 * (size_t)K + kLmTail));
    }
    L.total = o;
    return L;
}

// An upper bound on the RK4 steps of the interval rule: n_k <= span_k/dt + 1.
long long steps_bound(const std::vector<double> &t, double dt)
{
    return (long long)std::ceil(t.back() / dt) + (long long)t.size() + 1;
}

bool finite_n(const double *v, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

}  // namespace

struct iod_batch {
    iod_options opt{};
    size_t budget = 0;
    int max_resident = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<int> cls_max{1024, 4096, INT_MAX};
    std::vector<int> cls_block{128, 128, 128};
    // RK4 step bound by size class (iod_batch_set_step_sizes; empty: opt.dt for all)
    std::vector<int> dt_max;
    std::vector<double> dt_val;
    std::map<long long, Req> reqs;
    std::deque<long long> queue;
    long long next_ticket = 1;
    std::vector<SlotH> slots;
    std::vector<int> free_slots;
    DevBuf d_slots, d_ids, d_queues, d_tiles, d_actions;
    DevBuf d_wq, d_ring, d_seq;   // dependency-driven scheduler
    unsigned long long ring_cap = 0;
    std::vector<BatchSlot> h_slots;
    size_t in_use = 0, high_water = 0;
    long long deferred = 0;    // admissions put off because an allocation failed
    long long finished = 0, rounds_run = 0;
    // tile tables per distinct block size
    std::vector<int> grp_block, grp_grid, tile_off, tile_n;
    std::vector<size_t> grp_smem;
    size_t tiles_cap = 0;
    bool dirty = true;
    cudaGraphExec_t graph = nullptr;
    int graph_rounds = 0;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();

    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    double dt_of(int m) const
    {
        for (size_t c = 0; c < dt_max.size(); ++c)
            if (m <= dt_max[c]) return dt_val[c];
        return opt.dt;
    }

    int class_of(int m) const
    {
        for (size_t c = 0; c < cls_max.size(); ++c)
            if (m <= cls_max[c]) return (int)c;
        return (int)cls_max.size() - 1;
    }
    bool mixed() const { return opt.precision == IOD_MIXED; }
    int trace_cap_for(const Req &r) const { return opt.record_trace ? r.iters + 2 : 0; }

    size_t bytes_for(const Req &r) const
    {
        const int nt = (r.m + cls_block[class_of(r.m)] - 1) / cls_block[class_of(r.m)];
        return layout((int)r.t.size(), r.m, nt, trace_cap_for(r), steps_bound(r.t, dt_of(r.m)), mixed(),
                      opt.refine_iters > 0).total;
    }

    void drop_graph()
    {
        if (graph) cudaGraphExecDestroy(graph);
        graph = nullptr;
        graph_rounds = 0;
    }

    ~iod_batch()
    {
        cudaStreamSynchronize(stream);
        drop_graph();
        for (auto &s : slots) dev_free(s.buf);
        dev_free(d_slots);
        dev_free(d_ids);
        dev_free(d_queues);
        dev_free(d_tiles);
        dev_free(d_actions);
        dev_free(d_wq);
        dev_free(d_ring);
        dev_free(d_seq);
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
};

namespace {

int admit(iod_batch *b)
{
    std::vector<int> ids;
    while (!b->queue.empty()) {
        const long long tk = b->queue.front();
        Req &r = b->reqs[tk];
        if (r.state != kQueued) {
            b->queue.pop_front();
            continue;
        }
        if (b->free_slots.empty()) break;
        const size_t bytes = b->bytes_for(r);
        if (b->in_use + bytes > b->budget) break;
        b->queue.pop_front();
        const int si = b->free_slots.back();
        b->free_slots.pop_back();
        SlotH &S = b->slots[si];
        S = SlotH();
        S.ticket = tk;
        S.cls = b->class_of(r.m);
        const int block = b->cls_block[S.cls];
        S.n_tiles = (r.m + block - 1) / block;
        S.trace_cap = b->trace_cap_for(r);
        S.steps_bound = steps_bound(r.t, b->dt_of(r.m));
        const int K = (int)r.t.size();
        const Layout L = layout(K, r.m, S.n_tiles, S.trace_cap, S.steps_bound, b->mixed(), b->opt.refine_iters > 0);
        int rc = dev_alloc(S.buf, L.total);
        if (rc) {
            b->free_slots.push_back(si);
            S.ticket = -1;
            if (b->in_use > 0) {
                // device memory comes back as resident problems retire: the request
                // stays first in the queue and admission backs off until the next call
                b->queue.push_front(tk);
                ++b->deferred;
                break;
            }
            r.state = kFailed;     // nothing resident whose memory could come back
            continue;
        }
        S.bytes = L.total;
        S.smem_mix = b->mixed() ? mixed_smem_bytes(K, S.steps_bound) : 0;
        S.smem_fp64 = swarm_smem_bytes(K, IOD_RK4);
        S.cost = (double)S.steps_bound;
        char *base = (char *)S.buf.ptr;
        // inputs: t, alpha~, beta~ (range unused), chief state; counters cleared
        std::vector<double> host(4 * (size_t)K, 0.0);
        for (int k = 0; k < K; ++k) {
            host[k] = r.t[k];
            host[K + k] = r.ang[2 * k];
            host[2 * K + k] = r.ang[2 * k + 1];
        }
        cudaError_t e = cudaMemcpyAsync(base + L.obs, host.data(), sizeof(double) * 4 * K,
                                        cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(base + L.misc, 0, kMiscBytes, b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(base + L.misc + kMiscChief, r.chief, sizeof(r.chief), cudaMemcpyHostToDevice,
                                b->stream);
        if (e != cudaSuccess) return cuda_error(e, "batch admission copy");
        // descriptor
        BatchSlot D{};
        KParams &P = D.P;
        double *obs = (double *)(base + L.obs);
        P.mu = r.mu;
        P.n_obs = K;
        P.integrator = IOD_RK4;
        P.dynamics = IOD_CR3BP;
        P.ecc = 0.0;
        P.f0 = 0.0;
        P.cost_form = b->opt.cost_form;
        P.use_range = 0;
        P.dt = b->dt_of(r.m);
        P.rtol = b->opt.rtol;
        P.atol = b->opt.atol;
        P.h0 = b->opt.h0;
        P.max_steps = b->opt.max_steps;
        for (int d = 0; d < 6; ++d) {
            P.lo[d] = r.bounds[d];
            P.hi[d] = r.bounds[6 + d];
        }
        P.w = r.w;
        P.c1 = r.c1;
        P.c2 = r.c2;
        P.seed = r.seed;
        P.tol_tau = b->opt.tol_tau;
        P.tol_window = b->opt.tol_window;
        P.constriction = b->opt.constriction;
        P.kappa = P.constriction ? constriction_kappa(r.c1, r.c2) : 1.0;
        P.init_grid = b->opt.init_grid;
        P.init_cone = b->opt.init_cone;
        P.velocity_init = b->opt.velocity_init;
        P.per_dim_random = b->opt.per_dim_random;
        if (P.init_cone)
            cone_frame(r.ang[0], r.ang[1], r.sigma[0], r.sigma[1], b->opt.cone_sigmas, b->opt.cone_rho_min,
                       b->opt.cone_rho_max, P.cone);
        P.total_steps = 0;   // written by the set-up kernel
        P.m = r.m;
        P.stride = r.m;
        P.offset = 0;
        P.m_total = r.m;
        P.t = obs;
        P.ra = obs + K;
        P.dec = obs + 2 * K;
        P.rng = nullptr;
        P.rc = obs + 4 * K;
        P.h = obs + 7 * K;
        P.nsteps = (const int *)(obs + 8 * K);
        P.cst = (const Consts *)(base + L.misc);
        P.gb = (GBest *)(base + L.misc + kMiscGBest);
        double *sw = (double *)(base + L.swarm);
        P.x = sw;
        P.v = sw + 6 * (size_t)r.m;
        P.p = sw + 12 * (size_t)r.m;
        P.pJ = sw + 18 * (size_t)r.m;
        P.J = sw + 19 * (size_t)r.m;
        P.blk = (BlockBest *)(base + L.blk);
        P.trace_J = S.trace_cap ? (double *)(base + L.trace) : nullptr;
        P.trace_idx = S.trace_cap ? (int *)((double *)(base + L.trace) + S.trace_cap) : nullptr;
        P.trace_cap = S.trace_cap;
        P.moon_r2 = b->opt.moon_fp64_radius * b->opt.moon_fp64_radius;
        if (b->mixed()) {
            P.mix = (const mix::Step *)(base + L.mix);
            P.chief_cs = (const double *)(base + L.cs);
            P.obsdir = (const mix::ObsDir *)(base + L.od);
            P.chunk_time = (const float *)(base + L.ct);
        }
        const int last = b->opt.fp64_last_iters < r.iters ? b->opt.fp64_last_iters : r.iters;
        D.n_mixed = b->mixed() ? r.iters - last : -1;
        D.n_iters = r.iters;
        D.n_tiles = S.n_tiles;
        D.active = 1;
        D.chief = (const double *)(base + L.misc + kMiscChief);
        D.sig_ra = r.sigma[0];
        D.sig_dec = r.sigma[1];
        D.sig_rng = 0.0;
        D.vmax_frac = b->opt.vmax_frac;
        D.rc_w = obs + 4 * K;
        D.h_w = obs + 7 * K;
        D.ns_w = (int *)(obs + 8 * K);
        D.cst_w = (Consts *)(base + L.misc);
        D.mix_w = (mix::Step *)P.mix;
        D.cs_w = (double *)P.chief_cs;
        D.od_w = (mix::ObsDir *)P.obsdir;
        D.ct_w = (float *)P.chunk_time;
        D.refine_iters = b->opt.refine_iters;
        D.gate_cost = b->opt.refine_gate > 0.0 ? b->opt.refine_gate * (double)K : 0.0;
        D.lm_R = b->opt.refine_iters > 0 ? (double *)(base + L.lm) : nullptr;
        b->h_slots[si] = D;
        e = cudaMemcpyAsync((BatchSlot *)b->d_slots.ptr + si, &b->h_slots[si], sizeof(BatchSlot),
                            cudaMemcpyHostToDevice, b->stream);
        if (e != cudaSuccess) return cuda_error(e, "batch descriptor copy");
        r.state = kResident;
        r.slot = si;
        r.t_admit = b->now();
        b->in_use += L.total;
        b->high_water = std::max(b->high_water, b->in_use);
        ids.push_back(si);
        b->dirty = true;
    }
    if (!ids.empty()) {
        cudaError_t e = cudaMemcpyAsync(b->d_ids.ptr, ids.data(), sizeof(int) * ids.size(),
                                        cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = launch_batch_setup((BatchSlot *)b->d_slots.ptr, (const int *)b->d_ids.ptr,
                                                     (int)ids.size(), b->stream);
        // the host copies above come from pageable vectors that die here
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return cuda_error(e, "batch set-up");
    }
    return IOD_OK;
}

// Tile tables: one per distinct block size (classes that share a block size share a
// table and a launch), longest work first so the tail of each round is short.
int rebuild_tiles(iod_batch *b)
{
    std::vector<int> blocks;
    for (int blk : b->cls_block)
        if (std::find(blocks.begin(), blocks.end(), blk) == blocks.end()) blocks.push_back(blk);
    const int ng = (int)blocks.size();
    std::vector<std::vector<int2>> per(ng);
    b->grp_block = blocks;
    b->grp_smem.assign(ng, 0);
    std::vector<int> order;
    for (int s = 0; s < b->max_resident; ++s)
        if (b->slots[s].ticket >= 0) order.push_back(s);
    std::sort(order.begin(), order.end(), [&](int a, int c) { return b->slots[a].cost > b->slots[c].cost; });
    for (int s : order) {
        const SlotH &S = b->slots[s];
        const int g = (int)(std::find(blocks.begin(), blocks.end(), b->cls_block[S.cls]) - blocks.begin());
        for (int t = 0; t < S.n_tiles; ++t) per[g].push_back(make_int2(s, t));
        b->grp_smem[g] = std::max(b->grp_smem[g], std::max(S.smem_mix, S.smem_fp64));
    }
    size_t total = 0;
    b->tile_off.assign(ng, 0);
    b->tile_n.assign(ng, 0);
    for (int g = 0; g < ng; ++g) {
        b->tile_off[g] = (int)total;
        b->tile_n[g] = (int)per[g].size();
        total += per[g].size();
    }
    if (total > b->tiles_cap) {
        cudaStreamSynchronize(b->stream);
        dev_free(b->d_tiles);
        const size_t cap = std::max(total, 2 * b->tiles_cap);
        int rc = dev_alloc(b->d_tiles, sizeof(int2) * cap);
        if (rc) {
            b->tiles_cap = 0;
            return rc;
        }
        b->tiles_cap = cap;
    }
    std::vector<int2> flat;
    flat.reserve(total);
    for (int g = 0; g < ng; ++g) flat.insert(flat.end(), per[g].begin(), per[g].end());
    if (total) {
        cudaError_t e = cudaMemcpyAsync(b->d_tiles.ptr, flat.data(), sizeof(int2) * total,
                                        cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return cuda_error(e, "tile table copy");
    }
    // shared-memory limit set here, outside any stream capture
    size_t mx = 0;
    for (size_t v : b->grp_smem) mx = std::max(mx, v);
    cudaError_t pe = batch_round_prepare(mx);
    if (pe != cudaSuccess) return cuda_error(pe, "batch kernel attributes");
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    b->grp_grid.assign(ng, 0);
    for (int g = 0; g < ng; ++g)
        if (b->tile_n[g])
            b->grp_grid[g] = std::min(b->tile_n[g], std::max(1, batch_round_occupancy(blocks[g], b->grp_smem[g])) * sms);
    b->dirty = false;
    b->drop_graph();
    return IOD_OK;
}

cudaError_t queue_rounds(iod_batch *b, int rounds)
{
    BatchSlot *slots = (BatchSlot *)b->d_slots.ptr;
    BatchQueue *q = (BatchQueue *)b->d_queues.ptr;
    const int2 *tiles = (const int2 *)b->d_tiles.ptr;
    for (int r = 0; r < rounds; ++r) {
        cudaError_t e = launch_batch_plan(slots, b->max_resident, b->stream);
        if (e != cudaSuccess) return e;
        for (size_t g = 0; g < b->grp_block.size(); ++g) {
            e = launch_batch_round(slots, tiles + b->tile_off[g], b->tile_n[g], q + g, b->grp_block[g],
                                   b->grp_grid[g], b->grp_smem[g], b->stream);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

int retire(iod_batch *b)
{
    cudaError_t e = launch_batch_plan((BatchSlot *)b->d_slots.ptr, b->max_resident, b->stream);
    // the planned actions live in the descriptors: read them all back in one copy
    std::vector<BatchSlot> dev(b->max_resident);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dev.data(), b->d_slots.ptr, sizeof(BatchSlot) * dev.size(), cudaMemcpyDeviceToHost,
                            b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_error(e, "batch plan");
    for (int s = 0; s < b->max_resident; ++s) {
        SlotH &S = b->slots[s];
        if (S.ticket < 0 || dev[s].action != kActNone) continue;
        Req &r = b->reqs[S.ticket];
        const KParams &P = b->h_slots[s].P;
        e = cudaMemcpy(&r.gb, P.gb, sizeof(GBest), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && S.trace_cap) {
            const int n = std::min(S.trace_cap, r.gb.iter + 1);
            r.trace_J.resize(n);
            r.trace_idx.resize(n);
            if (n > 0) {
                e = cudaMemcpy(r.trace_J.data(), P.trace_J, sizeof(double) * n, cudaMemcpyDeviceToHost);
                if (e == cudaSuccess)
                    e = cudaMemcpy(r.trace_idx.data(), P.trace_idx, sizeof(int) * n, cudaMemcpyDeviceToHost);
            }
        }
        if (e != cudaSuccess) return cuda_error(e, "batch result read");
        if (r.state == kResident) r.state = r.gb.status ? kFailed : kDone;
        r.t_done = b->now();
        r.slot = -1;
        b->in_use -= S.bytes;
        // the descriptor stays in the device array: mark it inactive before its memory is
        // freed, so that no later plan or scheduler launch reads the freed problem state
        static const int kInactive = 0;
        b->h_slots[s].active = 0;
        e = cudaMemcpyAsync(&((BatchSlot *)b->d_slots.ptr)[s].active, &kInactive, sizeof(int),
                            cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return cuda_error(e, "batch retire");
        dev_free(S.buf);
        S = SlotH();
        b->free_slots.push_back(s);
        ++b->finished;
        b->dirty = true;
    }
    return IOD_OK;
}

}  // namespace

extern "C" {

int iod_batch_create(const iod_options *opt, size_t device_budget_bytes, int max_resident, iod_batch **out)
{
    if (!out) return set_last_error(IOD_EINVAL, "out is NULL");
    *out = nullptr;
    iod_options o;
    if (opt)
        o = *opt;
    else
        iod_options_default(&o);
    if (o.integrator != IOD_RK4) return set_last_error(IOD_EINVAL, "batches run the RK4 integrator");
    if (o.use_range) return set_last_error(IOD_EINVAL, "batches take angle observations only");
    if (o.dynamics != IOD_CR3BP) return set_last_error(IOD_EINVAL, "batches run the CR3BP dynamics");
    if (!(o.dt > 0) || o.fp64_last_iters < 0 || !(o.moon_fp64_radius >= 0) || !(o.vmax_frac > 0))
        return set_last_error(IOD_EINVAL, "invalid options");
    if (o.precision != IOD_FP64 && o.precision != IOD_MIXED) return set_last_error(IOD_EINVAL, "precision");
    if (!(o.tol_tau >= 0) || !std::isfinite(o.tol_tau) ||
        (o.tol_tau > 0 && (o.tol_window < 1 || o.tol_window >= kTolHist)) ||
        (o.constriction != 0 && o.constriction != 1) || (o.init_grid != 0 && o.init_grid != 1))
        return set_last_error(IOD_EINVAL, "invalid Algorithm 2 / constriction / grid options");
    if ((o.init_cone != 0 && o.init_cone != 1) ||
        (o.init_cone && (!(o.cone_rho_min >= 0) || !(o.cone_rho_max > o.cone_rho_min) ||
                         !std::isfinite(o.cone_rho_max) || !(o.cone_sigmas > 0) || !std::isfinite(o.cone_sigmas))))
        return set_last_error(IOD_EINVAL, "invalid line-of-sight initialisation options");
    if ((o.velocity_init != 0 && o.velocity_init != 1) || (o.per_dim_random != 0 && o.per_dim_random != 1))
        return set_last_error(IOD_EINVAL, "velocity_init and per_dim_random must be 0 or 1");
    if (o.refine_iters < 0 || o.refine_iters > 10000)
        return set_last_error(IOD_EINVAL, "refine_iters must lie in [0, 10000]");
    if (!(o.refine_gate >= 0.0) || !std::isfinite(o.refine_gate) || (o.refine_gate > 0.0 && o.refine_iters == 0))
        return set_last_error(IOD_EINVAL, "refine_gate must be finite and >= 0, and > 0 only with refine_iters");
    if (o.shard_offset != 0 || o.shard_total != 0)
        return set_last_error(IOD_EINVAL, "batch requests are not sharded (shard_offset = shard_total = 0)");
    if (max_resident < 1 || device_budget_bytes == 0) return set_last_error(IOD_EINVAL, "empty batch");
    iod_batch *b = new (std::nothrow) iod_batch();
    if (!b) return set_last_error(IOD_ENOMEM, "host allocation");
    b->opt = o;
    b->budget = device_budget_bytes;
    b->max_resident = max_resident;
    b->slots.resize(max_resident);
    b->h_slots.resize(max_resident);
    for (int s = max_resident - 1; s >= 0; --s) b->free_slots.push_back(s);
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete b;
        return cuda_error(e, "cudaStreamCreate");
    }
    b->own_stream = true;
    int rc = dev_alloc(b->d_slots, sizeof(BatchSlot) * (size_t)max_resident);
    if (!rc) rc = dev_alloc(b->d_ids, sizeof(int) * (size_t)max_resident);
    if (!rc) rc = dev_alloc(b->d_queues, sizeof(BatchQueue) * 16);
    if (rc) {
        delete b;
        return rc;
    }
    e = cudaMemsetAsync(b->d_slots.ptr, 0, sizeof(BatchSlot) * (size_t)max_resident, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_queues.ptr, 0, sizeof(BatchQueue) * 16, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        delete b;
        return cuda_error(e, "batch create");
    }
    *out = b;
    return IOD_OK;
}

int iod_batch_set_stream(iod_batch *b, void *cuda_stream)
{
    if (!b) return set_last_error(IOD_EINVAL, "batch is NULL");
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
    if (b->own_stream) cudaStreamDestroy(b->stream);
    b->own_stream = false;
    b->stream = (cudaStream_t)cuda_stream;
    b->drop_graph();
    return IOD_OK;
}

int iod_batch_set_block_sizes(iod_batch *b, int n_classes, const int *max_swarm, const int *block)
{
    if (!b || n_classes < 1 || n_classes > 8 || !max_swarm || !block) return set_last_error(IOD_EINVAL, "bad classes");
    for (int c = 0; c < n_classes; ++c) {
        if (block[c] < 32 || block[c] > max_block_threads() || block[c] % 32) return set_last_error(IOD_EINVAL, "block size");
        if (c && max_swarm[c] <= max_swarm[c - 1]) return set_last_error(IOD_EINVAL, "classes must increase");
    }
    for (auto &s : b->slots)
        if (s.ticket >= 0) return set_last_error(IOD_ESTATE, "block sizes change only while nothing is resident");
    b->cls_max.assign(max_swarm, max_swarm + n_classes);
    b->cls_max.back() = INT_MAX;
    b->cls_block.assign(block, block + n_classes);
    b->dirty = true;
    return IOD_OK;
}

int iod_batch_set_step_sizes(iod_batch *b, int n_classes, const int *max_swarm, const double *dt)
{
    if (!b || n_classes < 1 || n_classes > 8 || !max_swarm || !dt) return set_last_error(IOD_EINVAL, "bad classes");
    for (int c = 0; c < n_classes; ++c) {
        if (!(dt[c] > 0) || !std::isfinite(dt[c])) return set_last_error(IOD_EINVAL, "dt must be finite and > 0");
        if (c && max_swarm[c] <= max_swarm[c - 1]) return set_last_error(IOD_EINVAL, "classes must increase");
    }
    for (auto &s : b->slots)
        if (s.ticket >= 0) return set_last_error(IOD_ESTATE, "step sizes change only while nothing is resident");
    b->dt_max.assign(max_swarm, max_swarm + n_classes);
    b->dt_max.back() = INT_MAX;
    b->dt_val.assign(dt, dt + n_classes);
    return IOD_OK;
}

int iod_batch_submit(iod_batch *b, const iod_request *q, long long *ticket)
{
    const NvtxRange nvtx_range("iod_batch_submit");
    if (!b || !q || !ticket) return set_last_error(IOD_EINVAL, "NULL argument");
    if (!(q->mu > 0 && q->mu < 0.5) || q->n_obs < 1 || q->swarm_size < 1 || q->iters < 0)
        return set_last_error(IOD_EINVAL, "bad request sizes");
    if (!q->chief_state || !q->obs_times || !q->obs_angles || !q->sigma || !q->bounds)
        return set_last_error(IOD_EINVAL, "NULL request array");
    if (!finite_n(q->chief_state, 6) || !finite_n(q->obs_times, q->n_obs) ||
        !finite_n(q->obs_angles, 2 * (size_t)q->n_obs) || !finite_n(q->sigma, 2) || !finite_n(q->bounds, 12) ||
        !std::isfinite(q->w) || !std::isfinite(q->c1) || !std::isfinite(q->c2))
        return set_last_error(IOD_EINVAL, "non-finite request value");
    if (b->opt.constriction && !(q->c1 + q->c2 > 4.0))
        return set_last_error(IOD_EINVAL, "the constriction factor needs c1 + c2 > 4");
    if (!(q->obs_times[0] >= 0)) return set_last_error(IOD_EINVAL, "obs_times must be >= 0");
    if (b->opt.init_cone && q->obs_times[0] != 0.0)
        return set_last_error(IOD_EINVAL, "init_cone needs the first observation at t = 0");
    for (int k = 1; k < q->n_obs; ++k)
        if (!(q->obs_times[k] > q->obs_times[k - 1])) return set_last_error(IOD_EINVAL, "obs_times must increase");
    if (!(q->sigma[0] > 0) || !(q->sigma[1] > 0)) return set_last_error(IOD_EINVAL, "sigma must be > 0");
    for (int d = 0; d < 6; ++d)
        if (!(q->bounds[d] < q->bounds[6 + d])) return set_last_error(IOD_EINVAL, "bounds: lo must be < hi");
    Req r;
    r.mu = q->mu;
    std::memcpy(r.chief, q->chief_state, sizeof r.chief);
    r.t.assign(q->obs_times, q->obs_times + q->n_obs);
    r.ang.assign(q->obs_angles, q->obs_angles + 2 * (size_t)q->n_obs);
    std::memcpy(r.sigma, q->sigma, sizeof r.sigma);
    std::memcpy(r.bounds, q->bounds, sizeof r.bounds);
    r.m = q->swarm_size;
    r.iters = q->iters;
    r.w = q->w;
    r.c1 = q->c1;
    r.c2 = q->c2;
    r.seed = q->seed;
    const size_t smax_need = std::max(swarm_smem_bytes(q->n_obs, IOD_RK4),
                                      b->mixed() ? mixed_smem_bytes(q->n_obs, steps_bound(r.t, b->dt_of(q->swarm_size))) : 0);
    int dev = 0, smax = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (smax > 0 && smax_need + 2048 > (size_t)smax) return set_last_error(IOD_EINVAL, "n_obs too large");
    if (b->bytes_for(r) > b->budget) return set_last_error(IOD_ENOMEM, "request alone exceeds the device budget");
    r.t_submit = b->now();
    const long long tk = b->next_ticket++;
    b->reqs.emplace(tk, std::move(r));
    b->queue.push_back(tk);
    *ticket = tk;
    return IOD_OK;
}

int iod_batch_step(iod_batch *b, int rounds)
{
    const NvtxRange nvtx_range("iod_batch_step");
    if (!b || rounds < 0) return set_last_error(IOD_EINVAL, "bad step");
    int rc = admit(b);
    if (rc) return rc;
    if (b->dirty && (rc = rebuild_tiles(b))) return rc;
    bool any = false;
    for (auto &s : b->slots) any = any || s.ticket >= 0;
    if (any && rounds > 0) {
        cudaError_t e = cudaSuccess;
        cudaStreamCaptureStatus cs;
        const bool can_capture = b->stream != nullptr && b->stream != cudaStreamLegacy &&
                                 b->stream != cudaStreamPerThread &&
                                 cudaStreamIsCapturing(b->stream, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone;
        if (can_capture) {
            if (!b->graph || b->graph_rounds != rounds) {
                b->drop_graph();
                cudaGraph_t g = nullptr;
                e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    cudaError_t le = queue_rounds(b, rounds);
                    e = cudaStreamEndCapture(b->stream, &g);
                    if (le != cudaSuccess) e = le;
                }
                if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
                if (g) cudaGraphDestroy(g);
                if (e != cudaSuccess) {
                    b->drop_graph();
                    return cuda_error(e, "batch graph capture");
                }
                b->graph_rounds = rounds;
            }
            e = cudaGraphLaunch(b->graph, b->stream);
        } else {
            e = queue_rounds(b, rounds);
        }
        if (e != cudaSuccess) return cuda_error(e, "batch rounds");
        b->rounds_run += rounds;
    }
    return retire(b);
}

int iod_batch_run(iod_batch *b, double seconds)
{
    const NvtxRange nvtx_range("iod_batch_run");
    if (!b || !(seconds >= 0) || !std::isfinite(seconds)) return set_last_error(IOD_EINVAL, "bad run time");
    for (int blk : b->cls_block)
        if (blk != b->cls_block[0]) return set_last_error(IOD_EINVAL, "iod_batch_run needs one block size");
    int rc = admit(b);
    if (rc) return rc;
    if (b->dirty && (rc = rebuild_tiles(b))) return rc;
    int total_tiles = 0, any = 0;
    size_t smem = 0;
    for (auto &S : b->slots)
        if (S.ticket >= 0) {
            total_tiles += S.n_tiles;
            smem = std::max(smem, std::max(S.smem_mix, S.smem_fp64));
            any = 1;
        }
    if (any) {
        const int block = b->cls_block[0];
        int dev = 0, sms = 1, coop = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        if (!coop) return set_last_error(IOD_EINVAL, "the GPU has no cooperative launch");
        // the throughput form (more resident blocks, slower chains) once the tiles are more
        // than twice what the latency form holds at once
        const int occ_lat = wq_occupancy(block, smem, 0);
        const int thr = (long long)total_tiles >= 2LL * occ_lat * sms ? 1 : 0;
        const int occ = thr ? wq_occupancy(block, smem, 1) : occ_lat;
        if (occ < 1) return set_last_error(IOD_EINVAL, "scheduler kernel does not fit on an SM");
        const int grid = occ * sms;
        // ring: every published-unconsumed item plus every waiting claimant fits twice
        unsigned long long need = 1024;
        while (need < 2ull * (unsigned long long)(total_tiles + grid)) need <<= 1;
        if (!b->d_wq.ptr) {
            if ((rc = dev_alloc(b->d_wq, sizeof(WorkQueue)))) return rc;
            cudaError_t e = cudaMemsetAsync(b->d_wq.ptr, 0, sizeof(WorkQueue), b->stream);
            if (e != cudaSuccess) return cuda_error(e, "scheduler init");
        }
        if (need > b->ring_cap) {
            cudaStreamSynchronize(b->stream);
            dev_free(b->d_ring);
            dev_free(b->d_seq);
            b->ring_cap = 0;
            if ((rc = dev_alloc(b->d_ring, sizeof(int2) * need))) return rc;
            if ((rc = dev_alloc(b->d_seq, sizeof(unsigned long long) * need))) return rc;
            // no stamp matches an index until it is published
            cudaError_t e = cudaMemsetAsync(b->d_seq.ptr, 0xFF, sizeof(unsigned long long) * need, b->stream);
            if (e != cudaSuccess) return cuda_error(e, "scheduler ring init");
            b->ring_cap = need;
        }
        const unsigned long long budget_ns = seconds > 0 ? (unsigned long long)(seconds * 1e9) : 0ull;
        cudaError_t e = launch_wq_seed((BatchSlot *)b->d_slots.ptr, b->max_resident, (WorkQueue *)b->d_wq.ptr,
                                       (int2 *)b->d_ring.ptr, (unsigned long long *)b->d_seq.ptr, b->ring_cap,
                                       b->stream);
        if (e == cudaSuccess)
            e = launch_wq_run((BatchSlot *)b->d_slots.ptr, (WorkQueue *)b->d_wq.ptr, (int2 *)b->d_ring.ptr,
                              (unsigned long long *)b->d_seq.ptr, b->ring_cap, budget_ns, block, grid, smem,
                              thr, b->stream);
        if (e != cudaSuccess) return cuda_error(e, "scheduler launch");
        WorkQueue wq;
        e = cudaMemcpyAsync(&wq, b->d_wq.ptr, sizeof wq, cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return cuda_error(e, "scheduler run");
        if (wq.status & (kWqTimeout | kWqCopyLost)) {
            // fail whatever did not finish; the queue's stamps are reset for the next run
            BatchSlot *d = (BatchSlot *)b->d_slots.ptr;
            for (int s = 0; s < b->max_resident; ++s) {
                if (b->slots[s].ticket < 0) continue;
                int st = 4;
                cudaMemcpyAsync(&((GBest *)b->h_slots[s].P.gb)->status, &st, sizeof(int),
                                cudaMemcpyHostToDevice, b->stream);
            }
            (void)d;
            cudaMemsetAsync(b->d_seq.ptr, 0xFF, sizeof(unsigned long long) * b->ring_cap, b->stream);
            cudaStreamSynchronize(b->stream);
            retire(b);
            return set_last_error(IOD_ETIMEOUT, (wq.status & kWqCopyLost)
                                                    ? "a chief-table copy never landed; the launch was stopped"
                                                    : "a scheduler wait gave up");
        }
        b->rounds_run += 1;
    }
    return retire(b);
}

int iod_batch_poll(iod_batch *b, long long ticket, iod_result_t *out)
{
    if (!b || !out) return set_last_error(IOD_EINVAL, "NULL argument");
    auto it = b->reqs.find(ticket);
    if (it == b->reqs.end()) return set_last_error(IOD_EINVAL, "unknown ticket");
    const Req &r = it->second;
    if (r.state == kQueued || r.state == kResident) return IOD_EBUSY;
    if (r.state == kCancelled) return IOD_ECANCELLED;
    if (r.state == kFailed) return set_last_error(r.gb.status ? IOD_ETIMEOUT : IOD_ENOMEM, "request failed");
    std::memcpy(out->state, r.gb.g, sizeof out->state);
    out->cost = r.gb.gJ;
    if (r.gb.flags & kFlagRefined) {
        std::memcpy(out->pso_state, r.gb.g_pso, sizeof out->pso_state);
        out->pso_cost = r.gb.gJ_pso;
        out->refine_iters = r.gb.lm_iters;
    } else {
        std::memcpy(out->pso_state, r.gb.g, sizeof out->pso_state);
        out->pso_cost = r.gb.gJ;
        out->refine_iters = 0;
    }
    out->fallback = (r.gb.flags & kFlagFallback) ? 1 : 0;
    out->gbest_index = r.gb.gidx;
    out->iters_done = r.gb.iter;
    out->rk_steps = (long long)r.gb.steps;
    out->fp64_steps = (long long)r.gb.steps64;
    out->schedule = IOD_SCHED_GRID;   // batches run their own persistent scheduler
    if (out->gcost_trace && out->gidx_trace && out->trace_capacity > 0) {
        const int n = std::min((int)r.trace_J.size(), out->trace_capacity);
        std::memcpy(out->gcost_trace, r.trace_J.data(), sizeof(double) * n);
        std::memcpy(out->gidx_trace, r.trace_idx.data(), sizeof(int) * n);
    }
    return IOD_OK;
}

int iod_batch_times(iod_batch *b, long long ticket, double *t_submit, double *t_admit, double *t_done)
{
    if (!b) return set_last_error(IOD_EINVAL, "batch is NULL");
    auto it = b->reqs.find(ticket);
    if (it == b->reqs.end()) return set_last_error(IOD_EINVAL, "unknown ticket");
    if (t_submit) *t_submit = it->second.t_submit;
    if (t_admit) *t_admit = it->second.t_admit;
    if (t_done) *t_done = it->second.t_done;
    return IOD_OK;
}

int iod_batch_cancel(iod_batch *b, long long ticket)
{
    if (!b) return set_last_error(IOD_EINVAL, "batch is NULL");
    auto it = b->reqs.find(ticket);
    if (it == b->reqs.end()) return set_last_error(IOD_EINVAL, "unknown ticket");
    Req &r = it->second;
    if (r.state == kQueued) {
        r.state = kCancelled;
        return IOD_OK;
    }
    if (r.state != kResident) return IOD_OK;
    r.state = kCancelled;
    int zero = 0;
    cudaError_t e = cudaMemcpyAsync(&((BatchSlot *)b->d_slots.ptr)[r.slot].active, &zero, sizeof(int),
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    return e == cudaSuccess ? IOD_OK : cuda_error(e, "batch cancel");
}

int iod_batch_get_stats(iod_batch *b, iod_batch_stats *out)
{
    if (!b || !out) return set_last_error(IOD_EINVAL, "NULL argument");
    out->resident = 0;
    for (auto &s : b->slots) out->resident += s.ticket >= 0;
    out->queued = 0;
    for (long long tk : b->queue) out->queued += b->reqs[tk].state == kQueued;
    out->finished = b->finished;
    out->rounds = b->rounds_run;
    out->bytes_in_use = b->in_use;
    out->deferred_admissions = b->deferred;
    out->bytes_high_water = b->high_water;
    out->budget = b->budget;
    return IOD_OK;
}

void iod_batch_destroy(iod_batch *b) { delete b; }

namespace {
// Probes of the step-size autotuner: the sample's own initial swarm (its first n
// particles, Philox initialisation in its box), and the lines of sight from the chief to
// each probe at every epoch under a DOPRI5 reference propagation (tolerance 1e-13) of
// both.
struct ProbeSet {
    int n = 0, K = 0;
    std::vector<double> x;      // [6][n] initial states
    std::vector<double> los;    // [K][n][3] unit lines of sight (reference)
};

int create_sample(const iod_request *q, const iod_options &o, iod_problem **p)
{
    return iod_create(q->mu, q->chief_state, q->n_obs, q->obs_times, q->obs_angles, q->sigma, q->bounds, &o, p);
}

// Unit lines of sight [K][n][3] of n states x ([6][n], host) propagated by problem p.
int lines_of_sight(iod_problem *p, const iod_request *q, const std::vector<double> &x, int n,
                   std::vector<double> &los)
{
    const int K = q->n_obs;
    DevBuf buf;
    int rc = dev_alloc(buf, sizeof(double) * (6 * (size_t)n + 6 * (size_t)K * n));
    if (rc) return rc;
    double *dx = (double *)buf.ptr, *dout = dx + 6 * (size_t)n;
    cudaError_t e = cudaMemcpy(dx, x.data(), sizeof(double) * 6 * n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        dev_free(buf);
        return cuda_error(e, "probe copy");
    }
    rc = iod_propagate(p, dx, n, dout);
    std::vector<double> out(6 * (size_t)K * n), rc3(3 * (size_t)K);
    if (!rc) {
        e = cudaMemcpy(out.data(), dout, sizeof(double) * out.size(), cudaMemcpyDeviceToHost);
        rc = e == cudaSuccess ? iod_chief_positions(p, rc3.data()) : cuda_error(e, "probe read");
    }
    dev_free(buf);
    if (rc) return rc;
    los.assign(3 * (size_t)K * n, 0.0);
    for (int k = 0; k < K; ++k)
        for (int i = 0; i < n; ++i) {
            double r[3], rr = 0.0;
            for (int a = 0; a < 3; ++a) {
                r[a] = out[((size_t)k * 6 + a) * n + i] - rc3[3 * (size_t)k + a];
                rr += r[a] * r[a];
            }
            rr = std::sqrt(rr);
            for (int a = 0; a < 3; ++a) los[((size_t)k * n + i) * 3 + a] = rr > 0 ? r[a] / rr : 0.0;
        }
    return IOD_OK;
}

int probe_states(const iod_request *q, const iod_options &base, int n, ProbeSet &ps)
{
    iod_options o = base;
    o.integrator = IOD_RK4;
    o.precision = IOD_FP64;
    o.refine_iters = 0;
    o.refine_gate = 0.0;
    o.record_trace = 0;
    o.threads_per_particle = 1;
    iod_problem *p = nullptr;
    int rc = create_sample(q, o, &p);
    if (rc) return rc;
    rc = iod_run(p, n, 0, q->w, q->c1, q->c2, q->seed);     // initial positions only
    ps.n = n;
    ps.K = q->n_obs;
    ps.x.assign(6 * (size_t)n, 0.0);
    if (!rc) rc = iod_swarm_get(p, ps.x.data(), nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
    iod_destroy(p);
    if (rc) return rc;
    o.integrator = IOD_DOPRI5;
    o.rtol = o.atol = 1e-13;
    o.h0 = 1e-3;
    if ((rc = create_sample(q, o, &p))) return rc;
    rc = lines_of_sight(p, q, ps.x, n, ps.los);
    iod_destroy(p);
    return rc;
}

// Largest angle between the reference lines of sight and those of an RK4 propagation
// at step bound dt (each side with its own chief trajectory), over probes and epochs.
int probe_angle_error(const iod_request *q, const iod_options &base, double dt, const ProbeSet &ps, double *err)
{
    iod_options o = base;
    o.integrator = IOD_RK4;
    o.precision = IOD_FP64;
    o.refine_iters = 0;
    o.refine_gate = 0.0;
    o.record_trace = 0;
    o.dt = dt;
    iod_problem *p = nullptr;
    int rc = create_sample(q, o, &p);
    if (rc) return rc;
    std::vector<double> los;
    rc = lines_of_sight(p, q, ps.x, ps.n, los);
    iod_destroy(p);
    if (rc) return rc;
    double worst = 0.0;
    for (size_t j = 0; j < los.size(); j += 3) {
        const double *a = &ps.los[j], *b2 = &los[j];
        const double cx = a[1] * b2[2] - a[2] * b2[1], cy = a[2] * b2[0] - a[0] * b2[2],
                     cz = a[0] * b2[1] - a[1] * b2[0];
        const double ang = std::atan2(std::sqrt(cx * cx + cy * cy + cz * cz),
                                      a[0] * b2[0] + a[1] * b2[1] + a[2] * b2[2]);
        worst = std::max(worst, ang);
    }
    *err = worst;
    return IOD_OK;
}

// Time one iteration of a sample problem run alone with the given block size and
// precision (events around one iod_continue after initialisation and a warm-up).
int time_iteration(const iod_request *q, const iod_options &base, int precision, int block, double *ms)
{
    iod_options o = base;
    o.refine_iters = 0;        // the sample is timed as a swarm (the refinement is not tuned)
    o.refine_gate = 0.0;
    o.precision = precision;
    o.block_size = block;
    o.threads_per_particle = 1;   // the batch kernels run one thread per particle
    o.fp64_last_iters = 0;
    o.record_trace = 0;
    iod_problem *p = nullptr;
    int rc = iod_create(q->mu, q->chief_state, q->n_obs, q->obs_times, q->obs_angles, q->sigma, q->bounds, &o, &p);
    if (rc) return rc;
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    iod_set_stream(p, st);
    cudaEvent_t a, z;
    cudaEventCreate(&a);
    cudaEventCreate(&z);
    rc = iod_run(p, q->swarm_size, 0, q->w, q->c1, q->c2, q->seed);
    if (!rc) rc = iod_continue(p, 1);
    if (!rc) {
        cudaEventRecord(a, st);
        rc = iod_continue(p, 1);
        cudaEventRecord(z, st);
    }
    cudaError_t e = cudaStreamSynchronize(st);
    float f = 0.0f;
    if (!rc && e == cudaSuccess) cudaEventElapsedTime(&f, a, z);
    *ms = f;
    cudaEventDestroy(a);
    cudaEventDestroy(z);
    iod_destroy(p);
    cudaStreamDestroy(st);
    if (!rc && e != cudaSuccess) rc = cuda_error(e, "autotune timing");
    return rc;
}
}  // namespace

int iod_batch_autotune(iod_batch *b, int n_classes, const int *max_swarm, const iod_request *samples,
                       int n_cand, const int *cand, int uniform, int *block_out, double *ms_out)
{
    const NvtxRange nvtx_range("iod_batch_autotune");
    if (!b || n_classes < 1 || n_classes > 8 || !max_swarm || !samples || n_cand < 1 || !cand || !block_out)
        return set_last_error(IOD_EINVAL, "bad autotune arguments");
    for (auto &s : b->slots)
        if (s.ticket >= 0) return set_last_error(IOD_ESTATE, "autotune while problems are resident");
    std::vector<double> T((size_t)n_classes * n_cand, 0.0);
    for (int c = 0; c < n_classes; ++c) {
        const iod_request *q = &samples[c];
        const int last = std::min(b->opt.fp64_last_iters, q->iters);
        const double n32 = b->mixed() ? (double)(q->iters - last) : 0.0;
        const double n64 = b->mixed() ? (double)last + 1.0 : (double)q->iters;
        for (int j = 0; j < n_cand; ++j) {
            double ms32 = 0.0, ms64 = 0.0;
            int rc = 0;
            iod_options oc = b->opt;
            oc.dt = b->dt_of(q->swarm_size);        // the class's step bound
            if (n32 > 0) rc = time_iteration(q, oc, IOD_MIXED, cand[j], &ms32);
            if (!rc && n64 > 0) rc = time_iteration(q, oc, IOD_FP64, cand[j], &ms64);
            if (rc) return rc;
            T[(size_t)c * n_cand + j] = n32 * ms32 + n64 * ms64;
        }
    }
    std::vector<int> best(n_classes, cand[0]);
    if (uniform) {
        int bj = 0;
        double bt = -1.0;
        for (int j = 0; j < n_cand; ++j) {
            double tot = 0.0;
            for (int c = 0; c < n_classes; ++c) tot += T[(size_t)c * n_cand + j];
            if (bt < 0 || tot < bt) {
                bt = tot;
                bj = j;
            }
        }
        for (int c = 0; c < n_classes; ++c) best[c] = cand[bj];
    } else {
        for (int c = 0; c < n_classes; ++c) {
            int bj = 0;
            for (int j = 1; j < n_cand; ++j)
                if (T[(size_t)c * n_cand + j] < T[(size_t)c * n_cand + bj]) bj = j;
            best[c] = cand[bj];
        }
    }
    int rc = iod_batch_set_block_sizes(b, n_classes, max_swarm, best.data());
    if (rc) return rc;
    for (int c = 0; c < n_classes; ++c) block_out[c] = best[c];
    if (ms_out) std::memcpy(ms_out, T.data(), sizeof(double) * T.size());
    return IOD_OK;
}

int iod_batch_autotune_dt(iod_batch *b, int n_classes, const int *max_swarm, const iod_request *samples,
                          int n_dt, const double *dt_cand, double angle_budget, int n_probe, double *dt_out,
                          double *err_out)
{
    const NvtxRange nvtx_range("iod_batch_autotune_dt");
    if (!b || n_classes < 1 || n_classes > 8 || !max_swarm || !samples || n_dt < 1 || !dt_cand || !dt_out ||
        !(angle_budget > 0) || n_probe < 1 || n_probe > 4096)
        return set_last_error(IOD_EINVAL, "bad step-size autotune arguments");
    for (int j = 0; j < n_dt; ++j)
        if (!(dt_cand[j] > 0) || !std::isfinite(dt_cand[j])) return set_last_error(IOD_EINVAL, "dt candidates");
    for (auto &s : b->slots)
        if (s.ticket >= 0) return set_last_error(IOD_ESTATE, "autotune while problems are resident");
    std::vector<double> E((size_t)n_classes * n_dt, 0.0), chosen(n_classes);
    for (int c = 0; c < n_classes; ++c) {
        const iod_request *q = &samples[c];
        ProbeSet ps;
        int rc = probe_states(q, b->opt, n_probe, ps);
        if (rc) return rc;
        double best = -1.0, smallest = dt_cand[0];
        for (int j = 0; j < n_dt; ++j) {
            double err = 0.0;
            if ((rc = probe_angle_error(q, b->opt, dt_cand[j], ps, &err))) return rc;
            E[(size_t)c * n_dt + j] = err;
            smallest = std::min(smallest, dt_cand[j]);
            if (err <= angle_budget && dt_cand[j] > best) best = dt_cand[j];
        }
        chosen[c] = best > 0 ? best : smallest;
    }
    int rc = iod_batch_set_step_sizes(b, n_classes, max_swarm, chosen.data());
    if (rc) return rc;
    std::memcpy(dt_out, chosen.data(), sizeof(double) * n_classes);
    if (err_out) std::memcpy(err_out, E.data(), sizeof(double) * E.size());
    return IOD_OK;
}

}  // extern "C"
