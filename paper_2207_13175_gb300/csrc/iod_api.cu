// iod_api.cu -- host implementation of the C ABI declared in include/iod.h.
//
// Validation, device memory ownership, stream ordering and launch sequencing live
// here; all arithmetic of the method runs in the kernels of iod_kernels.cu.
#include "iod.h"
#include "iod_internal.h"

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

using iod::BlockBest;
using iod::Consts;
using iod::GBest;
using iod::KParams;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string &msg)
{
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *where)
{
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? IOD_ENOMEM : IOD_ECUDA;
}

#define IOD_CUDA(call, where)                               \
    do {                                                    \
        cudaError_t _e = (call);                            \
        if (_e != cudaSuccess) return cuda_fail(_e, where); \
    } while (0)

bool finite_all(const double *v, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

int max_smem_optin()
{
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
    return v;
}

int sm_count()
{
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    return v > 0 ? v : 1;
}

}  // namespace

int iod::set_last_error(int code, const char *msg) { return fail(code, msg); }

namespace iod {

std::mutex g_alloc_mu;
Allocator g_alloc;


int dev_alloc(DevBuf &b, size_t bytes)
{
    Allocator a;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        a = g_alloc;
    }
    void *p = nullptr;
    if (a.alloc) {
        p = a.alloc(bytes, a.ctx);
        if (!p) return fail(IOD_ENOMEM, "allocator hook returned NULL for " + std::to_string(bytes) + " bytes");
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return cuda_fail(e, "cudaMalloc");
        }
    }
    b.ptr = p;
    b.bytes = bytes;
    b.a = a;
    return IOD_OK;
}

void dev_free(DevBuf &b)
{
    if (!b.ptr) return;
    if (b.a.release)
        b.a.release(b.ptr, b.a.ctx);
    else
        cudaFree(b.ptr);
    b.ptr = nullptr;
    b.bytes = 0;
}


int cuda_error(cudaError_t e, const char *where) { return cuda_fail(e, where); }

}  // namespace iod

using iod::DevBuf;
using iod::dev_alloc;
using iod::dev_free;
using iod::g_alloc;
using iod::g_alloc_mu;


struct iod_problem {
    int device = 0;
    cudaStream_t stream = nullptr;
    iod_options opt{};
    double mu = 0;
    double chief[6] = {};
    int n_obs = 0;
    double sigma[2] = {};
    double lo[6] = {}, hi[6] = {};
    // device memory
    DevBuf obs;      // t, ra, dec, rng, rc[3], h (8 n_obs doubles) then nsteps (n_obs ints)
    DevBuf misc;     // Consts, GBest, chief state
    DevBuf swarm;    // x, v, p [6][stride] each, then pJ, J [stride]
    DevBuf blk;      // BlockBest per block
    DevBuf trace;    // gJ [cap] then gidx [cap]
    DevBuf mix;      // mixed precision: chief stage table, chief states, observed directions
    DevBuf lm;       // refinement scratch: kLmVecs residual vectors and the carried state, start state, output
    DevBuf split;    // balanced iteration: SplitCtl, plan, flags, hand-off
    long long total_steps = 0;   // RK4 steps per propagation (sum of n_k)
    int max_interval_steps = 0;  // largest n_k
    long long mix_cap = 0;       // steps the mixed-precision tables are laid out for
    int phase = 0;               // mixed precision: 0 = FP32 exploration, 1 = FP64 refinement
    int m = 0, stride = 0, m_cap = 0, grid_cap = 0, trace_cap = 0;
    int block = 64;
    int tpp = 1;                 // threads per particle of the current swarm (1 or 2)
    int sched = 0;               // 1: balanced FP64 iterations (iter_kernel_balanced)
    int sched_mixed = 0;         // 1: balanced FP32 iterations of IOD_MIXED (iter_mixed_balanced)
    int last_sched = IOD_SCHED_GRID;   // work distribution of the last iteration launched
    int wps = 4;                 // balanced FP64: warps per SM (one to three per sub-partition)
    int split_m = -1, split_nw = -1, split_gs = -1;   // what the current plan was made for
    double w = 0, c1 = 0, c2 = 0;
    uint64_t seed = 0;
    bool started = false;
    int iters_done = 0;
    iod::ConeInit cone{};

    double *d_t() const { return (double *)obs.ptr; }
    double *d_ra() const { return d_t() + n_obs; }
    double *d_dec() const { return d_t() + 2 * n_obs; }
    double *d_rng() const { return d_t() + 3 * n_obs; }
    double *d_rc() const { return d_t() + 4 * n_obs; }
    double *d_h() const { return d_t() + 7 * n_obs; }
    int *d_ns() const { return (int *)(d_t() + 8 * n_obs); }
    Consts *d_cst() const { return (Consts *)misc.ptr; }
    GBest *d_gb() const { return (GBest *)((char *)misc.ptr + iod::kMiscGBest); }
    double *d_chief() const { return (double *)((char *)misc.ptr + iod::kMiscChief); }

    // mixed-precision tables, laid out for mix_cap steps (a bound on the interval rule's
    // step count, known before the set-up kernel counts the steps: the set-up writes the
    // chief's step-boundary states into this buffer)
    size_t mix_cs_offset() const { return (sizeof(iod::mix::Step) * (size_t)mix_cap + 255) & ~(size_t)255; }
    size_t mix_dir_offset() const
    {
        return mix_cs_offset() + ((sizeof(double) * 6 * (size_t)(mix_cap + 1) + 255) & ~(size_t)255);
    }
    size_t mix_ct_offset() const
    {
        return (mix_dir_offset() + sizeof(iod::mix::ObsDir) * (size_t)n_obs + 255) & ~(size_t)255;
    }
    size_t mix_bytes() const
    {
        const long long ch = iod::mixed_chunk_steps();
        return mix_ct_offset() + sizeof(float) * (size_t)((mix_cap + ch - 1) / ch + 1);
    }

    KParams params() const
    {
        KParams P{};
        P.mu = mu;
        P.n_obs = n_obs;
        P.integrator = opt.integrator;
        P.dynamics = opt.dynamics;
        P.ecc = opt.dynamics == IOD_ER3BP ? opt.ecc : 0.0;
        P.f0 = opt.dynamics == IOD_ER3BP ? opt.f0 : 0.0;
        P.cost_form = opt.cost_form;
        P.use_range = opt.use_range;
        P.dt = opt.dt;
        P.rtol = opt.rtol;
        P.atol = opt.atol;
        P.h0 = opt.h0;
        P.max_steps = opt.max_steps;
        for (int d = 0; d < 6; ++d) {
            P.lo[d] = lo[d];
            P.hi[d] = hi[d];
        }
        P.w = w;
        P.c1 = c1;
        P.c2 = c2;
        P.seed = seed;
        P.tol_tau = opt.tol_tau;
        P.tol_window = opt.tol_window;
        P.constriction = opt.constriction;
        P.kappa = opt.constriction ? iod::constriction_kappa(c1, c2) : 1.0;
        P.init_grid = opt.init_grid;
        P.init_cone = opt.init_cone;
        P.velocity_init = opt.velocity_init;
        P.pair = tpp == 2;
        P.per_dim_random = opt.per_dim_random;
        P.cone = cone;
        P.m = m;
        P.stride = stride;
        P.offset = opt.shard_total > 0 ? opt.shard_offset : 0;
        P.m_total = opt.shard_total > 0 ? opt.shard_total : m;
        P.t = d_t();
        P.ra = d_ra();
        P.dec = d_dec();
        P.rng = opt.use_range ? d_rng() : nullptr;
        P.rc = d_rc();
        P.h = d_h();
        P.nsteps = d_ns();
        P.cst = d_cst();
        P.mix = (const iod::mix::Step *)mix.ptr;
        P.chief_cs = mix.ptr ? (const double *)((char *)mix.ptr + mix_cs_offset()) : nullptr;
        P.obsdir = mix.ptr ? (const iod::mix::ObsDir *)((char *)mix.ptr + mix_dir_offset()) : nullptr;
        P.chunk_time = mix.ptr ? (const float *)((char *)mix.ptr + mix_ct_offset()) : nullptr;
        P.moon_r2 = opt.moon_fp64_radius * opt.moon_fp64_radius;
        P.total_steps = total_steps;
        double *sw = (double *)swarm.ptr;
        P.x = sw;
        P.v = sw ? sw + 6 * (size_t)stride : nullptr;
        P.p = sw ? sw + 12 * (size_t)stride : nullptr;
        P.pJ = sw ? sw + 18 * (size_t)stride : nullptr;
        P.J = sw ? sw + 19 * (size_t)stride : nullptr;
        P.gb = d_gb();
        P.blk = (BlockBest *)blk.ptr;
        P.trace_J = opt.record_trace ? (double *)trace.ptr : nullptr;
        P.trace_idx = opt.record_trace && trace.ptr ? (int *)((double *)trace.ptr + trace_cap) : nullptr;
        P.trace_cap = opt.record_trace ? trace_cap : 0;
        P.split = (iod::SplitCtl *)split.ptr;
        P.chief0 = d_chief();
        return P;
    }

    ~iod_problem()
    {
        if (obs.ptr || misc.ptr || swarm.ptr) cudaStreamSynchronize(stream);
        dev_free(obs);
        dev_free(misc);
        dev_free(swarm);
        dev_free(blk);
        dev_free(trace);
        dev_free(mix);
        dev_free(lm);
        dev_free(split);
    }
};

namespace iod {

// ER3BP: true anomaly after nondimensional time tau from f0 (unit mean motion).  The
// mean anomaly advances by tau; Newton's method solves Kepler's equation E - e sin E = M
// from E = M; the half-angle relation tan((f - E)/2) = b sin E/(1 - b cos E) with
// b = e/(1 + sqrt(1 - e^2)) gives a continuous (unwrapped) f.
double er3bp_true_anomaly(double e, double f0, double tau)
{
    if (e == 0.0) return f0 + tau;
    const double b = e / (1.0 + std::sqrt(1.0 - e * e));
    const double E0 = f0 - 2.0 * std::atan(b * std::sin(f0) / (1.0 + b * std::cos(f0)));
    const double M = (E0 - e * std::sin(E0)) + tau;
    double E = M;
    for (int it = 0; it < 100; ++it) {
        const double dE = (E - e * std::sin(E) - M) / (1.0 - e * std::cos(E));
        E -= dE;
        if (std::fabs(dE) <= 1e-15 * std::fmax(1.0, std::fabs(E))) break;
    }
    return E + 2.0 * std::atan(b * std::sin(E) / (1.0 - b * std::cos(E)));
}

double constriction_kappa(double c1, double c2)
{
    const double phi = c1 + c2;
    const double disc = phi * phi - 4.0 * phi;
    return 2.0 / std::fabs(2.0 - phi - std::sqrt(disc));
}

// Direction of (alpha0, beta0) as in Eqs. 7-8 and its tangent directions; products only,
// so the result does not depend on floating-point contraction.
void cone_frame(double alpha0, double beta0, double sig_ra, double sig_dec, double k, double rho_min,
                double rho_max, ConeInit &out)
{
    const double ca = std::cos(alpha0), sa = std::sin(alpha0), cb = std::cos(beta0), sb = std::sin(beta0);
    out.u[0] = cb * ca;
    out.u[1] = cb * sa;
    out.u[2] = sb;
    out.ea[0] = -sa;
    out.ea[1] = ca;
    out.ea[2] = 0.0;
    out.eb[0] = -sb * ca;
    out.eb[1] = -sb * sa;
    out.eb[2] = cb;
    out.smax[0] = k * sig_ra * cb;
    out.smax[1] = k * sig_dec;
    out.rho[0] = rho_min;
    out.rho[1] = rho_max;
}

}  // namespace iod

namespace {

int validate_options(const iod_options &o)
{
    if (o.integrator != IOD_RK4 && o.integrator != IOD_DOPRI5) return fail(IOD_EINVAL, "integrator");
    if (!(o.dt > 0) || !std::isfinite(o.dt)) return fail(IOD_EINVAL, "dt must be finite and > 0");
    if (!(o.rtol >= 0) || !(o.atol >= 0) || !(o.rtol > 0 || o.atol > 0) || !std::isfinite(o.rtol) ||
        !std::isfinite(o.atol))
        return fail(IOD_EINVAL, "rtol/atol");
    if (!(o.h0 > 0) || !std::isfinite(o.h0)) return fail(IOD_EINVAL, "h0 must be finite and > 0");
    if (o.max_steps < 1) return fail(IOD_EINVAL, "max_steps must be >= 1");
    if (o.precision != IOD_FP64 && o.precision != IOD_MIXED) return fail(IOD_EINVAL, "precision");
    if (o.precision == IOD_MIXED && o.integrator != IOD_RK4)
        return fail(IOD_EINVAL, "IOD_MIXED needs the RK4 integrator");
    if (o.fp64_last_iters < 0) return fail(IOD_EINVAL, "fp64_last_iters must be >= 0");
    if (!(o.moon_fp64_radius >= 0) || !std::isfinite(o.moon_fp64_radius))
        return fail(IOD_EINVAL, "moon_fp64_radius must be finite and >= 0");
    if (o.cost_form != IOD_COST_CHI2 && o.cost_form != IOD_COST_QUARTIC) return fail(IOD_EINVAL, "cost_form");
    if (o.gbest_order != IOD_GBEST_SYNC && o.gbest_order != IOD_GBEST_LAGGED)
        return fail(IOD_EINVAL, "gbest_order");
    if (!(o.vmax_frac > 0) || !std::isfinite(o.vmax_frac)) return fail(IOD_EINVAL, "vmax_frac must be > 0");
    if (o.use_range && (!(o.sigma_range > 0) || !std::isfinite(o.sigma_range)))
        return fail(IOD_EINVAL, "sigma_range must be > 0 when use_range");
    if (!(o.tol_tau >= 0) || !std::isfinite(o.tol_tau)) return fail(IOD_EINVAL, "tol_tau must be finite and >= 0");
    if (o.tol_tau > 0 && (o.tol_window < 1 || o.tol_window >= iod::kTolHist))
        return fail(IOD_EINVAL, "tol_window must lie in [1, " + std::to_string(iod::kTolHist - 1) + "]");
    if (o.constriction != 0 && o.constriction != 1) return fail(IOD_EINVAL, "constriction must be 0 or 1");
    if (o.init_grid != 0 && o.init_grid != 1) return fail(IOD_EINVAL, "init_grid must be 0 or 1");
    if (o.init_cone != 0 && o.init_cone != 1) return fail(IOD_EINVAL, "init_cone must be 0 or 1");
    if (o.velocity_init != 0 && o.velocity_init != 1) return fail(IOD_EINVAL, "velocity_init must be 0 or 1");
    if (o.dynamics != IOD_CR3BP && o.dynamics != IOD_ER3BP) return fail(IOD_EINVAL, "dynamics");
    if (o.threads_per_particle < 0 || o.threads_per_particle > 2)
        return fail(IOD_EINVAL, "threads_per_particle must be 0, 1 or 2");
    if (o.threads_per_particle == 2 && (o.precision != IOD_FP64 || o.dynamics != IOD_CR3BP))
        return fail(IOD_EINVAL, "two threads per particle run FP64 circular problems only");
    if (o.schedule < IOD_SCHED_AUTO || o.schedule > IOD_SCHED_BALANCED)
        return fail(IOD_EINVAL, "schedule must be IOD_SCHED_AUTO, IOD_SCHED_GRID or IOD_SCHED_BALANCED");
    if (o.dynamics == IOD_ER3BP) {
        if (!(o.ecc >= 0.0 && o.ecc < 1.0) || !std::isfinite(o.f0))
            return fail(IOD_EINVAL, "IOD_ER3BP needs 0 <= ecc < 1 and a finite f0");
        if (o.precision != IOD_FP64) return fail(IOD_EINVAL, "IOD_ER3BP runs in IOD_FP64 only");
    }
    if (o.per_dim_random != 0 && o.per_dim_random != 1) return fail(IOD_EINVAL, "per_dim_random must be 0 or 1");
    if (o.init_cone && (!(o.cone_rho_min >= 0) || !(o.cone_rho_max > o.cone_rho_min) ||
                        !std::isfinite(o.cone_rho_max) || !(o.cone_sigmas > 0) || !std::isfinite(o.cone_sigmas)))
        return fail(IOD_EINVAL, "init_cone needs 0 <= cone_rho_min < cone_rho_max and cone_sigmas > 0");
    if (o.block_size < 0 || o.block_size > iod::max_block_threads() || (o.block_size % 32) != 0)
        return fail(IOD_EINVAL, "block_size must be 0 or a multiple of 32 up to " +
                                    std::to_string(iod::max_block_threads()));
    if (o.shard_total < 0 || o.shard_offset < 0 || (o.shard_total == 0 && o.shard_offset != 0) ||
        (o.shard_total > 0 && o.shard_offset >= o.shard_total))
        return fail(IOD_EINVAL, "shard_offset must lie in [0, shard_total) (both 0 when not sharded)");
    if (o.shard_total > 0 && o.precision != IOD_FP64)
        return fail(IOD_EINVAL, "sharded swarms run in IOD_FP64");
    if (o.shard_total > 0 && o.tol_tau > 0)
        return fail(IOD_EINVAL, "sharded swarms leave Algorithm 2's test to the caller (tol_tau = 0)");
    return IOD_OK;
}

// a shard holds m particles starting at shard_offset: they must fit in the whole swarm
int check_shard(const iod_problem *p, int m)
{
    if (p->opt.shard_total > 0 && (long long)p->opt.shard_offset + m > (long long)p->opt.shard_total)
        return fail(IOD_EINVAL, "shard_offset + swarm_size exceeds shard_total");
    return IOD_OK;
}

int ensure_swarm(iod_problem *p, int m, int trace_needed)
{
    const int grid = std::max((m * p->tpp + p->block - 1) / p->block, sm_count());
    const bool grow_swarm = m > p->m_cap;
    const bool grow_blk = grid > p->grid_cap;
    const bool grow_trace = p->opt.record_trace && trace_needed > p->trace_cap;
    if (grow_swarm || grow_blk || grow_trace) IOD_CUDA(cudaStreamSynchronize(p->stream), "cudaStreamSynchronize");
    if (grow_swarm || m != p->stride) {
        if (grow_swarm) {
            dev_free(p->swarm);
            int rc = dev_alloc(p->swarm, sizeof(double) * 20 * (size_t)m);
            if (rc) {
                p->m_cap = 0;
                return rc;
            }
            p->m_cap = m;
        }
    }
    p->m = m;
    p->stride = m;
    if (grow_blk) {
        dev_free(p->blk);
        int rc = dev_alloc(p->blk, sizeof(BlockBest) * (size_t)grid);
        if (rc) {
            p->grid_cap = 0;
            return rc;
        }
        p->grid_cap = grid;
    }
    if (grow_trace) {
        dev_free(p->trace);
        int rc = dev_alloc(p->trace, (sizeof(double) + sizeof(int)) * (size_t)trace_needed);
        if (rc) {
            p->trace_cap = 0;
            return rc;
        }
        p->trace_cap = trace_needed;
    }
    return IOD_OK;
}

// Threads per particle for a swarm of m: two (the lane-pair kernels) when asked, or
// automatically for FP64 circular swarms small enough.  Measured on GB300 (paper-scale
// problem, per iteration): RK4 1.17x faster up to 4,096 particles, 1.09x at 8,192, 0.72x
// at 16,384, so pairs while they still fit one warp per FP64 sub-partition (4 per SM);
// DOPRI5 1.05x at 1,024 and 4,096 particles, 0.97x at 9,728, 0.56x at 65,536, so pairs
// up to half that size.
int pick_tpp(const iod_problem *p, int m)
{
    const bool can = p->opt.precision == IOD_FP64 && p->opt.dynamics == IOD_CR3BP;
    if (p->opt.threads_per_particle == 2) return 2;
    if (p->opt.threads_per_particle == 1 || !can) return 1;
    const long long cap = 32LL * 4 * sm_count();
    return (p->opt.integrator == IOD_RK4 ? 2LL * m : 4LL * m) <= cap ? 2 : 1;
}

int pick_block(const iod_problem *p, int m)
{
    if (p->opt.block_size > 0) return p->opt.block_size;
    m *= p->tpp;                                     // threads, not particles
    // mixed precision: each block streams the chief's table through shared memory, so
    // larger blocks share every staged chunk among more warps (measured: 32-thread
    // blocks 6.6 ms, 64-256 about 4.4 ms per 65,536-particle iteration)
    if (p->opt.precision == IOD_MIXED) return 128;
    // spread particles evenly over the SMs: the smallest multiple of 32 that keeps the
    // busiest SM within one block of the average, capped at the kernels' limit
    const int sms = sm_count();
    int best = 64;
    double best_eff = -1.0;
    for (int b = 32; b <= iod::max_block_threads(); b += 32) {
        const int grid = (m + b - 1) / b;
        const int rounds = (grid + sms - 1) / sms;
        const double eff = (double)m / ((double)rounds * sms * b);
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best = b;
        }
    }
    return best < 32 ? 32 : best;
}

// Work distribution of the FP64 RK4 iterations (iod_options.schedule).  The balanced form
// needs one thread per particle, RK4 (circular or elliptic problem), at least as many 32-particle
// groups as FP64 sub-partitions and a group's propagation short enough for its hand-off
// wait; automatically it is taken when it lowers the busiest sub-partition's load by more
// than 3%: in group-times, the grid form's busiest sub-partition holds ceil(warps per SM
// / 4) warps, the balanced form's at most G / warps plus one epoch (cuts fall on epoch
// boundaries, each at most half an epoch from its ideal place).
int pick_sched(const iod_problem *p, int m)
{
    if (p->opt.schedule == IOD_SCHED_GRID) return 0;
    const int nsm = sm_count();
    const long long groups = (m + 31) / 32, nw = 4LL * nsm;
    const bool dp = p->opt.integrator == IOD_DOPRI5;
    const bool can = p->tpp == 1 && groups >= nw &&
                     (dp ? p->opt.dynamics == IOD_CR3BP : p->total_steps <= 1000000);
    if (!can) return 0;
    if (p->opt.schedule == IOD_SCHED_BALANCED) return 1;
    if (dp) {
        // adaptive steps: the work per epoch is the chief's, known on the device only; the
        // grid form's busiest sub-partition against the balanced average, 3% margin
        const long long blocks = (m + p->block - 1) / p->block;
        const long long per_sm = (blocks + nsm - 1) / nsm * ((p->block + 31) / 32);
        return (double)((per_sm + 3) / 4) > 1.03 * ((double)groups / (double)nw + 0.05) ? 1 : 0;
    }
    const long long blocks = (m + p->block - 1) / p->block;
    const long long per_sm = (blocks + nsm - 1) / nsm * ((p->block + 31) / 32);
    const long long grid_load = (per_sm + 3) / 4;
    const double T = (double)p->total_steps + iod::kBalancedEpochWeight * p->n_obs;
    const double bal_load = (double)groups / (double)nw + ((double)p->max_interval_steps + iod::kBalancedEpochWeight) / T;
    return (double)grid_load > 1.03 * bal_load ? 1 : 0;
}

// Mixed precision, FP32 iterations: the balanced form (iter_mixed_balanced) cuts
// super-groups of 384 particles between SMs (one 384-thread block per SM, three warps per
// sub-partition).  It needs at least one super-group per SM; automatically it is taken
// when the grid form's 128-thread blocks load the busiest sub-partition with more than
// 1.15 times the balanced form's warp-groups (the grid form runs its busiest
// sub-partitions at 4 warps, faster per warp than 3: measured 3.92 ms grid against 4.46
// ms balanced at exactly 4 warps per sub-partition, 3.87 against 3.65 at 65,536 particles).
int pick_sched_mixed(const iod_problem *p, int m)
{
    if (p->opt.schedule == IOD_SCHED_GRID || p->opt.precision != IOD_MIXED) return 0;
    const long long nsm = sm_count(), sgroups = (m + iod::kMixedBalancedThreads - 1) / iod::kMixedBalancedThreads;
    if (sgroups < nsm || p->total_steps > 1000000) return 0;
    if (p->opt.schedule == IOD_SCHED_BALANCED) return 1;
    const long long grid_load = ((m + 127) / 128 + nsm - 1) / nsm;                 // warps per sub-partition
    const double bal_load = 3.0 * (double)sgroups / (double)nsm;
    return (double)grid_load > 1.15 * bal_load ? 1 : 0;
}

// Warps per SM of the balanced FP64 form: up to three per sub-partition (more warps hide
// more of the FP64 latency), as long as every warp still gets a whole group's work.
int pick_wps(int m, bool dopri5 = false)
{
    const long long groups = (m + 31) / 32, nsm = sm_count();
    if (dopri5) return groups >= 8 * nsm ? 8 : 4;     // its registers allow ten warps per SM
    return groups >= 12 * nsm ? 12 : groups >= 8 * nsm ? 8 : 4;
}

// Balanced forms: the SplitCtl record, plan, flags and hand-off buffers (allocated once;
// the launch counter in SplitCtl only grows, so a flag never matches a stale launch), and
// the plan for the current swarm size and form (kind 0: FP64 warps over 32-particle
// groups; kind 1: mixed-precision blocks over 384-particle super-groups).
int ensure_balanced(iod_problem *p, int kind)
{
    const int nsm = sm_count();
    const int nw = iod::kBalancedMaxWarpsPerSm * nsm;
    const size_t hand_fp64 = (size_t)iod::kDpHandRows * 32 * (size_t)nw,
                 hand_mixed = 13 * (size_t)iod::kMixedBalancedThreads * nsm;
    const size_t ctl = 256, seg = sizeof(iod::SplitSeg) * (size_t)nw, flg = sizeof(unsigned int) * (size_t)nw;
    const size_t seg_off = ctl, flg_off = (seg_off + seg + 255) & ~(size_t)255, hand_off = (flg_off + flg + 255) & ~(size_t)255;
    const size_t bytes = hand_off + sizeof(double) * std::max(hand_fp64, hand_mixed);
    if (!p->split.ptr) {
        int rc = dev_alloc(p->split, bytes);
        if (rc) return rc;
        char *b = (char *)p->split.ptr;
        iod::SplitCtl c{};
        c.stamp = 0;
        c.nw = nw;
        c.seg = (iod::SplitSeg *)(b + seg_off);
        c.flag = (unsigned int *)(b + flg_off);
        c.hand = (double *)(b + hand_off);
        IOD_CUDA(cudaMemsetAsync(b + flg_off, 0, flg, p->stream), "cudaMemsetAsync");
        IOD_CUDA(cudaMemcpyAsync(b, &c, sizeof c, cudaMemcpyHostToDevice, p->stream), "cudaMemcpyAsync");
        IOD_CUDA(cudaStreamSynchronize(p->stream), "cudaStreamSynchronize");
        p->split_m = -1;
    }
    int nw_run, gsize;
    if (kind == 0) {
        p->wps = pick_wps(p->m, p->opt.integrator == IOD_DOPRI5);
        nw_run = p->wps * nsm;
        gsize = 32;
    } else {
        nw_run = nsm;
        gsize = iod::kMixedBalancedThreads;
    }
    if (p->split_m != p->m || p->split_nw != nw_run || p->split_gs != gsize) {
        cudaError_t e = iod::launch_split_plan(p->params(), nw_run, gsize, p->stream);
        if (e != cudaSuccess) return cuda_fail(e, "plan kernel launch");
        p->split_m = p->m;
        p->split_nw = nw_run;
        p->split_gs = gsize;
    }
    return IOD_OK;
}

int queue_iters(iod_problem *p, int iters)
{
    const bool mixed = p->opt.precision == IOD_MIXED && p->phase == 0;
    const bool balanced = mixed ? p->sched_mixed == 1 : p->sched == 1;
    if (balanced && iters > 0) {
        int rc = ensure_balanced(p, mixed ? 1 : 0);
        if (rc) return rc;
    }
    const KParams P = p->params();
    for (int n = 0; n < iters; ++n) {
        cudaError_t e;
        int used = IOD_SCHED_GRID;
        if (mixed && p->sched_mixed == 1) {
            e = iod::launch_iter_mixed_balanced(P, p->opt.gbest_order, sm_count(), p->stream);
            used = IOD_SCHED_BALANCED;
            if (e == cudaErrorCooperativeLaunchTooLarge && p->opt.schedule == IOD_SCHED_AUTO) {
                (void)cudaGetLastError();
                p->sched_mixed = 0;
                e = iod::launch_iter_mixed(P, p->block, p->opt.gbest_order, p->stream);
                used = IOD_SCHED_GRID;
            }
        } else if (mixed) {
            e = iod::launch_iter_mixed(P, p->block, p->opt.gbest_order, p->stream);
        } else if (p->sched == 1) {
            e = iod::launch_iter_balanced(P, p->opt.gbest_order, sm_count(), p->wps, p->stream);
            used = IOD_SCHED_BALANCED;
            if (e == cudaErrorCooperativeLaunchTooLarge && p->opt.schedule == IOD_SCHED_AUTO) {
                // the GPU cannot hold one block per SM now: the automatic choice falls back
                // to the grid form (an explicit IOD_SCHED_BALANCED fails instead)
                (void)cudaGetLastError();
                p->sched = 0;
                e = iod::launch_iter(P, p->block, p->opt.gbest_order, p->stream);
                used = IOD_SCHED_GRID;
            }
        } else {
            e = iod::launch_iter(P, p->block, p->opt.gbest_order, p->stream);
        }
        if (e != cudaSuccess) return cuda_fail(e, "iteration kernel launch");
        p->last_sched = used;
        ++p->iters_done;
    }
    return IOD_OK;
}

// Mixed precision: re-evaluate every personal best in FP64 and enter the FP64 phase.
int enter_fp64_phase(iod_problem *p)
{
    if (p->opt.precision != IOD_MIXED || p->phase == 1) return IOD_OK;
    cudaError_t e = iod::launch_rescore(p->params(), p->block, p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "rescore kernel launch");
    p->phase = 1;
    return IOD_OK;
}

}  // namespace

extern "C" {

int iod_options_default(iod_options *o)
{
    if (!o) return fail(IOD_EINVAL, "options pointer is NULL");
    std::memset(o, 0, sizeof *o);
    o->integrator = IOD_RK4;
    o->dt = 1e-3;
    o->rtol = 1e-12;
    o->atol = 1e-12;
    o->h0 = 1e-3;
    o->max_steps = 10000000LL;
    o->precision = IOD_FP64;
    o->cost_form = IOD_COST_CHI2;
    o->gbest_order = IOD_GBEST_SYNC;
    o->vmax_frac = 1.0;
    o->use_range = 0;
    o->sigma_range = 0.0;
    o->record_trace = 1;
    o->block_size = 0;
    o->fp64_last_iters = 50;
    o->moon_fp64_radius = 0.02;
    o->tol_tau = 0.0;
    o->tol_window = 10;
    o->constriction = 0;
    o->init_grid = 0;
    o->init_cone = 0;
    o->cone_rho_min = 0.0;
    o->cone_rho_max = 0.0;
    o->cone_sigmas = 3.0;
    o->velocity_init = 0;
    o->per_dim_random = 0;
    o->threads_per_particle = 0;
    o->schedule = IOD_SCHED_AUTO;
    o->refine_iters = 0;
    o->shard_offset = 0;
    o->shard_total = 0;
    o->refine_gate = 0.0;
    o->dynamics = IOD_CR3BP;
    o->ecc = 0.0;
    o->f0 = 0.0;
    return IOD_OK;
}

int iod_create_ranged(double mu, const double chief_state[6], int n_obs, const double *obs_times,
                      const double *obs_angles, const double *obs_ranges, const double sigma[2],
                      const double bounds[12], const iod_options *opt, iod_problem **out)
{
    const iod::NvtxRange nvtx_range("iod_create");
    if (!out) return fail(IOD_EINVAL, "out is NULL");
    *out = nullptr;
    iod_options o;
    if (opt)
        o = *opt;
    else
        iod_options_default(&o);
    int rc = validate_options(o);
    if (rc) return rc;
    if (o.refine_iters != 0)
        return fail(IOD_EINVAL, "refine_iters applies to batches; single problems call iod_refine");
    if (o.refine_gate != 0.0) return fail(IOD_EINVAL, "refine_gate applies to batches");
    if (!(mu > 0 && mu < 0.5)) return fail(IOD_EINVAL, "mu must lie in (0, 0.5)");
    if (n_obs < 1) return fail(IOD_EINVAL, "n_obs must be >= 1");
    if (!chief_state || !obs_times || !obs_angles || !sigma || !bounds)
        return fail(IOD_EINVAL, "NULL input array");
    if (o.use_range && !obs_ranges) return fail(IOD_EINVAL, "use_range needs obs_ranges");
    if (!finite_all(chief_state, 6)) return fail(IOD_EINVAL, "chief_state not finite");
    if (!finite_all(obs_times, (size_t)n_obs)) return fail(IOD_EINVAL, "obs_times not finite");
    if (!finite_all(obs_angles, 2 * (size_t)n_obs)) return fail(IOD_EINVAL, "obs_angles not finite");
    if (o.use_range && !finite_all(obs_ranges, (size_t)n_obs)) return fail(IOD_EINVAL, "obs_ranges not finite");
    if (!(obs_times[0] >= 0)) return fail(IOD_EINVAL, "obs_times must be >= 0");
    for (int k = 1; k < n_obs; ++k)
        if (!(obs_times[k] > obs_times[k - 1])) return fail(IOD_EINVAL, "obs_times must be strictly increasing");
    if (!(sigma[0] > 0) || !(sigma[1] > 0) || !finite_all(sigma, 2)) return fail(IOD_EINVAL, "sigma must be finite and > 0");
    if (o.init_cone && obs_times[0] != 0.0) return fail(IOD_EINVAL, "init_cone needs the first observation at t = 0");
    if (!finite_all(bounds, 12)) return fail(IOD_EINVAL, "bounds not finite");
    for (int d = 0; d < 6; ++d)
        if (!(bounds[d] < bounds[6 + d])) return fail(IOD_EINVAL, "bounds: lo must be < hi");
    // the mixed kernels also stage one float per chunk of steps; bound the step count by
    // the interval rule (at most span/dt + 1 steps per interval)
    const double span_steps = obs_times[n_obs - 1] / o.dt + 2.0 * n_obs;
    const size_t smem_fp64 = iod::swarm_smem_bytes(n_obs, o.integrator),
                 smem_mix = o.precision == IOD_MIXED
                                ? iod::mixed_smem_bytes(n_obs, span_steps < 4e9 ? (long long)span_steps : 4000000000LL)
                                : 0;
    const size_t smem = (smem_fp64 > smem_mix ? smem_fp64 : smem_mix) + 1024;
    const int smax = max_smem_optin();
    if (smax > 0 && smem > (size_t)smax)
        return fail(IOD_EINVAL, "n_obs too large for one block's shared-memory observation table");

    iod_problem *p = new (std::nothrow) iod_problem();
    if (!p) return fail(IOD_ENOMEM, "host allocation");
    p->opt = o;
    p->mu = mu;
    p->n_obs = n_obs;
    std::memcpy(p->chief, chief_state, sizeof p->chief);
    std::memcpy(p->sigma, sigma, sizeof p->sigma);
    std::memcpy(p->lo, bounds, sizeof p->lo);
    std::memcpy(p->hi, bounds + 6, sizeof p->hi);
    if (o.init_cone)
        iod::cone_frame(obs_angles[0], obs_angles[1], sigma[0], sigma[1], o.cone_sigmas, o.cone_rho_min,
                        o.cone_rho_max, p->cone);
    cudaGetDevice(&p->device);

    auto bail = [&](int code) {
        delete p;
        return code;
    };
    if ((rc = dev_alloc(p->obs, (8 * sizeof(double) + sizeof(int)) * (size_t)n_obs))) return bail(rc);
    if ((rc = dev_alloc(p->misc, iod::kMiscBytes))) return bail(rc);
    std::vector<double> host(8 * (size_t)n_obs, 0.0);
    for (int k = 0; k < n_obs; ++k) {
        // the integrators' independent variable: time, or elapsed true anomaly (ER3BP)
        host[k] = o.dynamics == IOD_ER3BP ? iod::er3bp_true_anomaly(o.ecc, o.f0, obs_times[k]) - o.f0
                                          : obs_times[k];
        host[n_obs + k] = obs_angles[2 * k];
        host[2 * n_obs + k] = obs_angles[2 * k + 1];
        host[3 * n_obs + k] = o.use_range ? obs_ranges[k] : 0.0;
    }
    cudaError_t e = cudaMemcpy(p->obs.ptr, host.data(), sizeof(double) * 4 * n_obs, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_chief(), chief_state, sizeof(double) * 6, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMemcpy (create)"));
    double *chief_cs = nullptr;
    if (o.precision == IOD_MIXED) {
        // the interval rule takes at most span/dt + 1 steps per interval
        p->mix_cap = (long long)std::ceil(obs_times[n_obs - 1] / o.dt) + n_obs + 1;
        if ((rc = dev_alloc(p->mix, p->mix_bytes()))) return bail(rc);
        chief_cs = (double *)((char *)p->mix.ptr + p->mix_cs_offset());
    }
    const KParams P = p->params();
    e = iod::launch_setup(P, o.vmax_frac, sigma[0], sigma[1], o.sigma_range, p->d_chief(), p->d_rc(),
                          p->d_ns(), p->d_h(), p->d_cst(), p->d_gb(), nullptr, chief_cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess) return bail(cuda_fail(e, "set-up kernel"));
    GBest gb;
    e = cudaMemcpy(&gb, p->d_gb(), sizeof gb, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMemcpy (create status)"));
    if (gb.status & iod::kStatusChiefDiverged)
        return bail(fail(IOD_EDIVERGED, "chief propagation produced non-finite states"));
    if (o.integrator == IOD_RK4) {
        std::vector<int> ns(n_obs);
        e = cudaMemcpy(ns.data(), p->d_ns(), sizeof(int) * n_obs, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMemcpy (interval table)"));
        for (int k = 0; k < n_obs; ++k) {
            p->total_steps += ns[k];
            p->max_interval_steps = std::max(p->max_interval_steps, ns[k]);
        }
    }
    if (o.precision == IOD_MIXED) {
        if (p->total_steps > p->mix_cap) return bail(fail(IOD_EINVAL, "interval table exceeds its step bound"));
        const KParams Pm = p->params();
        e = iod::launch_setup_mixed(Pm, (iod::mix::Step *)p->mix.ptr, chief_cs,
                                    (iod::mix::ObsDir *)((char *)p->mix.ptr + p->mix_dir_offset()),
                                    (float *)((char *)p->mix.ptr + p->mix_ct_offset()), nullptr);
        if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
        if (e != cudaSuccess) return bail(cuda_fail(e, "mixed-precision set-up kernel"));
    }
    *out = p;
    return IOD_OK;
}

int iod_create(double mu, const double chief_state[6], int n_obs, const double *obs_times,
               const double *obs_angles, const double sigma[2], const double bounds[12],
               const iod_options *opt, iod_problem **out)
{
    if (opt && opt->use_range) return fail(IOD_EINVAL, "use_range needs iod_create_ranged");
    return iod_create_ranged(mu, chief_state, n_obs, obs_times, obs_angles, nullptr, sigma, bounds,
                             opt, out);
}

int iod_set_stream(iod_problem *p, void *cuda_stream)
{
    if (!p) return fail(IOD_EINVAL, "problem is NULL");
    if (p->stream != (cudaStream_t)cuda_stream) {
        // order the new stream after everything already queued on the old one
        IOD_CUDA(cudaStreamSynchronize(p->stream), "cudaStreamSynchronize");
    }
    p->stream = (cudaStream_t)cuda_stream;
    return IOD_OK;
}

int iod_set_allocator(void *(*alloc)(size_t, void *), void (*release)(void *, void *), void *ctx)
{
    if ((alloc == nullptr) != (release == nullptr)) return fail(IOD_EINVAL, "alloc and release go together");
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc.alloc = alloc;
    g_alloc.release = release;
    g_alloc.ctx = ctx;
    return IOD_OK;
}

int iod_run(iod_problem *p, int swarm_size, int iters, double w, double c1, double c2, uint64_t seed)
{
    const iod::NvtxRange nvtx_range("iod_run");
    if (!p) return fail(IOD_EINVAL, "problem is NULL");
    if (swarm_size < 1) return fail(IOD_EINVAL, "swarm_size must be >= 1");
    if (iters < 0) return fail(IOD_EINVAL, "iters must be >= 0");
    if (!std::isfinite(w) || !std::isfinite(c1) || !std::isfinite(c2))
        return fail(IOD_EINVAL, "coefficients must be finite");
    if (p->opt.constriction && !(c1 + c2 > 4.0))
        return fail(IOD_EINVAL, "the constriction factor needs c1 + c2 > 4");
    if (int rs = check_shard(p, swarm_size)) return rs;
    p->tpp = pick_tpp(p, swarm_size);
    p->block = pick_block(p, swarm_size);
    p->sched = pick_sched(p, swarm_size);
    p->sched_mixed = pick_sched_mixed(p, swarm_size);
    int rc = ensure_swarm(p, swarm_size, iters + 1);
    if (rc) return rc;
    p->w = w;
    p->c1 = c1;
    p->c2 = c2;
    p->seed = seed;
    p->iters_done = 0;
    p->started = false;
    IOD_CUDA(cudaMemsetAsync(p->d_gb(), 0, sizeof(GBest), p->stream), "cudaMemsetAsync");
    p->phase = 0;
    const bool mixed = p->opt.precision == IOD_MIXED;
    if (!mixed && p->sched == 1 && (rc = ensure_balanced(p, 0))) return rc;
    const KParams P = p->params();
    cudaError_t e;
    p->last_sched = IOD_SCHED_GRID;
    if (mixed) {
        e = iod::launch_init_mixed(P, p->block, p->stream);
    } else if (p->sched == 1) {
        e = iod::launch_iter_balanced(P, 2, sm_count(), p->wps, p->stream);
        p->last_sched = IOD_SCHED_BALANCED;
        if (e == cudaErrorCooperativeLaunchTooLarge && p->opt.schedule == IOD_SCHED_AUTO) {
            (void)cudaGetLastError();
            p->sched = 0;
            p->last_sched = IOD_SCHED_GRID;
            e = iod::launch_init(P, p->block, p->stream);
        }
    } else {
        e = iod::launch_init(P, p->block, p->stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "initialisation kernel launch");
    p->started = true;
    if (!mixed || iters == 0) return queue_iters(p, iters);
    // FP32 exploration, FP64 re-evaluation of the bests, FP64 refinement
    const int last = p->opt.fp64_last_iters < iters ? p->opt.fp64_last_iters : iters;
    if ((rc = queue_iters(p, iters - last))) return rc;
    if ((rc = enter_fp64_phase(p))) return rc;
    return queue_iters(p, last);
}

int iod_continue(iod_problem *p, int iters)
{
    const iod::NvtxRange nvtx_range("iod_continue");
    if (!p) return fail(IOD_EINVAL, "problem is NULL");
    if (!p->started) return fail(IOD_ESTATE, "iod_continue before iod_run or iod_swarm_set");
    if (iters < 0) return fail(IOD_EINVAL, "iters must be >= 0");
    const int need = p->iters_done + iters + 1;
    if (p->opt.record_trace && need > p->trace_cap) {
        // keep the recorded part of the trace while growing it
        IOD_CUDA(cudaStreamSynchronize(p->stream), "cudaStreamSynchronize");
        std::vector<double> tj(p->trace_cap);
        std::vector<int> ti(p->trace_cap);
        if (p->trace_cap) {
            IOD_CUDA(cudaMemcpy(tj.data(), p->trace.ptr, sizeof(double) * p->trace_cap, cudaMemcpyDeviceToHost), "cudaMemcpy");
            IOD_CUDA(cudaMemcpy(ti.data(), (double *)p->trace.ptr + p->trace_cap, sizeof(int) * p->trace_cap,
                                cudaMemcpyDeviceToHost), "cudaMemcpy");
        }
        const int old = p->trace_cap;
        const int cap = need > 2 * old ? need : 2 * old;
        dev_free(p->trace);
        p->trace_cap = 0;
        int rc = dev_alloc(p->trace, (sizeof(double) + sizeof(int)) * (size_t)cap);
        if (rc) return rc;
        p->trace_cap = cap;
        if (old) {
            IOD_CUDA(cudaMemcpy(p->trace.ptr, tj.data(), sizeof(double) * old, cudaMemcpyHostToDevice), "cudaMemcpy");
            IOD_CUDA(cudaMemcpy((double *)p->trace.ptr + cap, ti.data(), sizeof(int) * old, cudaMemcpyHostToDevice),
                     "cudaMemcpy");
        }
    }
    return queue_iters(p, iters);
}

int iod_result(iod_problem *p, iod_result_t *out)
{
    const iod::NvtxRange nvtx_range("iod_result");
    if (!p || !out) return fail(IOD_EINVAL, "NULL argument");
    if (!p->started) return fail(IOD_ESTATE, "iod_result before iod_run");
    IOD_CUDA(cudaStreamSynchronize(p->stream), "cudaStreamSynchronize");
    GBest gb;
    // the result fields sit before Algorithm 2's cost record: read only those 96 bytes
    IOD_CUDA(cudaMemcpy(&gb, p->d_gb(), offsetof(GBest, hist), cudaMemcpyDeviceToHost), "cudaMemcpy (result)");
    std::memcpy(out->state, gb.g, sizeof out->state);
    out->cost = gb.gJ;
    std::memcpy(out->pso_state, gb.g, sizeof out->pso_state);     // single problems: no refinement
    out->pso_cost = gb.gJ;
    out->refine_iters = 0;
    out->fallback = 0;
    out->gbest_index = gb.gidx;
    out->iters_done = gb.iter;
    out->rk_steps = (long long)gb.steps;
    out->fp64_steps = (long long)gb.steps64;
    out->schedule = p->last_sched;
    if (out->gcost_trace && out->gidx_trace && out->trace_capacity > 0 && p->opt.record_trace && p->trace.ptr) {
        int n = gb.iter + 1;
        if (n > p->trace_cap) n = p->trace_cap;
        if (n > out->trace_capacity) n = out->trace_capacity;
        if (n > 0) {
            IOD_CUDA(cudaMemcpy(out->gcost_trace, p->trace.ptr, sizeof(double) * n, cudaMemcpyDeviceToHost), "cudaMemcpy");
            IOD_CUDA(cudaMemcpy(out->gidx_trace, (double *)p->trace.ptr + p->trace_cap, sizeof(int) * n,
                                cudaMemcpyDeviceToHost), "cudaMemcpy");
        }
    }
    if (gb.status & iod::kStatusCheck)
        return fail(IOD_ECUDA, "an argument check of the IOD_CHECK build failed (launch or table inconsistent)");
    if (gb.status & iod::kStatusCopyCheck)
        return fail(IOD_ECUDA, "a chief-table copy failed its alignment or shared-memory check (not issued)");
    if (gb.status & (iod::kStatusCopyTimeout | iod::kStatusHandoffTimeout))
        return fail(IOD_ETIMEOUT, (gb.status & iod::kStatusHandoffTimeout)
                                      ? "a hand-off wait of the balanced schedule gave up"
                                      : "a chief-table copy wait gave up");
    return IOD_OK;
}

int iod_swarm_get(iod_problem *p, double *x, double *v, double *pbest, double *pbest_cost,
                  double *cost, double g[6], double *g_cost, int *g_index, int *iter)
{
    if (!p) return fail(IOD_EINVAL, "problem is NULL");
    if (!p->started) return fail(IOD_ESTATE, "no swarm yet");
    IOD_CUDA(cudaStreamSynchronize(p->stream), "cudaStreamSynchronize");
    const size_t M = (size_t)p->m, S = (size_t)p->stride;
    const double *sw = (const double *)p->swarm.ptr;
    struct { double *dst; size_t off; size_t rows; } parts[] = {
        {x, 0, 6}, {v, 6 * S, 6}, {pbest, 12 * S, 6}, {pbest_cost, 18 * S, 1}, {cost, 19 * S, 1}};
    for (auto &pt : parts) {
        if (!pt.dst) continue;
        for (size_t r = 0; r < pt.rows; ++r)
            IOD_CUDA(cudaMemcpy(pt.dst + r * M, sw + pt.off + r * S, sizeof(double) * M, cudaMemcpyDeviceToHost),
                     "cudaMemcpy (swarm)");
    }
    GBest gb;
    IOD_CUDA(cudaMemcpy(&gb, p->d_gb(), sizeof gb, cudaMemcpyDeviceToHost), "cudaMemcpy (gbest)");
    if (g) std::memcpy(g, gb.g, sizeof(double) * 6);
    if (g_cost) *g_cost = gb.gJ;
    if (g_index) *g_index = gb.gidx;
    if (iter) *iter = gb.iter;
    return IOD_OK;
}

int iod_swarm_set(iod_problem *p, int m, const double *x, const double *v, const double *pbest,
                  const double *pbest_cost, const double g[6], double g_cost, int g_index, int iter,
                  double w, double c1, double c2, uint64_t seed)
{
    if (!p) return fail(IOD_EINVAL, "problem is NULL");
    if (m < 1 || !x || !v || !pbest || !pbest_cost || !g) return fail(IOD_EINVAL, "bad swarm arguments");
    if (iter < 0 || g_index < 0 || g_index >= m) return fail(IOD_EINVAL, "bad iteration or index");
    if (!std::isfinite(w) || !std::isfinite(c1) || !std::isfinite(c2))
        return fail(IOD_EINVAL, "coefficients must be finite");
    if (p->opt.constriction && !(c1 + c2 > 4.0))
        return fail(IOD_EINVAL, "the constriction factor needs c1 + c2 > 4");
    if (int rs = check_shard(p, m)) return rs;
    p->tpp = pick_tpp(p, m);
    p->block = pick_block(p, m);
    p->sched = pick_sched(p, m);
    p->sched_mixed = pick_sched_mixed(p, m);
    int rc = ensure_swarm(p, m, iter + 2);
    if (rc) return rc;
    IOD_CUDA(cudaStreamSynchronize(p->stream), "cudaStreamSynchronize");
    const size_t M = (size_t)m, S = (size_t)p->stride;
    double *sw = (double *)p->swarm.ptr;
    const double *src[] = {x, v, pbest};
    for (int a = 0; a < 3; ++a)
        IOD_CUDA(cudaMemcpy(sw + 6 * S * a, src[a], sizeof(double) * 6 * M, cudaMemcpyHostToDevice), "cudaMemcpy");
    IOD_CUDA(cudaMemcpy(sw + 18 * S, pbest_cost, sizeof(double) * M, cudaMemcpyHostToDevice), "cudaMemcpy");
    GBest gb;
    std::memset(&gb, 0, sizeof gb);
    std::memcpy(gb.g, g, sizeof gb.g);
    gb.gJ = g_cost;
    gb.gidx = g_index;
    gb.iter = iter;
    IOD_CUDA(cudaMemcpy(p->d_gb(), &gb, sizeof gb, cudaMemcpyHostToDevice), "cudaMemcpy");
    p->w = w;
    p->c1 = c1;
    p->c2 = c2;
    p->seed = seed;
    p->iters_done = iter;
    p->started = true;
    return IOD_OK;
}

int iod_gbest_get(iod_problem *p, double g[6], double *g_cost, int *g_index, int *iter)
{
    if (!p) return fail(IOD_EINVAL, "problem is NULL");
    if (!p->started) return fail(IOD_ESTATE, "iod_gbest_get before iod_run or iod_swarm_set");
    GBest gb;
    IOD_CUDA(cudaMemcpyAsync(&gb, p->d_gb(), sizeof gb, cudaMemcpyDeviceToHost, p->stream), "cudaMemcpyAsync");
    IOD_CUDA(cudaStreamSynchronize(p->stream), "cudaStreamSynchronize");
    if (g) std::memcpy(g, gb.g, sizeof gb.g);
    if (g_cost) *g_cost = gb.gJ;
    if (g_index) *g_index = gb.gidx;
    if (iter) *iter = gb.iter;
    return IOD_OK;
}

int iod_gbest_set(iod_problem *p, const double g[6], double g_cost, int g_index)
{
    if (!p || !g) return fail(IOD_EINVAL, "problem or state is NULL");
    if (!p->started) return fail(IOD_ESTATE, "iod_gbest_set before iod_run or iod_swarm_set");
    for (int d = 0; d < 6; ++d)
        if (!std::isfinite(g[d])) return fail(IOD_EINVAL, "the global best state must be finite");
    if (std::isnan(g_cost) || g_index < 0) return fail(IOD_EINVAL, "the global best needs a cost and an index >= 0");
    const cudaError_t e = iod::launch_set_gbest(p->d_gb(), g, g_cost, g_index, p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "global best kernel launch");
    return IOD_OK;
}

namespace {
struct SnapHeader {
    char magic[8];
    int version, m, iter, integrator, n_obs, gidx, phase, flags;
    double w, c1, c2, gJ, g[6];
    uint64_t seed;
    unsigned long long steps;
    double hist[iod::kTolHist];   // Algorithm 2's record of past global best costs
};
constexpr int kSnapVersion = 2;
}  // namespace

int iod_snapshot(iod_problem *p, void *buf, size_t *len)
{
    if (!p || !len) return fail(IOD_EINVAL, "NULL argument");
    if (!p->started) return fail(IOD_ESTATE, "no swarm to snapshot");
    const size_t M = (size_t)p->m;
    const size_t need = sizeof(SnapHeader) + sizeof(double) * 20 * M;
    if (!buf) {
        *len = need;
        return IOD_OK;
    }
    if (*len < need) return fail(IOD_EINVAL, "snapshot buffer too small");
    IOD_CUDA(cudaStreamSynchronize(p->stream), "cudaStreamSynchronize");
    GBest gb;
    IOD_CUDA(cudaMemcpy(&gb, p->d_gb(), sizeof gb, cudaMemcpyDeviceToHost), "cudaMemcpy");
    SnapHeader h;
    std::memset(&h, 0, sizeof h);
    std::memcpy(h.magic, "IODSNAP1", 8);
    h.version = kSnapVersion;
    h.m = p->m;
    h.iter = gb.iter;
    h.integrator = p->opt.integrator;
    h.n_obs = p->n_obs;
    h.gidx = gb.gidx;
    h.phase = p->phase;
    h.w = p->w;
    h.c1 = p->c1;
    h.c2 = p->c2;
    h.gJ = gb.gJ;
    std::memcpy(h.g, gb.g, sizeof h.g);
    h.seed = p->seed;
    h.steps = gb.steps;
    h.flags = gb.flags;
    std::memcpy(h.hist, gb.hist, sizeof h.hist);
    std::memcpy(buf, &h, sizeof h);
    double *body = (double *)((char *)buf + sizeof h);
    const size_t S = (size_t)p->stride;
    for (int r = 0; r < 20; ++r)
        IOD_CUDA(cudaMemcpy(body + r * M, (double *)p->swarm.ptr + r * S, sizeof(double) * M, cudaMemcpyDeviceToHost),
                 "cudaMemcpy (snapshot)");
    *len = need;
    return IOD_OK;
}

int iod_restore(iod_problem *p, const void *buf, size_t len)
{
    if (!p || !buf || len < sizeof(SnapHeader)) return fail(IOD_EINVAL, "bad snapshot");
    SnapHeader h;
    std::memcpy(&h, buf, sizeof h);
    if (std::memcmp(h.magic, "IODSNAP1", 8) != 0 || h.version != kSnapVersion) return fail(IOD_EINVAL, "not a snapshot");
    if (h.n_obs != p->n_obs || h.integrator != p->opt.integrator) return fail(IOD_EINVAL, "snapshot of another problem");
    if (h.m < 1 || len < sizeof h + sizeof(double) * 20 * (size_t)h.m) return fail(IOD_EINVAL, "truncated snapshot");
    p->tpp = pick_tpp(p, h.m);
    p->block = pick_block(p, h.m);
    p->sched = pick_sched(p, h.m);
    p->sched_mixed = pick_sched_mixed(p, h.m);
    int rc = ensure_swarm(p, h.m, h.iter + 2);
    if (rc) return rc;
    IOD_CUDA(cudaStreamSynchronize(p->stream), "cudaStreamSynchronize");
    const double *body = (const double *)((const char *)buf + sizeof h);
    const size_t M = (size_t)h.m, S = (size_t)p->stride;
    for (int r = 0; r < 20; ++r)
        IOD_CUDA(cudaMemcpy((double *)p->swarm.ptr + r * S, body + r * M, sizeof(double) * M, cudaMemcpyHostToDevice),
                 "cudaMemcpy (restore)");
    GBest gb;
    std::memset(&gb, 0, sizeof gb);
    std::memcpy(gb.g, h.g, sizeof gb.g);
    gb.gJ = h.gJ;
    gb.gidx = h.gidx;
    gb.iter = h.iter;
    gb.steps = h.steps;
    gb.flags = h.flags;
    std::memcpy(gb.hist, h.hist, sizeof gb.hist);
    IOD_CUDA(cudaMemcpy(p->d_gb(), &gb, sizeof gb, cudaMemcpyHostToDevice), "cudaMemcpy");
    p->w = h.w;
    p->c1 = h.c1;
    p->c2 = h.c2;
    p->seed = h.seed;
    p->iters_done = h.iter;
    p->phase = h.phase;
    p->started = true;
    return IOD_OK;
}

void iod_destroy(iod_problem *p) { delete p; }

const char *iod_strerror(int code)
{
    switch (code) {
    case IOD_OK: return "ok";
    case IOD_EINVAL: return "invalid argument";
    case IOD_ENOMEM: return "out of device memory";
    case IOD_ECUDA: return "CUDA error";
    case IOD_ETIMEOUT: return "device wait timed out";
    case IOD_EBUSY: return "busy";
    case IOD_ECANCELLED: return "cancelled";
    case IOD_ESTATE: return "call out of order";
    case IOD_EDIVERGED: return "propagation diverged";
    default: return "unknown status";
    }
}

const char *iod_last_error(void) { return g_last_error.c_str(); }

int iod_selftest_wait(double limit_s, int set_flag, int *timed_out, double *waited_s)
{
    if (!timed_out || !waited_s || !(limit_s > 0.0 && limit_s <= 10.0))
        return fail(IOD_EINVAL, "iod_selftest_wait needs 0 < limit_s <= 10 and two output pointers");
    struct Probe {
        unsigned int flag;
        int timed_out;
        unsigned long long waited_ns;
    };
    Probe *d = nullptr;
    IOD_CUDA(cudaMalloc(&d, sizeof(Probe)), "cudaMalloc");
    Probe h{};
    h.flag = set_flag ? 1u : 0u;
    h.timed_out = -1;
    cudaError_t e = cudaMemcpy(d, &h, sizeof h, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = iod::launch_wait_probe(&d->flag, 1u, (unsigned long long)(limit_s * 1e9), &d->timed_out, &d->waited_ns,
                                   nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof h, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "wait probe");
    *timed_out = h.timed_out;
    *waited_s = (double)h.waited_ns * 1e-9;
    return IOD_OK;
}

int iod_selftest_fp64_issue(int warps, int lanes, int n, double *cycles_per_fma)
{
    if (warps < 1 || warps > 32 || lanes < 1 || lanes > 32 || n < 1 || n > 1000000 || !cycles_per_fma)
        return fail(IOD_EINVAL, "iod_selftest_fp64_issue needs 1 <= warps, lanes <= 32, 1 <= n <= 1e6 and an output");
    long long *d_cyc = nullptr;
    double *d_sink = nullptr;
    IOD_CUDA(cudaMalloc(&d_cyc, sizeof(long long) * 32), "cudaMalloc");
    cudaError_t e = cudaMalloc(&d_sink, sizeof(double) * 32 * 32);
    long long h[32] = {0};
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // the first launch warms up
        e = iod::launch_fp64_issue_probe(warps, lanes, n, d_cyc, d_sink, nullptr);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    if (e == cudaSuccess) e = cudaMemcpy(h, d_cyc, sizeof(long long) * (size_t)warps, cudaMemcpyDeviceToHost);
    cudaFree(d_cyc);
    cudaFree(d_sink);
    if (e != cudaSuccess) return cuda_fail(e, "FP64 issue probe");
    long long mx = 0;
    for (int w = 0; w < warps; ++w) mx = h[w] > mx ? h[w] : mx;
    *cycles_per_fma = (double)mx / (double)n;
    return IOD_OK;
}

int iod_eval(iod_problem *p, const double *x, int m, double *J)
{
    const iod::NvtxRange nvtx_range("iod_eval");
    if (!p || !x || !J || m < 1) return fail(IOD_EINVAL, "bad eval arguments");
    KParams P = p->params();
    cudaError_t e = p->opt.precision == IOD_MIXED ? iod::launch_eval_mixed(P, x, m, J, 64, p->stream)
                                                  : iod::launch_eval(P, x, m, J, 64, p->stream);
    return e == cudaSuccess ? IOD_OK : cuda_fail(e, "eval kernel launch");
}

int iod_propagate(iod_problem *p, const double *x0, int m, double *out)
{
    const iod::NvtxRange nvtx_range("iod_propagate");
    if (!p || !x0 || !out || m < 1) return fail(IOD_EINVAL, "bad propagate arguments");
    KParams P = p->params();
    cudaError_t e = p->opt.precision == IOD_MIXED ? iod::launch_propagate_mixed(P, x0, m, out, 64, p->stream)
                                                  : iod::launch_propagate(P, x0, m, out, 64, p->stream);
    return e == cudaSuccess ? IOD_OK : cuda_fail(e, "propagate kernel launch");
}

int iod_refine(iod_problem *p, const double x0[6], int max_iters, int form, double x_out[6],
               double *cost_out, int *iters_out)
{
    const iod::NvtxRange nvtx_range("iod_refine");
    if (!p || !x0 || !x_out) return fail(IOD_EINVAL, "NULL argument");
    if (p->opt.integrator != IOD_RK4) return fail(IOD_EINVAL, "refinement uses the RK4 integrator");
    if (max_iters < 0 || (form != 0 && form != 1)) return fail(IOD_EINVAL, "bad refinement settings");
    if (!finite_all(x0, 6)) return fail(IOD_EINVAL, "x0 not finite");
    const int n = form == 0 ? 2 * p->n_obs : p->n_obs;
    const size_t need = sizeof(double) * (iod::kLmVecs * (size_t)n + iod::kLmTail + 6 + 16);
    if (p->lm.bytes < need) {
        IOD_CUDA(cudaStreamSynchronize(p->stream), "cudaStreamSynchronize");
        dev_free(p->lm);
        int rc = dev_alloc(p->lm, need);
        if (rc) return rc;
    }
    double *R = (double *)p->lm.ptr, *dx0 = R + iod::kLmVecs * (size_t)n + iod::kLmTail, *dout = dx0 + 6;
    IOD_CUDA(cudaMemcpyAsync(dx0, x0, 6 * sizeof(double), cudaMemcpyHostToDevice, p->stream), "cudaMemcpyAsync");
    cudaError_t e = iod::launch_lm(p->params(), dx0, max_iters, form, p->sigma[0], p->sigma[1], R, dout, p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "refinement kernel launch");
    double out[9];
    IOD_CUDA(cudaMemcpyAsync(out, dout, sizeof out, cudaMemcpyDeviceToHost, p->stream), "cudaMemcpyAsync");
    IOD_CUDA(cudaStreamSynchronize(p->stream), "cudaStreamSynchronize");
    std::memcpy(x_out, out, 6 * sizeof(double));
    if (cost_out) *cost_out = out[6];
    if (iters_out) *iters_out = (int)out[7];
    return out[8] == 2.0 ? fail(IOD_EDIVERGED, "refinement start state is not evaluable") : IOD_OK;
}

int iod_chief_positions(iod_problem *p, double *rc)
{
    if (!p || !rc) return fail(IOD_EINVAL, "NULL argument");
    IOD_CUDA(cudaStreamSynchronize(p->stream), "cudaStreamSynchronize");
    std::vector<double> tmp(3 * (size_t)p->n_obs);
    IOD_CUDA(cudaMemcpy(tmp.data(), p->d_rc(), sizeof(double) * tmp.size(), cudaMemcpyDeviceToHost), "cudaMemcpy");
    for (int k = 0; k < p->n_obs; ++k)
        for (int c = 0; c < 3; ++c) rc[3 * k + c] = tmp[(size_t)c * p->n_obs + k];
    return IOD_OK;
}

int iod_bounds_from_chief(const double chief_state[6], double r_max_km, double v_max_ms, double L_km,
                          double TU_s, double bounds[12])
{
    if (!chief_state || !bounds) return fail(IOD_EINVAL, "NULL argument");
    if (!(r_max_km > 0) || !(v_max_ms > 0) || !(L_km > 0) || !(TU_s > 0) || !finite_all(chief_state, 6))
        return fail(IOD_EINVAL, "limits and units must be finite and > 0");
    const double dr = r_max_km / L_km;
    const double dv = (v_max_ms / 1000.0) / (L_km / TU_s);
    for (int d = 0; d < 3; ++d) {
        bounds[d] = chief_state[d] - dr;
        bounds[6 + d] = chief_state[d] + dr;
        bounds[3 + d] = chief_state[3 + d] - dv;
        bounds[9 + d] = chief_state[3 + d] + dv;
    }
    return IOD_OK;
}

}  // extern "C"

namespace {
// observation synthesis in either dynamics (er = 1: ecc, f0 of the elliptic problem)
int simulate_obs(double mu, int er, double ecc, double f0, const double chief_state[6],
                 const double deputy_state[6], int n_obs, const double *obs_times, double rtol, double atol,
                 double h0, const double *noise, double *angles, double *ranges)
{
    if (!chief_state || !deputy_state || !obs_times || !angles || n_obs < 1) return fail(IOD_EINVAL, "bad arguments");
    if (!(mu > 0 && mu < 0.5) || !(h0 > 0) || !(rtol > 0 || atol > 0)) return fail(IOD_EINVAL, "bad settings");
    if (er && (!(ecc >= 0.0 && ecc < 1.0) || !std::isfinite(f0))) return fail(IOD_EINVAL, "need 0 <= ecc < 1, finite f0");
    if (!(obs_times[0] >= 0)) return fail(IOD_EINVAL, "obs_times must be >= 0");
    for (int k = 1; k < n_obs; ++k)
        if (!(obs_times[k] > obs_times[k - 1])) return fail(IOD_EINVAL, "obs_times must be strictly increasing");
    const size_t K = (size_t)n_obs;
    // layout: chief[6] deputy[6] t[K] noise[2K] angles[2K] ranges[K] chief_pos[3K] status
    DevBuf b;
    const size_t nd = 12 + 9 * K;
    int rc = dev_alloc(b, sizeof(double) * nd + 16);
    if (rc) return rc;
    double *d = (double *)b.ptr;
    double *dc = d, *dd = d + 6, *dt = d + 12, *dn = dt + K, *da = dn + 2 * K, *dr = da + 2 * K, *dp = dr + K;
    int *ds = (int *)(d + nd);
    std::vector<double> h(12 + 3 * K, 0.0);
    std::memcpy(h.data(), chief_state, 6 * sizeof(double));
    std::memcpy(h.data() + 6, deputy_state, 6 * sizeof(double));
    for (size_t k = 0; k < K; ++k)   // the integrators' independent variable
        h[12 + k] = er ? iod::er3bp_true_anomaly(ecc, f0, obs_times[k]) - f0 : obs_times[k];
    if (noise) std::memcpy(h.data() + 12 + K, noise, 2 * K * sizeof(double));
    cudaError_t e = cudaMemcpy(d, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = iod::launch_simulate(mu, ecc, f0, er, dc, dd, n_obs, dt, rtol, atol, h0, noise ? dn : nullptr, da,
                                 dr, dp, ds, nullptr);
    if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
    int status = 1;
    if (e == cudaSuccess) e = cudaMemcpy(angles, da, 2 * K * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && ranges) e = cudaMemcpy(ranges, dr, K * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&status, ds, sizeof(int), cudaMemcpyDeviceToHost);
    dev_free(b);
    if (e != cudaSuccess) return cuda_fail(e, "simulate");
    return status ? fail(IOD_EDIVERGED, "observation propagation failed") : IOD_OK;
}
}  // namespace

extern "C" {

int iod_simulate_obs(double mu, const double chief_state[6], const double deputy_state[6], int n_obs,
                     const double *obs_times, double rtol, double atol, double h0, const double *noise,
                     double *angles, double *ranges)
{
    return simulate_obs(mu, 0, 0.0, 0.0, chief_state, deputy_state, n_obs, obs_times, rtol, atol, h0, noise,
                        angles, ranges);
}

int iod_simulate_obs_er3bp(double mu, double ecc, double f0, const double chief_state[6],
                           const double deputy_state[6], int n_obs, const double *obs_times, double rtol,
                           double atol, double h0, const double *noise, double *angles, double *ranges)
{
    return simulate_obs(mu, 1, ecc, f0, chief_state, deputy_state, n_obs, obs_times, rtol, atol, h0, noise,
                        angles, ranges);
}

}  // extern "C"
