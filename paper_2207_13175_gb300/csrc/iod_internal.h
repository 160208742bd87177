// iod_internal.h -- structures shared by the host library and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

#include "iod_mixed.cuh"

namespace iod {

// Device-resident global best and run bookkeeping (one per problem).
struct GBest {
    double g[6];              // global best state
    double gJ;                // its cost
    int gidx;                 // its particle index
    int iter;                 // index of the last completed iteration (0 = initialisation)
    unsigned int done_blocks; // last-block-done counter of the running swarm kernel
    int status;               // nonzero: a device-side failure (bit flags below)
    unsigned long long steps; // integrator steps accumulated over all particles
    unsigned long long steps64; // mixed precision: steps taken in FP64 near the Moon
    int flags;                // kFlag* bits below
    int pad;
    double hist[32];          // global best cost after iteration n at hist[n % 32] (Algorithm 2)
    double g_pso[6];          // batches with refinement: the swarm's global best before it
    double gJ_pso;            // and its cost
    int lm_iters;             // Levenberg-Marquardt iterations taken
    int lm_status;            // its stop reason (0 iteration limit, 1 converged, 2 not evaluable)
    double lm_lam;            // its damping, carried between the refinement's actions
};

// Algorithm 2's window w compares J_n with J_{n-w}; the ring above holds w <= 31.
constexpr int kTolHist = 32;
// problem record in device memory: Consts at 0, GBest at kMiscGBest, chief state at kMiscChief
constexpr size_t kMiscGBest = 256, kMiscChief = 704, kMiscBytes = 768;
static_assert(sizeof(GBest) <= kMiscChief - kMiscGBest, "GBest overlaps the chief state");

// kStatusCheck: an argument check of the IOD_CHECK build failed
enum : int { kStatusChiefDiverged = 1, kStatusCopyTimeout = 2, kStatusHandoffTimeout = 4, kStatusCopyCheck = 8,
             kStatusCheck = 16 };
// kFlagRescored: personal bests re-evaluated in FP64; kFlagStarted: initialised;
// kFlagStopped: Algorithm 2's tolerance test ended the run (later iterations do nothing)
// kFlagRefined: the Levenberg-Marquardt refinement of a batch request has run
// kFlagLmStarted: the refinement has taken its start (g_pso kept; g, gJ are its current
// estimate and cost from then on)
// kFlagFallback: the request is being (or was) solved again in FP64 (the refinement gate)
enum : int { kFlagRescored = 1, kFlagStarted = 2, kFlagStopped = 4, kFlagRefined = 8, kFlagLmStarted = 16,
             kFlagFallback = 32 };
// Levenberg-Marquardt iterations per refinement action of a batch request: the action is
// resumable, so a serving slice can end between two of them
constexpr int kLmItersPerAction = 2;
// with a refinement gate, a refinement still above it after this many iterations stops and
// the request is solved again in FP64 (a fit that far off after as many iterations is not
// converging to the truth's minimum)
constexpr int kLmGateIters = 60;
// Levenberg-Marquardt scratch: kLmVecs vectors of the residual length (0 the estimate's
// residuals, 1-12 its central-difference columns, 13-20 the eight trials, 21-116 twelve
// columns about each of up to eight trial points, 117-122 the Jacobian's six columns),
// then kLmTail doubles carrying J^T J, J^T r and the Jacobian bookkeeping from one
// refinement action to the next.
constexpr int kLmJac = 21 + 12 * 8;
constexpr int kLmVecs = kLmJac + 6;
constexpr int kLmTail = 36 + 6 + 4;

// One block's best particle of the current launch (written by that block).
struct __align__(16) BlockBest {
    double J;
    int idx;
    int pad;
    double x[6];
};

// Problem constants computed on the device by the set-up kernel.
struct Consts {
    double w_ra, w_dec, w_rng;  // 1/sigma^2
    double vmax[6];             // vmax_frac * (hi - lo)
    double tend;                // last observation time
};

// Line-of-sight initialisation frame from the first observation (host-computed):
// direction u and tangent directions ea, eb of (alpha_0, beta_0), tilt half-widths,
// range interval.
struct ConeInit {
    double u[3], ea[3], eb[3];
    double smax[2];
    double rho[2];
};

// Everything a swarm kernel needs, passed by value.
// Balanced FP64 iteration: one resident warp per FP64 sub-partition (4 per SM).  The
// swarm's 32-particle groups are laid end to end, each as its epochs' propagation work;
// warp j takes the equal share from (group c0, epoch e0) to (group c1, epoch e1).  A
// group cut at an epoch boundary is propagated up to it by one warp (its first job) and
// finished by the next (its last job), which takes over the state and partial cost.
struct SplitSeg {
    int c0, e0, c1, e1;
};

struct SplitCtl {
    unsigned int stamp;      // balanced launches completed (the launch's last block counts it)
    int nw;                  // warps of the balanced launch (set by the plan)
    SplitSeg *seg;           // [nw] each warp's share
    unsigned int *flag;      // [nw] stamp of the launch in which warp j handed its group on
    double *hand;            // [nw][18][32] the hand-off per lane: RK4 state (6) and partial
                             // cost; DOPRI5 the integrator's loop state and partial cost
};

struct KParams {
    double mu;
    int n_obs;
    int integrator;
    int dynamics;        // 0 CR3BP, 1 ER3BP (independent variable: true anomaly - f0)
    double ecc, f0;      // ER3BP eccentricity and true anomaly at t = 0
    int cost_form;
    int use_range;
    double dt;           // RK4 step bound
    double rtol, atol, h0;
    long long max_steps;
    double lo[6], hi[6];
    double w, c1, c2;
    double kappa;        // constriction factor of Eq. 4 (host-computed; read when constriction)
    uint64_t seed;
    double tol_tau;      // Algorithm 2 tolerance (0: off) and window
    int tol_window;
    int constriction;    // 1: velocity update scaled by the constriction factor of Eq. 4
    int init_grid;       // 1: stratified initial positions
    int pair;            // 1: the FP64 RK4 swarm kernels run two threads per particle
    int velocity_init;   // 1: initial velocities uniform within the velocity limits
    int per_dim_random;  // 1: r1, r2 drawn per dimension
    int init_cone;       // 1: initial positions on the first line of sight (cone below)
    ConeInit cone;
    long long total_steps;  // RK4 steps per propagation (mixed precision)
    int m;               // particles
    int stride;          // SoA row stride (>= m)
    int offset;          // index of particle 0 in the whole swarm (sharded runs; else 0)
    int m_total;         // particles in the whole swarm (sharded runs; else m)
    // observation table (device, [n_obs] each; rc is [3][n_obs])
    const double *t, *ra, *dec, *rng, *rc, *h;
    const int *nsteps;
    const Consts *cst;
    // mixed precision: chief RK4 stage table [S], chief states at step boundaries [S+1][6],
    // observed-direction constants [n_obs]; moon_r2 = (FP64 radius about the Moon)^2
    const mix::Step *mix;
    const double *chief_cs;
    const mix::ObsDir *obsdir;
    const float *chunk_time;   // duration of each chunk of mixed_chunk_steps() steps
    double moon_r2;
    // swarm (device SoA [6][stride] for x, v, p; [stride] for pJ, J)
    double *x, *v, *p, *pJ, *J;
    GBest *gb;
    BlockBest *blk;
    double *trace_J;
    int *trace_idx;
    int trace_cap;
    SplitCtl *split;     // balanced iteration plan and hand-off buffers (null: not set up)
    const double *chief0;   // the chief's state at t = 0 (device; the DOPRI5 plan propagates it)
};

// One resident problem of a batch (device-resident descriptor).
struct BatchSlot {
    KParams P;                 // the problem, as the single-problem kernels see it
    int n_mixed;               // iterations in the FP32 phase (IOD_MIXED), -1 for FP64 problems
    int n_iters;               // iterations in total
    int n_tiles;               // blocks of this slot at its size class's block size
    int active;                // 1 while resident and not cancelled
    int action;                // this round's action (written by the plan kernel)
    int refine_iters;          // Levenberg-Marquardt iterations after the swarm (0: none)
    // set-up inputs and writable views of the tables the set-up kernel fills
    const double *chief;       // [6]
    double sig_ra, sig_dec, sig_rng, vmax_frac;
    double *rc_w, *h_w;
    int *ns_w;
    Consts *cst_w;
    mix::Step *mix_w;
    double *cs_w;
    mix::ObsDir *od_w;
    float *ct_w;
    double *lm_R;              // refinement scratch: kLmVecs residual vectors and kLmTail doubles
    double gate_cost;          // refined cost above which the request is solved again in FP64 (0: never)
};

enum : int { kActNone = 0, kActInitMixed = 1, kActIterMixed = 2, kActRescore = 3, kActInitFP64 = 4,
             kActIterFP64 = 5, kActRefine = 6, kActRestart = 7 };

// work queue of one round kernel (reset by its last block)
struct BatchQueue {
    unsigned int next, done;
};

// Dependency-driven scheduler state: a ring of (slot, tile) items with per-entry
// sequence stamps; indices only grow, so a stamp from an earlier launch never matches.
struct WorkQueue {
    unsigned long long head;   // next index to claim
    unsigned long long tail;   // next index to reserve for publishing
    int active;                // problems that will still publish work in this launch
    int status;                // kWqTimeout if a wait gave up, kWqCopyLost if a copy never landed
    unsigned long long t0;     // %globaltimer when the launch started
};
enum : int { kWqTimeout = 1, kWqCopyLost = 2 };

// kernel launchers (iod_kernels.cu); all return cudaError_t of the launch
cudaError_t launch_setup(const KParams &P, double vmax_frac, double sigma_ra, double sigma_dec,
                         double sigma_rng, const double *chief, double *rc_out, int *nsteps_out,
                         double *h_out, Consts *cst_out, GBest *gb, cudaStream_t st,
                         double *chief_cs = nullptr);
cudaError_t launch_setup_mixed(const KParams &P, mix::Step *steps, const double *chief_cs,
                               mix::ObsDir *obsdir, float *chunk_time, cudaStream_t st);
cudaError_t launch_init_mixed(const KParams &P, int block, cudaStream_t st);
cudaError_t launch_iter_mixed(const KParams &P, int block, int gbest_order, cudaStream_t st);
cudaError_t launch_rescore(const KParams &P, int block, cudaStream_t st);
cudaError_t launch_eval_mixed(const KParams &P, const double *x, int m, double *J, int block,
                              cudaStream_t st);
cudaError_t launch_propagate_mixed(const KParams &P, const double *x0, int m, double *out,
                                   int block, cudaStream_t st);
size_t mixed_smem_bytes(int n_obs, long long total_steps);
cudaError_t launch_batch_setup(BatchSlot *slots, const int *ids, int n, cudaStream_t st);
cudaError_t launch_batch_plan(BatchSlot *slots, int n_slots, cudaStream_t st);
cudaError_t launch_batch_round(BatchSlot *slots, const int2 *tiles, int n_tiles, BatchQueue *q,
                               int block, int grid, size_t smem, cudaStream_t st);
int batch_round_occupancy(int block, size_t smem);
cudaError_t launch_wq_seed(BatchSlot *slots, int n_slots, WorkQueue *q, int2 *ring,
                           unsigned long long *seq, unsigned long long cap, cudaStream_t st);
// throughput = 1: the scheduler form with more resident blocks (fewer registers per
// thread), for launches with more tiles than the other form holds at once
cudaError_t launch_wq_run(BatchSlot *slots, WorkQueue *q, int2 *ring, unsigned long long *seq,
                          unsigned long long cap, unsigned long long budget_ns, int block, int grid,
                          size_t smem, int throughput, cudaStream_t st);
int wq_occupancy(int block, size_t smem, int throughput);
cudaError_t launch_lm(const KParams &P, const double *x0, int max_iters, int form, double sig_ra,
                      double sig_dec, double *R, double *out, cudaStream_t st);
cudaError_t launch_set_gbest(GBest *gb, const double g[6], double gJ, int gidx, cudaStream_t st);
cudaError_t batch_round_prepare(size_t smem);   // call outside stream capture
int mixed_chunk_steps();
cudaError_t launch_init(const KParams &P, int block, cudaStream_t st);
cudaError_t launch_iter(const KParams &P, int block, int gbest_order, cudaStream_t st);
// balanced FP64 RK4 iteration (circular problem, one thread per particle): P.split set up
// by launch_split_plan for the current swarm and nw = wps x nsm warps; nsm blocks of
// 32 wps threads, cooperative
cudaError_t launch_split_plan(const KParams &P, int nw, int gsize, cudaStream_t st);
// balanced mixed-precision iteration: nsm blocks of kMixedBalancedThreads, cooperative;
// P.split planned with nw = nsm and gsize = kMixedBalancedThreads
cudaError_t launch_iter_mixed_balanced(const KParams &P, int gbest_order, int nsm, cudaStream_t st);
constexpr int kMixedBalancedThreads = 384;
// diagnostic: the hand-off wait on *flag (device) for stamp, limit_ns; results in device memory
cudaError_t launch_fp64_issue_probe(int warps, int lanes, int n, long long *cycles, double *sink, cudaStream_t st);
cudaError_t launch_wait_probe(const unsigned int *flag, unsigned int stamp, unsigned long long limit_ns,
                              int *timed_out, unsigned long long *waited_ns, cudaStream_t st);
// mode: 0 iteration (synchronous), 1 iteration (lagged), 2 initial evaluation
cudaError_t launch_iter_balanced(const KParams &P, int mode, int nsm, int wps, cudaStream_t st);
constexpr int kBalancedMaxWarpsPerSm = 12;
// the balanced DOPRI5 iteration: at most eight warps per SM (its ~190 registers per thread
// allow ten); an epoch's dense output and cost weigh about half an attempt; the hand-off
// holds 18 values per lane (DpState and the partial cost)
constexpr int kBalancedDpMaxWarpsPerSm = 8;
constexpr float kBalancedDpEpochWeight = 0.5f;
constexpr int kDpHandRows = 18;
constexpr double kBalancedEpochWeight = 1.25;   // an epoch's angles and cost, in RK4 steps
cudaError_t launch_eval(const KParams &P, const double *x, int m, double *J, int block,
                        cudaStream_t st);
cudaError_t launch_propagate(const KParams &P, const double *x0, int m, double *out, int block,
                             cudaStream_t st);
cudaError_t launch_simulate(double mu, double ecc, double f0, int er, const double *chief,
                            const double *deputy, int n, const double *t, double rtol, double atol,
                            double h0, const double *noise, double *angles, double *ranges,
                            double *chief_pos, int *status, cudaStream_t st);
size_t swarm_smem_bytes(int n_obs, int integrator);
// ER3BP true anomaly after nondimensional time tau from f0 (iod_api.cu)
double er3bp_true_anomaly(double e, double f0, double tau);
// constriction factor of Eq. 4, 2 / |2 - phi - sqrt(phi^2 - 4 phi)|, phi = c1 + c2 > 4
// (iod_api.cu; host code is compiled without floating-point contraction)
double constriction_kappa(double c1, double c2);
// line-of-sight initialisation frame of a first observation (alpha0, beta0) with
// half-widths k sigma and range interval [rho_min, rho_max] (iod_api.cu)
void cone_frame(double alpha0, double beta0, double sig_ra, double sig_dec, double k, double rho_min,
                double rho_max, ConeInit &out);
// record msg as the calling thread's last error and return code (iod_api.cu)
int set_last_error(int code, const char *msg);
// record a CUDA failure (IOD_ENOMEM for allocation failures, else IOD_ECUDA)
int cuda_error(cudaError_t e, const char *where);

// device allocations through the process-wide allocator hook (iod_api.cu)
struct Allocator {
    void *(*alloc)(size_t, void *) = nullptr;
    void (*release)(void *, void *) = nullptr;
    void *ctx = nullptr;
};
struct DevBuf {                 // remembers which allocator made it
    void *ptr = nullptr;
    size_t bytes = 0;
    Allocator a;
};
int dev_alloc(DevBuf &b, size_t bytes);
void dev_free(DevBuf &b);
int max_block_threads();

// An NVTX range over one C-ABI call (host side; header-only NVTX 3: without a profiler
// attached a push or pop is a check of a null function pointer).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace iod
