/*
 * iod.h -- C ABI of the GB300 (sm_103a) particle-swarm initial-orbit-determination
 * library for the Earth-Moon circular restricted three-body problem.
 *
 * The operation (Zuehlke et al., "Initial Orbit Determination for the CR3BP using
 * Particle Swarm Optimization"): a chief spacecraft with a known state observes a
 * deputy with angle (and optionally range) measurements at times t_k; a particle swarm
 * (Algorithm 1) searches the deputy's 6-D initial state.  Every iteration propagates
 * each candidate through the CR3BP equations of motion (Eqs. 1-3) to every t_k, forms
 * the chief-to-deputy line of sight and its azimuth/elevation (Eqs. 5-9), sums the
 * weighted squared residuals into the particle's cost (Eqs. 10-13), updates personal
 * and global bests and moves the particles inside a box built from the chief's known
 * state.  All of it runs in this library's CUDA kernels on one GPU.
 *
 * Conventions
 *  - Every int-returning call returns IOD_OK (0) or a negative IOD_E* code; nothing
 *    throws across the ABI.  iod_strerror() names a code, iod_last_error() gives the
 *    detail of the calling thread's last failure.
 *  - Units are nondimensional CR3BP units (LU = Earth-Moon distance, TU = 1/mean
 *    motion) unless a name says otherwise; angles are radians in the rotating
 *    barycentric (synodic) frame.
 *  - State vectors are (x, y, z, vx, vy, vz).  Device particle arrays are
 *    structure-of-arrays: component d of particle i at [d * m + i].
 *  - "host" pointers are ordinary CPU memory (pageable or pinned); "device" pointers
 *    are CUDA global memory on the current device.  The caller keeps ownership of every
 *    pointer it passes; the library copies what it needs during the call.
 *  - A problem owns the device memory it allocates (through the allocator hook if one
 *    is set, else cudaMalloc) and frees it in iod_destroy.
 *  - Work is queued on the problem's stream (iod_set_stream; default the legacy
 *    default stream).  Calls marked "async" return before the GPU finishes; calls
 *    marked "synchronising" wait for the stream.
 *  - A problem handle is not thread-safe: one thread (or external locking) per handle.
 */
#ifndef IOD_H
#define IOD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
#define IOD_OK 0
#define IOD_EINVAL (-1)      /* invalid argument (sizes, non-finite values, ordering) */
#define IOD_ENOMEM (-2)      /* device allocation failed */
#define IOD_ECUDA (-3)       /* a CUDA runtime call failed (detail in iod_last_error) */
#define IOD_ETIMEOUT (-4)    /* a bounded device wait ran out */
#define IOD_EBUSY (-5)       /* result not ready (batch interface) */
#define IOD_ECANCELLED (-6)  /* request cancelled (batch interface) */
#define IOD_ESTATE (-7)      /* call out of order (e.g. continue before run) */
#define IOD_EDIVERGED (-8)   /* the chief trajectory could not be propagated */

/* ---------------------------------------------------------------- option values */
#define IOD_RK4 0            /* fixed-step classical Runge-Kutta on the interval table */
#define IOD_DOPRI5 1         /* Dormand-Prince 5(4), dense output at t_k */
#define IOD_CR3BP 0          /* circular restricted three-body problem, Eqs. 1-3 */
#define IOD_ER3BP 1          /* elliptic restricted problem (see iod_options.dynamics) */
#define IOD_FP64 0           /* FP64 propagation and cost */
#define IOD_MIXED 1          /* FP32 relative (Encke) propagation, FP64 cost sums, FP64 refinement */
#define IOD_COST_CHI2 0      /* J = sum_k b_k^T W b_k */
#define IOD_COST_QUARTIC 1   /* J = b_total^T b_total = sum_k (b_k^T W b_k)^2 (Eqs. 11, 13 literal) */
#define IOD_GBEST_SYNC 0     /* move, evaluate, then global best of this iteration's positions */
#define IOD_GBEST_LAGGED 1   /* Algorithm 1's literal order: evaluate, move; global best after */
#define IOD_SCHED_AUTO 0     /* balanced where it lowers the busiest FP64 sub-partition's load */
#define IOD_SCHED_GRID 1     /* one thread per particle, blocks spread over the SMs */
#define IOD_SCHED_BALANCED 2 /* one warp per FP64 sub-partition, equal shares (iod_options.schedule) */

typedef struct iod_problem iod_problem;   /* opaque, library-owned */

typedef struct iod_options {
    int integrator;          /* IOD_RK4 (default) or IOD_DOPRI5 */
    double dt;               /* RK4: largest step (TU); interval k takes n_k = max(1, ceil(
                                (t_k - t_{k-1})/dt - 1e-9)) equal steps.  Default 1e-3 */
    double rtol, atol;       /* DOPRI5 tolerances.  Default 1e-12, 1e-12 */
    double h0;               /* DOPRI5 first step (TU).  Default 1e-3 */
    long long max_steps;     /* DOPRI5 attempts per propagation before J = +inf.  Default 1e7 */
    int precision;           /* IOD_FP64 (default) or IOD_MIXED (RK4 only): iterations are
                                propagated in FP32 as offsets from the chief until the last
                                fp64_last_iters, then every personal best is re-evaluated in
                                FP64 and the remaining iterations run in FP64 (iod_run with
                                iters = 0 initialises in FP32 and stays in that phase) */
    int cost_form;           /* IOD_COST_CHI2 (default) or IOD_COST_QUARTIC */
    int gbest_order;         /* IOD_GBEST_SYNC (default) or IOD_GBEST_LAGGED */
    double vmax_frac;        /* |v_d| <= vmax_frac * (hi_d - lo_d).  Default 1 */
    int use_range;           /* 1: range residuals enter with weight 1/sigma_range^2.  Default 0 */
    double sigma_range;      /* LU; read when use_range */
    int record_trace;        /* 1 (default): keep the global best cost/index of every iteration */
    int block_size;          /* threads per block of the swarm kernels; 0 = automatic */
    int fp64_last_iters;     /* IOD_MIXED: iterations at the end run in FP64.  Default 50 */
    double moon_fp64_radius; /* IOD_MIXED: steps starting closer than this to the Moon (LU)
                                are taken in FP64.  Default 0.02 */
    /* Variants of the particle swarm section (all off by default): */
    double tol_tau;          /* Algorithm 2: after iteration n > tol_window stop the run once
                                |(J_n - J_{n-w})/J_n| < tol_tau, J_n the global best cost after
                                iteration n (with IOD_MIXED, as scored in the phase that ran
                                it).  The test runs on the device; later iterations then do
                                nothing (IOD_MIXED still re-evaluates the personal bests in
                                FP64) and iters_done reports where it stopped.  0 = off */
    int tol_window;          /* w, 1..31.  Default 10 (Algorithm 2's window) */
    int constriction;        /* 1: the whole velocity update is multiplied by the constriction
                                factor of Eq. 4, kappa = 2/|2 - phi - sqrt(phi^2 - 4 phi)|,
                                phi = c1 + c2, which must exceed 4 (iod_run: IOD_EINVAL) */
    int init_grid;           /* 1: stratified ("grid-like") initial positions: along every
                                coordinate each of the swarm_size equal strata of the box
                                holds exactly one particle (a Latin hypercube; the strata are
                                dealt by the permutation (A_d i + B_d) mod m with B_d from
                                Philox stream 4), placed at its uniform draw inside it */
    int init_cone;           /* 1: sensor-feasible initial positions (the abstract's limit on
                                starting positions from the chief's position and the sensor):
                                at t_0 = 0 (required: IOD_EINVAL otherwise) each particle starts
                                at r_c(0) + rho d, rho uniform in [cone_rho_min, cone_rho_max]
                                and d the first observed direction u(alpha_0, beta_0) tilted in
                                its tangent plane by up to cone_sigmas * sigma per angle and
                                renormalised; clamped into the box; velocities uniform in the
                                box.  Combines with init_grid (the draws are stratified) */
    double cone_rho_min, cone_rho_max;   /* LU, 0 <= min < max */
    double cone_sigmas;      /* angular half-width in sigmas.  Default 3 */
    int velocity_init;       /* 0 (default): v = 0 at start; 1: each v_d uniform in
                                [-vmax_d, vmax_d], vmax_d = vmax_frac (hi_d - lo_d), from
                                Philox stream 5 (Algorithm 1 leaves the start unspecified) */
    int per_dim_random;      /* 0 (default): one (r1, r2) pair per particle per iteration, as
                                Algorithm 1 draws them; 1: one pair per dimension (stream 3,
                                block d; dimension 0 keeps the shared pair) */
    int threads_per_particle;/* 1: one thread per particle; 2: a lane pair per particle, each
                                lane evaluating one primary's attraction (FP64 circular
                                problems, RK4 or DOPRI5; results identical to 1); 0
                                (default): chosen by integrator and swarm size */
    /* Dynamics.  IOD_CR3BP (default): Eqs. 1-3.  IOD_ER3BP: the elliptic restricted
     * problem, named by the paper as future work, in Szebehely's pulsating rotating frame
     * with the true anomaly f as independent variable: x'' - 2y' = d(omega)/dx,
     * y'' + 2x' = d(omega)/dy, z'' = d(omega)/dz, omega = [(x^2 + y^2 - e z^2 cos f)/2 +
     * (1-mu)/r1 + mu/r2]/(1 + e cos f); ' = d/df.  The chief state, the estimated state
     * and the box are in that frame at t = 0; observation times (TU, mean motion 1) map to
     * true anomaly through Kepler's equation; dt bounds the RK4 step in f.  FP64 single
     * problems only (IOD_MIXED and batches: IOD_EINVAL). */
    int dynamics;
    double ecc;              /* IOD_ER3BP: eccentricity, 0 <= ecc < 1 */
    double f0;               /* IOD_ER3BP: true anomaly at t = 0 (rad) */
    /* Work distribution of the FP64 RK4 iterations (one thread per particle; circular
     * or elliptic problem; IOD_MIXED's FP64 iterations and the initial evaluation
     * included).  IOD_SCHED_GRID: one thread per
     * particle in blocks spread over the SMs.  IOD_SCHED_BALANCED: one to three resident
     * warps per FP64 sub-partition (one block of 4, 8 or 12 warps per SM, cooperative
     * launch), each taking an equal share of the swarm's propagation work: the 32-particle groups' work is laid
     * end to end and cut at epoch boundaries, and a group cut in two is propagated up to
     * the cut by one warp and finished by the next from the handed-over state and partial
     * cost.  Results are identical to IOD_SCHED_GRID.  Taken when the swarm has at least
     * as many 32-particle groups as the GPU has sub-partitions and a propagation is at most
     * 10^6 RK4 steps; otherwise the grid form runs.  IOD_MIXED's FP32 iterations have a
     * balanced form too: one 384-thread block per SM whose warps move through the epochs
     * together (they share the staged chief table), cutting super-groups of 384 particles
     * between SMs; taken from one super-group per SM upwards.  IOD_SCHED_AUTO (default):
     * balanced when, in addition, it lowers the busiest sub-partition's load (by more than
     * 3% in FP64, 15% in the FP32 iterations). */
    int schedule;
    /* Batches only (iod_batch_create; iod_create refuses a nonzero value -- single
     * problems call iod_refine): after a request's swarm iterations, refine its global
     * best by Levenberg-Marquardt (Sec. "Local Minimization", Eqs. 14-16), FP64, at most
     * refine_iters iterations, residuals of the cost form (CHI2: the 2K weighted angle
     * residuals; QUARTIC: the K per-epoch chi-squares).  The request's result is then the
     * refined state and cost, with the swarm's own best beside it (pso_state, pso_cost).
     * 0 (default): no refinement. */
    int refine_iters;
    /* Sharded swarms (single problems, IOD_FP64, tol_tau = 0): this problem holds particles
     * shard_offset .. shard_offset + swarm_size - 1 of a swarm of shard_total particles
     * split over several problems (processes, GPUs).  Every particle's random numbers
     * (Philox counters) and its stratum under init_grid are those of its index in the
     * whole swarm, and reported global best indices are whole-swarm indices; between
     * iterations the caller takes the best (cost, index) over the shards' global bests
     * (iod_gbest_get) and sets it on every shard (iod_gbest_set), after which every shard
     * continues exactly as its particles do in the unsharded run.  Algorithm 2's test is
     * then the caller's (it needs the whole swarm's best).  0 (default): not sharded. */
    int shard_offset;
    int shard_total;
    /* Batches with refine_iters > 0 only: a request whose refined cost exceeds
     * refine_gate * n_obs (or whose refinement is still above it after 60 iterations, when
     * it stops there) is solved once more from the start in FP64 (the same initial swarm,
     * FP64 iterations, the refinement), and that solve is its result (fallback = 1 in
     * iod_result_t; its rk_steps count both solves).  A converged fit costs about
     * 2 per epoch at the stated noise (CHI2) and far less without noise, so a gate of ten
     * or more singles out a swarm that ended in a false minimum.  0 (default): off. */
    double refine_gate;
} iod_options;

typedef struct iod_result_t {
    double state[6];         /* global best deputy initial state */
    double cost;             /* its cost J */
    int gbest_index;         /* particle index of the global best */
    int iters_done;          /* iterations completed after initialisation */
    long long rk_steps;      /* integrator steps (RK4 steps or DOPRI5 attempts), all particles */
    long long fp64_steps;    /* IOD_MIXED: how many of them were FP64 steps near the Moon */
    double *gcost_trace;     /* caller-owned, trace_capacity entries, or NULL: J(g) after the
                                initial evaluation (entry 0) and after each iteration */
    int *gidx_trace;         /* caller-owned, trace_capacity entries, or NULL */
    int trace_capacity;
    int schedule;            /* work distribution of the last swarm iteration launched (or of
                                the initial evaluation): IOD_SCHED_GRID or IOD_SCHED_BALANCED
                                (iod_options.schedule) */
    /* batch requests with iod_options.refine_iters > 0: the swarm's global best and its
       cost before the Levenberg-Marquardt refinement (state and cost above are the
       refined ones) and the refinement's iterations; otherwise equal to state and cost,
       and refine_iters = 0 */
    double pso_state[6];
    double pso_cost;
    int refine_iters;
    int fallback;            /* batch requests: 1 if the result is the FP64 solve that
                                iod_options.refine_gate asked for, else 0 */
} iod_result_t;

/* Fill *o with the defaults listed above.  Returns IOD_EINVAL if o is NULL. */
int iod_options_default(iod_options *o);

/* Create a problem (Sec. "Deputy Chief Scenario"; cost paragraph of the PSO section).
 *   mu          mass parameter, 0 < mu < 0.5
 *   chief_state host [6]: the chief's known state at t = 0
 *   n_obs       number of observation epochs, >= 1
 *   obs_times   host [n_obs]: TU, >= 0, strictly increasing
 *   obs_angles  host [n_obs][2]: observed (azimuth alpha, elevation beta) of the deputy
 *               from the chief, radians (Eqs. 7-8)
 *   sigma       host [2]: (sigma_alpha, sigma_beta) > 0; weights are 1/sigma^2 (Eq. 12)
 *   bounds      host [12]: lo[6] then hi[6], lo < hi, the box of candidate initial states
 *   opt         NULL for defaults
 *   out         receives the handle
 * Synchronising: computes the RK4 interval table and propagates the chief to every t_k
 * on the device.  IOD_EINVAL on bad sizes/values, IOD_EDIVERGED if the chief's
 * propagation fails, IOD_ENOMEM/IOD_ECUDA on device failures (nothing leaks). */
int iod_create(double mu, const double chief_state[6], int n_obs, const double *obs_times,
               const double *obs_angles, const double sigma[2], const double bounds[12],
               const iod_options *opt, iod_problem **out);

/* As iod_create, with observed ranges (host [n_obs], LU; read when opt->use_range). */
int iod_create_ranged(double mu, const double chief_state[6], int n_obs, const double *obs_times,
                      const double *obs_angles, const double *obs_ranges, const double sigma[2],
                      const double bounds[12], const iod_options *opt, iod_problem **out);

/* Queue all later work of p on cuda_stream (a cudaStream_t; NULL = legacy default). */
int iod_set_stream(iod_problem *p, void *cuda_stream);

/* Process-wide device allocator hook used for allocations made after the call:
 * alloc(bytes, ctx) returns device memory or NULL; release(ptr, ctx) frees it.  Pass
 * NULLs to restore cudaMalloc/cudaFree.  Problems free with the hook they allocated
 * with. */
int iod_set_allocator(void *(*alloc)(size_t, void *), void (*release)(void *, void *), void *ctx);

/* Run Algorithm 1: initialise swarm_size particles uniformly in the box (Philox4x32-10
 * stream 2, key = seed), evaluate them, then iterate `iters` times with inertia w,
 * cognitive c1 and social c2 (r1, r2 from Philox stream 3).  Async.  Re-running with
 * the same arguments reproduces the same result bit for bit.  IOD_EINVAL if
 * swarm_size < 1, iters < 0 or a coefficient is not finite. */
int iod_run(iod_problem *p, int swarm_size, int iters, double w, double c1, double c2,
            uint64_t seed);

/* Continue the current swarm for `iters` more iterations.  Async.  IOD_ESTATE before
 * iod_run.  With IOD_MIXED the iterations run in the phase the swarm is in (FP64 once
 * iod_run has reached its refinement phase). */
int iod_continue(iod_problem *p, int iters);

/* Wait for p's stream and report the global best (and traces if requested and
 * recorded).  Synchronising.  IOD_ESTATE before iod_run.  IOD_ETIMEOUT (the fields still
 * filled) if a bounded device wait of the run gave up: the mixed form's staging of the
 * chief table, or a hand-off between warps of the balanced schedule; the swarm is then
 * not to be trusted. */
int iod_result(iod_problem *p, iod_result_t *out);

/* Swarm state in host memory, structure-of-arrays [6][m] for x, v and pbest, [m] for
 * pbest_cost and cost.  iod_swarm_get is synchronising; any output may be NULL.
 * iod_swarm_set replaces the swarm (m particles, next iteration index iter + 1) with
 * the given state and run coefficients; it makes p ready for iod_continue. */
int iod_swarm_get(iod_problem *p, double *x, double *v, double *pbest, double *pbest_cost,
                  double *cost, double g[6], double *g_cost, int *g_index, int *iter);
int iod_swarm_set(iod_problem *p, int m, const double *x, const double *v, const double *pbest,
                  const double *pbest_cost, const double g[6], double g_cost, int g_index,
                  int iter, double w, double c1, double c2, uint64_t seed);

/* The global best record of a problem, for the exchange between the shards of one swarm
 * (iod_options.shard_total).  iod_gbest_get waits for p's stream and copies the state,
 * cost, whole-swarm index and the index of the last completed iteration (0 =
 * initialisation); any output may be NULL.  iod_gbest_set replaces the state, cost and
 * index (async, on p's stream: the values are passed by value, nothing of the caller's is
 * read later); the next iteration moves the particles towards it.  IOD_ESTATE before
 * iod_run, IOD_EINVAL for a non-finite state, a NaN cost or a negative index. */
int iod_gbest_get(iod_problem *p, double g[6], double *g_cost, int *g_index, int *iter);
int iod_gbest_set(iod_problem *p, const double g[6], double g_cost, int g_index);

/* Serialise the whole swarm state (positions, velocities, personal and global bests,
 * iteration counter, coefficients, seed) to buf.  Call with buf = NULL to get the size
 * in *len.  iod_restore loads such a buffer into a problem created with the same
 * inputs; continuing then reproduces an uninterrupted run bit for bit.  Synchronising. */
int iod_snapshot(iod_problem *p, void *buf, size_t *len);
int iod_restore(iod_problem *p, const void *buf, size_t len);

/* Free everything p owns (waits for its stream).  NULL is a no-op. */
void iod_destroy(iod_problem *p);

const char *iod_strerror(int code);
const char *iod_last_error(void);

/* Evaluate the cost J (Eqs. 5-13) of m candidate initial states with the problem's
 * precision.  x: device [6][m]; J: device [m].  Async. */
int iod_eval(iod_problem *p, const double *x, int m, double *J);

/* Diagnostic of the library's bounded device waits (no counterpart in the paper): runs
 * the wait that a warp of the balanced schedule performs before taking over a
 * hand-off, on a device flag that holds the awaited value already (set_flag = 1) or
 * that nothing sets (set_flag = 0), giving up after limit_s seconds.  Reports in
 * *timed_out whether the wait gave up (1) or returned (0), and in *waited_s the time
 * it waited by the GPU's global timer.  A wait that gives up ends its kernel normally:
 * the CUDA context stays usable.  Synchronising; uses the current device.  IOD_EINVAL
 * unless 0 < limit_s <= 10 and both pointers are non-NULL. */
int iod_selftest_wait(double limit_s, int set_flag, int *timed_out, double *waited_s);

/* Diagnostic of the FP64 pipe that the refinement's work distribution rests on: one
 * block of `warps` warps on one SM, in which lanes [0, lanes) of every warp run a
 * dependent chain of n FP64 FMAs.  Reports in *cycles_per_fma the SM clock cycles per FMA
 * of the slowest warp's chain (the second of two launches).  When an FP64 warp instruction
 * costs its sub-partition the same time whatever the number of active lanes, the result
 * does not depend on `lanes`.  Synchronising; uses the current device.  IOD_EINVAL unless
 * 1 <= warps <= 32, 1 <= lanes <= 32, 1 <= n <= 1e6 and the pointer is non-NULL. */
int iod_selftest_fp64_issue(int warps, int lanes, int n, double *cycles_per_fma);

/* Propagate m initial states to every observation time with p's integrator.  x0: device
 * [6][m]; out: device [n_obs][6][m].  Async. */
int iod_propagate(iod_problem *p, const double *x0, int m, double *out);

/* Levenberg-Marquardt refinement of a candidate initial state, e.g. the swarm's global
 * best (Sec. "Local Minimization", Eqs. 14-16), in FP64 with the problem's RK4 grid.
 *   x0        host [6] starting state
 *   max_iters iterations (each: a central-difference Jacobian and eight damped trials)
 *   form      0: least squares on the weighted angle residuals (2 n_obs entries; the
 *             minimised sum is the CHI2 cost); 1: on the per-epoch b_k^T W b_k (Eq. 15)
 *   x_out     host [6] refined state; cost_out: its sum of squared residuals;
 *   iters_out iterations run.  Synchronising.  IOD_EINVAL for a DOPRI5 problem. */
int iod_refine(iod_problem *p, const double x0[6], int max_iters, int form, double x_out[6],
               double *cost_out, int *iters_out);

/* Chief positions r_c(t_k) the problem uses: host [n_obs][3].  Synchronising. */
int iod_chief_positions(iod_problem *p, double *rc);

/* Box about a known chief state: +-r_max_km on each position axis and +-v_max_ms on
 * each velocity axis, converted with the length unit L_km and time unit TU_s.
 * bounds: host [12] = lo[6], hi[6]. */
int iod_bounds_from_chief(const double chief_state[6], double r_max_km, double v_max_ms,
                          double L_km, double TU_s, double bounds[12]);

/* Synthesise observations: propagate chief and deputy from t = 0 with DOPRI5 (rtol,
 * atol, first step h0) on the device in the CR3BP (Eqs. 1-3), form (alpha, beta, range)
 * at each t_k (Eqs. 5-9)
 * and add noise (host [n_obs][2] radians, or NULL).  angles: host [n_obs][2]; ranges:
 * host [n_obs] or NULL.  Synchronising. */
int iod_simulate_obs(double mu, const double chief_state[6], const double deputy_state[6],
                     int n_obs, const double *obs_times, double rtol, double atol, double h0,
                     const double *noise, double *angles, double *ranges);

/* As iod_simulate_obs, in the elliptic restricted problem (see iod_options.dynamics):
 * chief and deputy states in the pulsating frame at t = 0, eccentricity 0 <= ecc < 1,
 * true anomaly f0 at t = 0; times map to true anomaly by Kepler's equation.
 * Synchronising. */
int iod_simulate_obs_er3bp(double mu, double ecc, double f0, const double chief_state[6],
                           const double deputy_state[6], int n_obs, const double *obs_times,
                           double rtol, double atol, double h0, const double *noise,
                           double *angles, double *ranges);

/* ---------------------------------------------------------------- batches and serving
 * Many independent problems resident on one GPU at once (uneven observation counts,
 * swarm sizes and iteration counts), advanced together round by round: every round
 * gives each resident problem one step of Algorithm 1 (initialisation, an iteration,
 * or -- with IOD_MIXED -- the FP64 re-evaluation of its personal bests), all of it in a
 * few persistent kernels that pull (problem, block) tiles from a queue, captured as
 * CUDA graphs.  Requests are admitted while their device memory fits a budget and queue
 * otherwise; finished problems leave at the end of a step and their results stay on the
 * host until polled.  Batches run RK4 (IOD_FP64 or IOD_MIXED); the options of
 * iod_batch_create apply to every request.  A batch handle is not thread-safe.
 * Each problem's result is the one iod_run would give for the same inputs, with
 * IOD_MIXED always ending with the FP64 re-evaluation (also when fp64_last_iters = 0). */
typedef struct iod_batch iod_batch;

typedef struct iod_request {
    double mu;                    /* as iod_create */
    const double *chief_state;    /* host [6] */
    int n_obs;
    const double *obs_times;      /* host [n_obs] */
    const double *obs_angles;     /* host [n_obs][2] */
    const double *sigma;          /* host [2] */
    const double *bounds;         /* host [12] */
    int swarm_size;               /* >= 1 */
    int iters;                    /* >= 0 */
    double w, c1, c2;
    uint64_t seed;
} iod_request;

typedef struct iod_batch_stats {
    int resident;                 /* problems on the device */
    int queued;                   /* admitted later when memory frees up */
    long long finished;           /* results produced so far */
    long long rounds;             /* rounds run so far */
    size_t bytes_in_use;          /* device memory held by resident problems */
    size_t bytes_high_water;
    size_t budget;
    long long deferred_admissions;  /* admissions put off because the allocation failed
                                       while other problems were resident (the request
                                       stays queued and is retried on the next call) */
} iod_batch_stats;

/* Create a batch holding at most max_resident problems whose device memory totals at
 * most device_budget_bytes.  opt: NULL for defaults (integrator must be IOD_RK4). */
int iod_batch_create(const iod_options *opt, size_t device_budget_bytes, int max_resident,
                     iod_batch **out);
/* Use cuda_stream for the batch's work instead of its own non-blocking stream.  Graph
 * capture needs a stream other than the legacy default one. */
int iod_batch_set_stream(iod_batch *b, void *cuda_stream);
/* Threads per block by size class: a request with swarm_size <= max_swarm[c] (the first
 * such c, classes in increasing order) runs with block[c] threads per block. */
int iod_batch_set_block_sizes(iod_batch *b, int n_classes, const int *max_swarm, const int *block);
/* Copy a request into the batch; *ticket identifies it.  It becomes resident at the next
 * iod_batch_step / iod_batch_run that finds room.  IOD_ENOMEM if it alone exceeds the
 * budget.  If the device allocation for it fails at admission while other problems are
 * resident, admission backs off: the request stays first in the queue and is retried on
 * the next call (iod_batch_stats.deferred_admissions counts these); if nothing is
 * resident it fails and its poll returns IOD_ENOMEM.  Nothing leaks either way. */
int iod_batch_submit(iod_batch *b, const iod_request *req, long long *ticket);
/* Admit what fits, run `rounds` rounds, then retire finished problems.  Synchronising. */
int iod_batch_step(iod_batch *b, int rounds);
/* Admit what fits, then run the resident problems in one persistent launch for up to
 * `seconds` of device time (0: until every resident problem is done), each problem
 * starting its next step as soon as its previous one finishes (no rounds); then retire
 * finished problems.  Results equal iod_batch_step's.  Needs one block size for all
 * classes (IOD_EINVAL otherwise) and a GPU with cooperative launch.  IOD_ETIMEOUT if
 * a device-side wait gave up (the affected problems are failed).  Synchronising. */
int iod_batch_run(iod_batch *b, double seconds);
/* IOD_OK with the result (traces if the caller's arrays are set) once finished;
 * IOD_EBUSY while queued or resident; IOD_ECANCELLED; IOD_EINVAL for an unknown ticket. */
int iod_batch_poll(iod_batch *b, long long ticket, iod_result_t *out);
/* Host times (seconds since the batch was created) of submission, admission and
 * retirement; -1 for events that have not happened. */
int iod_batch_times(iod_batch *b, long long ticket, double *t_submit, double *t_admit, double *t_done);
/* Cancel a queued or resident request (resident ones leave at the next step). */
int iod_batch_cancel(iod_batch *b, long long ticket);
int iod_batch_get_stats(iod_batch *b, iod_batch_stats *out);
/* Autotuner: for each of n_classes sample requests (one per size class, max_swarm[c]
 * as in iod_batch_set_block_sizes) and each candidate block size, time one FP32 and
 * one FP64 iteration of the sample run alone (CUDA events) and weight them by the
 * sample's mix of iterations (iters - fp64_last_iters FP32, the rest FP64).  With
 * uniform = 0 each class gets its fastest size, else all classes get the size with
 * the smallest total (as iod_batch_run needs).  The chosen sizes are set on the
 * batch (nothing may be resident) and written to block_out[n_classes]; ms_out
 * [n_classes][n_cand] (or NULL) receives the weighted times.  Synchronising. */
int iod_batch_autotune(iod_batch *b, int n_classes, const int *max_swarm, const iod_request *samples,
                       int n_cand, const int *cand, int uniform, int *block_out, double *ms_out);
/* RK4 step bound by size class, with the classes of iod_batch_set_block_sizes' form: a
 * request with swarm_size <= max_swarm[c] (the first such c) integrates with dt[c] > 0
 * instead of iod_options.dt.  Nothing may be resident (IOD_ESTATE). */
int iod_batch_set_step_sizes(iod_batch *b, int n_classes, const int *max_swarm, const double *dt);
/* Step-size autotuner (no counterpart in the paper, whose integrator is unstated): for
 * each of n_classes sample requests (one per size class, max_swarm as above) take the
 * sample's first n_probe (1..4096) initial particles (its Philox initialisation) and
 * propagate them, and the chief, with DOPRI5 at rtol = atol = 1e-13 (the reference) and
 * with RK4 at each candidate step bound dt_cand[n_dt]; the error of a candidate is the
 * largest angle (rad) between its chief-to-probe line of sight and the reference's, over
 * probes and epochs.  Each class gets the largest candidate whose error is at most
 * angle_budget (the smallest candidate if none is); the choice is set on the batch
 * (iod_batch_set_step_sizes) and written to dt_out[n_classes]; err_out
 * [n_classes][n_dt] (or NULL) receives the errors.  Nothing may be resident.
 * Synchronising. */
int iod_batch_autotune_dt(iod_batch *b, int n_classes, const int *max_swarm, const iod_request *samples,
                          int n_dt, const double *dt_cand, double angle_budget, int n_probe,
                          double *dt_out, double *err_out);
void iod_batch_destroy(iod_batch *b);

/* ---------------------------------------------------------------- allocation-free scoring
 * The paper has no counterpart to this call; it is a library convenience.
 *
 * Some callers cannot call cudaMalloc once they are running: a flight or real-time
 * loop whose device memory is fixed at start-up, a host program that hands every
 * byte of device memory to its own pool, or code that must never trigger the implicit
 * device synchronisation an allocation can cause.  This entry point scores candidates
 * without allocating anything: it calls no cudaMalloc, cudaFree or allocating library
 * routine.  Its scratch (the per-block best candidates and a completion counter) is a
 * fixed array of about 128 KB inside the library, which every GPU that loads the
 * library keeps until the process exits.
 *
 * It computes what iod_eval computes for an RK4 problem with the default CHI2 cost and
 * no range term, plus the best candidate:
 *   mu        mass parameter, 0 < mu < 0.5
 *   n_obs     epochs, >= 1 (limited by one block's shared memory, ~3,700 on GB300)
 *   obs       device [6][n_obs]: t_k (TU, >= 0, strictly increasing -- not checked),
 *             observed alpha~, observed beta~ (rad), and the chief position r_c(t_k)
 *             as x, y, z rows (LU), e.g. from iod_chief_positions
 *   sigma_ra, sigma_dec > 0; dt > 0 the RK4 step bound (interval rule of iod_options)
 *   x         device [6][m] candidate initial states, 1 <= m <= 131,072
 *   J         device [m] output: each candidate's cost
 *   best      device [8] output: best cost, its index (as a double), its state [6]
 *             (lowest index on ties)
 *   cuda_stream  stream to queue on (NULL = legacy default).  Async.
 * Returns IOD_EINVAL for sizes or values out of range (m above 131,072 included).
 * The first call on each device looks up the scratch array's device address and sets
 * the kernel's shared-memory limit, with that device current; make that first call
 * before any stream capture.  The address belongs to the context the look-up ran in:
 * after cudaDeviceReset (or in another context) the first call looks it up again, so
 * that call too should come before any capture.  The scratch's counter is cleared at the start of every
 * call, so an interrupted call does not poison the next one.  All calls on a device
 * share the one scratch array: calls that overlap on the GPU (different streams, or
 * different host threads) race and must be serialised by the caller. */
int iod_score_noalloc(double mu, int n_obs, const double *obs, double sigma_ra, double sigma_dec,
                      double dt, const double *x, int m, double *J, double *best, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* IOD_H */
