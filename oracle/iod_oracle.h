/*
 * iod_oracle.h -- plain, slow, single-threaded FP64 CPU oracle for particle-swarm
 * initial orbit determination in the Earth-Moon CR3BP (Zuehlke et al., "Initial
 * Orbit Determination for the CR3BP using Particle Swarm Optimization").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or call
 * this code; only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no source with the CUDA library.
 *
 * Every function follows the paper's definition in the paper's order, with no
 * blocking, fusion or reordering, compiled with -ffp-contract=off (no FMA) and
 * libm's sqrt/atan2/asin.  Where the paper is silent the reading taken is written
 * beside the function.
 *
 * Parity status of each part (what pins it is listed in the tests):
 *   RHS, RK4, DOPRI5 + dense output, angles, cost, PSO   -- pinned
 *   Philox4x32-10                                         -- pinned by known-answer vectors
 *   ER3BP right-hand side and time mapping                -- pinned (e = 0 reduction,
 *                                                            equilibria, energy-rate identity,
 *                                                            Kepler's equation)
 */
#ifndef IOD_ORACLE_H
#define IOD_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define ORA_OK 0
#define ORA_EINVAL (-1)
#define ORA_EDIVERGED (-2)   /* non-finite state or integrator gave up */

/* integrators */
#define ORA_RK4 0
#define ORA_DOPRI5 1

/* cost forms (Eqs. 11-13) */
#define ORA_COST_CHI2 0      /* J = sum_k b_k^T W b_k */
#define ORA_COST_QUARTIC 1   /* J = b_total^T b_total = sum_k (b_k^T W b_k)^2 */

/* gbest orders (Algorithm 1) */
#define ORA_GBEST_SYNC 0     /* gbest from this iteration's evaluated positions */
#define ORA_GBEST_LAGGED 1   /* Algorithm 1's literal order: evaluate, then move */

/* ---- dynamics (Eqs. 1-3) ---- */
void ora_rhs(double mu, const double s[6], double ds[6]);
double ora_jacobi(double mu, const double s[6]);

/* ---- elliptic restricted three-body problem (the paper's future work) ---- */
#define ORA_CR3BP 0
#define ORA_ER3BP 1
/* pulsating rotating frame, derivatives with respect to the true anomaly f */
void ora_rhs_er3bp(double mu, double e, double f, const double s[6], double ds[6]);
/* true anomaly (continuous, not wrapped) reached after nondimensional time tau from
   true anomaly f0, by Kepler's equation; the primaries' mean motion is 1 */
double ora_er3bp_anomaly(double e, double f0, double tau);

/* ---- propagation to observation times (Sec. "Particle Swarm Optimizer", cost paragraph) ---- */
int ora_rk4_grid(int n, const double *t, double dt, int *nsteps, double *h);
void ora_rk4_step(double mu, double h, double s[6]);
int ora_propagate_rk4(double mu, const double s0[6], int n, const double *t, double dt,
                      double *out, long long *steps);

typedef struct {
    double rtol, atol, h0;
    long long max_steps;
} ora_dopri5_opts;

/* one Dormand-Prince 5(4) attempt from (t, s) with step h.  k1 = f(s) on entry;
   writes the 5th-order solution s1, the 7 stage derivatives k[7][6] and returns the
   scaled error norm. */
double ora_dopri5_attempt(double mu, double h, const double s[6], const double k1[6],
                          double s1[6], double k[7][6], double rtol, double atol);
/* continuous extension at theta in [0,1] of the last attempt */
void ora_dopri5_dense(double h, const double s[6], double k[7][6], double theta, double out[6]);
int ora_propagate_dopri5(double mu, const double s0[6], int n, const double *t,
                         const ora_dopri5_opts *o, double *out, long long *accepted,
                         long long *rejected);

/* ---- measurement model and cost (Eqs. 5-13) ---- */
void ora_angles(const double rho[3], double *alpha, double *beta, double *range);

typedef struct {
    double mu;
    int n_obs;
    const double *t;       /* [n_obs] TU, strictly increasing, >= 0 */
    const double *ra;      /* [n_obs] observed azimuth (rad) */
    const double *dec;     /* [n_obs] observed elevation (rad) */
    const double *rng;     /* [n_obs] observed range (LU); read only when use_range */
    double sigma_ra, sigma_dec, sigma_rng;
    const double *rc;      /* [n_obs][3] chief position at t_k */
    int integrator;        /* ORA_RK4 / ORA_DOPRI5 */
    double dt;             /* RK4 step bound */
    ora_dopri5_opts dp;    /* DOPRI5 settings */
    int cost_form;         /* ORA_COST_* */
    int use_range;         /* 0: angles only (w_1 = 0) */
    int dynamics;          /* ORA_CR3BP or ORA_ER3BP */
    double ecc, f0;        /* ER3BP: eccentricity of the primaries, true anomaly at t = 0 */
} ora_problem;

int ora_propagate(const ora_problem *P, const double s0[6], double *out, long long *steps);
double ora_cost_from_states(const ora_problem *P, const double *states /*[n_obs][6]*/);
double ora_cost(const ora_problem *P, const double x[6], long long *steps);
double ora_cost_sphere(const double *center /*[6]*/, const double x[6]);

/* ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) ---- */
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double ora_u01(uint32_t hi_word, uint32_t lo_word);

/* ---- particle swarm (Algorithm 1) ---- */
#define ORA_OBJ_IOD 0
#define ORA_OBJ_SPHERE 1

typedef struct {
    int objective;          /* ORA_OBJ_IOD (ctx = ora_problem*) or ORA_OBJ_SPHERE (ctx = double[6]) */
    const void *ctx;
    double lo[6], hi[6];
    double w, c1, c2;
    double vmax_frac;       /* |v_d| <= vmax_frac * (hi_d - lo_d) */
    int gbest_order;        /* ORA_GBEST_* */
    uint64_t seed;
    double tol_tau;         /* Algorithm 2: stop when |(J_n - J_{n-w})/J_n| < tol_tau, n > w; 0 = off */
    int tol_window;         /* w (Algorithm 2 uses 10) */
    int constriction;       /* 1: v <- kappa (w v + ...), kappa of Eq. 4 with phi = c1 + c2 */
    int init_grid;          /* 1: stratified (Latin hypercube) initial positions */
    int init_cone;          /* 1 (IOD objective, t_0 = 0): initial positions on the first
                               observation's line of sight, see ora_pso_init */
    double cone_rho_min, cone_rho_max;   /* range interval along it (LU) */
    double cone_sigmas;     /* angular half-width in units of sigma_alpha, sigma_beta */
    int velocity_init;      /* 0: v = 0; 1: v_d uniform in [-vmax_d, vmax_d] (Philox stream 5) */
    int per_dim_random;     /* 1: r1, r2 drawn per dimension (stream 3, block d) */
} ora_pso;

/* swarm state, AoS [m][6] rows */
typedef struct {
    int m;
    double *x, *v, *p;      /* [m][6] */
    double *pJ, *J;         /* [m] */
    double g[6];
    double gJ;
    int gidx;
    long long steps;        /* integrator steps taken so far (IOD objective) */
    int iters_done;         /* iterations run by ora_pso_run (fewer than asked if Algorithm 2 stopped it) */
} ora_swarm;

int ora_pso_init(const ora_pso *S, ora_swarm *W);
int ora_pso_iterate(const ora_pso *S, ora_swarm *W, int n);
int ora_pso_run(const ora_pso *S, ora_swarm *W, int iters, double *gJ_trace, int *gidx_trace);
double ora_constriction(double c1, double c2);

/* ---- Levenberg-Marquardt refinement (Eqs. 14-16) ---- */
#define ORA_LM_RESIDUALS 0   /* residual vector: weighted angle residuals, 2 n_obs entries */
#define ORA_LM_EPOCH_CHI2 1  /* residual vector: per-epoch b_k^T W b_k, n_obs entries (Eq. 15) */
int ora_lm_residuals(const ora_problem *P, const double x[6], int form, double *r);
int ora_lm_refine(const ora_problem *P, const double x0[6], int max_iters, int form,
                  double x_out[6], double *cost_out, int *iters_out);

/* ---- scenario helpers ---- */
void ora_bounds_from_chief(const double chief[6], double r_max_km, double v_max_ms,
                           double L_km, double TU_s, double lo[6], double hi[6]);
int ora_simulate_obs(double mu, const double chief0[6], const double deputy0[6], int n,
                     const double *t, const ora_dopri5_opts *o, const double *noise /*[n][2] or NULL*/,
                     double *ra, double *dec, double *rng, double *rc /*[n][3]*/);
/* the same with ER3BP dynamics (ecc, f0); ecc = 0 is the CR3BP in the same code path */
int ora_simulate_obs_er3bp(double mu, double ecc, double f0, const double chief0[6],
                           const double deputy0[6], int n, const double *t, const ora_dopri5_opts *o,
                           const double *noise, double *ra, double *dec, double *rng, double *rc);

#ifdef __cplusplus
}
#endif
#endif
