/*
 * iod_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see iod_oracle.h).
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared -o liboracle.so iod_oracle.c -lm
 * No FMA contraction, no fast-math: each line is the formula it cites, evaluated in
 * the order written.  Single-threaded.
 */
#include "iod_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------
 * Dynamics: Eqs. 1-3, CR3BP in the rotating barycentric (synodic) frame, nondim.
 * Earth at (-mu, 0, 0), Moon at (1 - mu, 0, 0).  (The garbled "mu" without its
 * backslash in Eq. 2 is read as the mass parameter mu.)
 * ------------------------------------------------------------------------------ */
void ora_rhs(double mu, const double s[6], double ds[6])
{
    const double x = s[0], y = s[1], z = s[2];
    const double vx = s[3], vy = s[4], vz = s[5];
    const double d1x = x + mu;               /* x + mu       */
    const double d2x = x - (1.0 - mu);       /* x - (1 - mu) */
    const double r1sq = d1x * d1x + y * y + z * z;
    const double r2sq = d2x * d2x + y * y + z * z;
    const double r1cube = r1sq * sqrt(r1sq); /* ((x+mu)^2+y^2+z^2)^(3/2) */
    const double r2cube = r2sq * sqrt(r2sq);
    ds[0] = vx;
    ds[1] = vy;
    ds[2] = vz;
    ds[3] = 2.0 * vy + x - (1.0 - mu) * d1x / r1cube - mu * d2x / r2cube;   /* Eq. 1 */
    ds[4] = -2.0 * vx + y - (1.0 - mu) * y / r1cube - mu * y / r2cube;      /* Eq. 2 */
    ds[5] = -(1.0 - mu) * z / r1cube - mu * z / r2cube;                     /* Eq. 3 */
}

/* Jacobi constant C = x^2 + y^2 + 2(1-mu)/r1 + 2 mu/r2 - v^2 (Szebehely); the
   integral of Eqs. 1-3, used only by tests. */
double ora_jacobi(double mu, const double s[6])
{
    const double d1x = s[0] + mu, d2x = s[0] - (1.0 - mu);
    const double r1 = sqrt(d1x * d1x + s[1] * s[1] + s[2] * s[2]);
    const double r2 = sqrt(d2x * d2x + s[1] * s[1] + s[2] * s[2]);
    const double v2 = s[3] * s[3] + s[4] * s[4] + s[5] * s[5];
    return s[0] * s[0] + s[1] * s[1] + 2.0 * (1.0 - mu) / r1 + 2.0 * mu / r2 - v2;
}

/* ------------------------------------------------------------------------------
 * Elliptic restricted three-body problem, named by the paper as future work.  Standard
 * form (Szebehely, Theory of Orbits, ch. 10): pulsating rotating frame scaled by the
 * primaries' instantaneous distance, independent variable the true anomaly f,
 *   x'' - 2 y' = d(omega)/dx,  y'' + 2 x' = d(omega)/dy,  z'' = d(omega)/dz,
 *   omega = [ (x^2 + y^2 - e z^2 cos f)/2 + (1-mu)/r1 + mu/r2 ] / (1 + e cos f).
 * e = 0 gives Eqs. 1-3.  Directions from chief to deputy are unchanged by the common
 * scaling, so the measurement model (Eqs. 5-9) applies as it stands.
 * ------------------------------------------------------------------------------ */
void ora_rhs_er3bp(double mu, double e, double f, const double s[6], double ds[6])
{
    const double x = s[0], y = s[1], z = s[2];
    const double vx = s[3], vy = s[4], vz = s[5];
    const double d1x = x + mu;
    const double d2x = x - (1.0 - mu);
    const double r1sq = d1x * d1x + y * y + z * z;
    const double r2sq = d2x * d2x + y * y + z * z;
    const double r1cube = r1sq * sqrt(r1sq);
    const double r2cube = r2sq * sqrt(r2sq);
    const double ecf = e * cos(f);
    const double scale = 1.0 / (1.0 + ecf);
    const double wx = (x - (1.0 - mu) * d1x / r1cube - mu * d2x / r2cube) * scale;
    const double wy = (y - (1.0 - mu) * y / r1cube - mu * y / r2cube) * scale;
    const double wz = (-ecf * z - (1.0 - mu) * z / r1cube - mu * z / r2cube) * scale;
    ds[0] = vx;
    ds[1] = vy;
    ds[2] = vz;
    ds[3] = 2.0 * vy + wx;
    ds[4] = -2.0 * vx + wy;
    ds[5] = wz;
}

/* Time to true anomaly for the ER3BP: mean anomaly M = M0 + tau (unit mean motion),
   Kepler's equation E - e sin E = M by Newton's method from E = M, and the half-angle
   relation tan((f - E)/2) = b sin E / (1 - b cos E), b = e / (1 + sqrt(1 - e^2)),
   which keeps f continuous (not wrapped) as tau grows. */
double ora_er3bp_anomaly(double e, double f0, double tau)
{
    if (e == 0.0) return f0 + tau;
    const double b = e / (1.0 + sqrt(1.0 - e * e));
    const double E0 = f0 - 2.0 * atan(b * sin(f0) / (1.0 + b * cos(f0)));
    const double M = (E0 - e * sin(E0)) + tau;
    double E = M;
    for (int it = 0; it < 100; ++it) {
        const double dE = (E - e * sin(E) - M) / (1.0 - e * cos(E));
        E -= dE;
        if (fabs(dE) <= 1e-15 * fmax(1.0, fabs(E))) break;
    }
    return E + 2.0 * atan(b * sin(E) / (1.0 - b * cos(E)));
}

/* the dynamics a propagation runs: CR3BP, or ER3BP about true anomaly f0 + s where s
   is the integrator's independent variable */
typedef struct {
    double mu, e, f0;
    int er;
} dynctx;

static void rhs_ctx(const dynctx *D, double s_ind, const double s[6], double ds[6])
{
    if (D->er)
        ora_rhs_er3bp(D->mu, D->e, D->f0 + s_ind, s, ds);
    else
        ora_rhs(D->mu, s, ds);
}

static int finite6(const double s[6])
{
    for (int i = 0; i < 6; ++i)
        if (!isfinite(s[i])) return 0;
    return 1;
}

/* ------------------------------------------------------------------------------
 * Fixed-step RK4 to the measurement times.  The paper propagates each particle "to
 * all measurement times t_k" and names no integrator.  Reading: interval k runs from
 * t_{k-1} to t_k (t_{-1} = 0) in n_k equal steps, n_k = max(1, ceil(dt_k/dt - 1e-9)),
 * h_k = dt_k / n_k, so every step lands exactly on t_k; n_k = 0 when dt_k = 0.
 * ------------------------------------------------------------------------------ */
int ora_rk4_grid(int n, const double *t, double dt, int *nsteps, double *h)
{
    if (n < 1 || !(dt > 0.0)) return ORA_EINVAL;
    double prev = 0.0;
    for (int k = 0; k < n; ++k) {
        const double span = t[k] - prev;
        if (!(span >= 0.0)) return ORA_EINVAL;
        if (span == 0.0) {
            nsteps[k] = 0;
            h[k] = 0.0;
        } else {
            double q = ceil(span / dt - 1e-9);
            if (q < 1.0) q = 1.0;
            nsteps[k] = (int)q;
            h[k] = span / q;
        }
        prev = t[k];
    }
    return ORA_OK;
}

/* classical fourth-order Runge-Kutta step from independent variable s_ind */
static void rk4_step_ctx(const dynctx *D, double s_ind, double h, double s[6])
{
    double k1[6], k2[6], k3[6], k4[6], tmp[6];
    rhs_ctx(D, s_ind, s, k1);
    for (int i = 0; i < 6; ++i) tmp[i] = s[i] + 0.5 * h * k1[i];
    rhs_ctx(D, s_ind + 0.5 * h, tmp, k2);
    for (int i = 0; i < 6; ++i) tmp[i] = s[i] + 0.5 * h * k2[i];
    rhs_ctx(D, s_ind + 0.5 * h, tmp, k3);
    for (int i = 0; i < 6; ++i) tmp[i] = s[i] + h * k3[i];
    rhs_ctx(D, s_ind + h, tmp, k4);
    for (int i = 0; i < 6; ++i)
        s[i] = s[i] + h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

void ora_rk4_step(double mu, double h, double s[6])
{
    const dynctx D = {mu, 0.0, 0.0, 0};
    rk4_step_ctx(&D, 0.0, h, s);
}

static int propagate_rk4_ctx(const dynctx *D, const double s0[6], int n, const double *t,
                             double dt, double *out, long long *steps);

int ora_propagate_rk4(double mu, const double s0[6], int n, const double *t, double dt,
                      double *out, long long *steps)
{
    const dynctx D = {mu, 0.0, 0.0, 0};
    return propagate_rk4_ctx(&D, s0, n, t, dt, out, steps);
}

/* step j of interval k starts at independent variable t_{k-1} + j h_k (t_{-1} = 0) */
static int propagate_rk4_ctx(const dynctx *D, const double s0[6], int n, const double *t,
                             double dt, double *out, long long *steps)
{
    int *ns = (int *)malloc(sizeof(int) * (size_t)n);
    double *hs = (double *)malloc(sizeof(double) * (size_t)n);
    if (!ns || !hs) { free(ns); free(hs); return ORA_EINVAL; }
    int rc = ora_rk4_grid(n, t, dt, ns, hs);
    if (rc != ORA_OK) { free(ns); free(hs); return rc; }
    double s[6];
    memcpy(s, s0, sizeof s);
    long long taken = 0;
    for (int k = 0; k < n; ++k) {
        const double base = k == 0 ? 0.0 : t[k - 1];
        for (int j = 0; j < ns[k]; ++j) rk4_step_ctx(D, base + j * hs[k], hs[k], s);
        taken += ns[k];
        memcpy(out + 6 * (size_t)k, s, sizeof s);
    }
    free(ns);
    free(hs);
    if (steps) *steps += taken;
    return finite6(s) ? ORA_OK : ORA_EDIVERGED;
}

/* ------------------------------------------------------------------------------
 * Dormand-Prince 5(4) (Dormand & Prince 1980), FSAL, local extrapolation.  Error norm
 * and step controller as in Hairer, Norsett & Wanner, Solving ODEs I, Sec. II.4:
 *   err = sqrt(mean_i (e_i / (atol + rtol max(|y_i|, |y1_i|)))^2),  e = h sum_j E_j k_j
 *   accept iff err <= 1;  h <- h min(5, max(0.2, 0.9 err^(-1/5)))
 * Output at t_k by the fourth-order continuous extension (Shampine 1986; HNW II.6).
 * The integrator is unnamed in the paper; this is the reading for the DOPRI5 option.
 * ------------------------------------------------------------------------------ */
static const double DP_C2 = 1.0 / 5.0, DP_C3 = 3.0 / 10.0, DP_C4 = 4.0 / 5.0, DP_C5 = 8.0 / 9.0;
static const double DP_A21 = 1.0 / 5.0;
static const double DP_A31 = 3.0 / 40.0, DP_A32 = 9.0 / 40.0;
static const double DP_A41 = 44.0 / 45.0, DP_A42 = -56.0 / 15.0, DP_A43 = 32.0 / 9.0;
static const double DP_A51 = 19372.0 / 6561.0, DP_A52 = -25360.0 / 2187.0,
                    DP_A53 = 64448.0 / 6561.0, DP_A54 = -212.0 / 729.0;
static const double DP_A61 = 9017.0 / 3168.0, DP_A62 = -355.0 / 33.0, DP_A63 = 46732.0 / 5247.0,
                    DP_A64 = 49.0 / 176.0, DP_A65 = -5103.0 / 18656.0;
static const double DP_B1 = 35.0 / 384.0, DP_B3 = 500.0 / 1113.0, DP_B4 = 125.0 / 192.0,
                    DP_B5 = -2187.0 / 6784.0, DP_B6 = 11.0 / 84.0;
/* E_j = b_j - bhat_j (fifth minus fourth order weights) */
static const double DP_E1 = 71.0 / 57600.0, DP_E3 = -71.0 / 16695.0, DP_E4 = 71.0 / 1920.0,
                    DP_E5 = -17253.0 / 339200.0, DP_E6 = 22.0 / 525.0, DP_E7 = -1.0 / 40.0;

/* one attempt from independent variable tc (stage i at tc + c_i h) */
static double dopri5_attempt_ctx(const dynctx *D, double tc, double h, const double s[6],
                                 const double k1[6], double s1[6], double k[7][6], double rtol,
                                 double atol)
{
    double tmp[6];
    memcpy(k[0], k1, sizeof(double) * 6);
    for (int i = 0; i < 6; ++i) tmp[i] = s[i] + h * (DP_A21 * k[0][i]);
    rhs_ctx(D, tc + DP_C2 * h, tmp, k[1]);
    for (int i = 0; i < 6; ++i) tmp[i] = s[i] + h * (DP_A31 * k[0][i] + DP_A32 * k[1][i]);
    rhs_ctx(D, tc + DP_C3 * h, tmp, k[2]);
    for (int i = 0; i < 6; ++i)
        tmp[i] = s[i] + h * (DP_A41 * k[0][i] + DP_A42 * k[1][i] + DP_A43 * k[2][i]);
    rhs_ctx(D, tc + DP_C4 * h, tmp, k[3]);
    for (int i = 0; i < 6; ++i)
        tmp[i] = s[i] + h * (DP_A51 * k[0][i] + DP_A52 * k[1][i] + DP_A53 * k[2][i] +
                             DP_A54 * k[3][i]);
    rhs_ctx(D, tc + DP_C5 * h, tmp, k[4]);
    for (int i = 0; i < 6; ++i)
        tmp[i] = s[i] + h * (DP_A61 * k[0][i] + DP_A62 * k[1][i] + DP_A63 * k[2][i] +
                             DP_A64 * k[3][i] + DP_A65 * k[4][i]);
    rhs_ctx(D, tc + h, tmp, k[5]);
    for (int i = 0; i < 6; ++i)
        s1[i] = s[i] + h * (DP_B1 * k[0][i] + DP_B3 * k[2][i] + DP_B4 * k[3][i] +
                            DP_B5 * k[4][i] + DP_B6 * k[5][i]);
    rhs_ctx(D, tc + h, s1, k[6]);
    double sum = 0.0;
    for (int i = 0; i < 6; ++i) {
        const double e = h * (DP_E1 * k[0][i] + DP_E3 * k[2][i] + DP_E4 * k[3][i] +
                              DP_E5 * k[4][i] + DP_E6 * k[5][i] + DP_E7 * k[6][i]);
        const double sc = atol + rtol * fmax(fabs(s[i]), fabs(s1[i]));
        sum += (e / sc) * (e / sc);
    }
    return sqrt(sum / 6.0);
}

double ora_dopri5_attempt(double mu, double h, const double s[6], const double k1[6],
                          double s1[6], double k[7][6], double rtol, double atol)
{
    const dynctx D = {mu, 0.0, 0.0, 0};
    return dopri5_attempt_ctx(&D, 0.0, h, s, k1, s1, k, rtol, atol);
}

/* y(t + theta h) = y + h sum_i b_i(theta) k_i with the fourth-order polynomials
   b_i(theta) of the Dormand-Prince continuous extension (HNW I, Sec. II.6). */
void ora_dopri5_dense(double h, const double s[6], double k[7][6], double theta, double out[6])
{
    const double th = theta;
    const double a = th * th * (3.0 - 2.0 * th);       /* theta^2 (3 - 2 theta) */
    const double q = th * th * (th - 1.0) * (th - 1.0); /* theta^2 (theta - 1)^2 */
    const double b1 = a * DP_B1 + th * (th - 1.0) * (th - 1.0) -
                      q * 5.0 * (2558722523.0 - 31403016.0 * th) / 11282082432.0;
    const double b3 = a * DP_B3 + q * 100.0 * (882725551.0 - 15701508.0 * th) / 32700410799.0;
    const double b4 = a * DP_B4 - q * 25.0 * (443332067.0 - 31403016.0 * th) / 1880347072.0;
    const double b5 = a * DP_B5 + q * 32805.0 * (23143187.0 - 3489224.0 * th) / 199316789632.0;
    const double b6 = a * DP_B6 - q * 55.0 * (29972135.0 - 7076736.0 * th) / 822651844.0;
    const double b7 = th * th * (th - 1.0) + q * 10.0 * (7414447.0 - 829305.0 * th) / 29380423.0;
    for (int i = 0; i < 6; ++i)
        out[i] = s[i] + h * (b1 * k[0][i] + b3 * k[2][i] + b4 * k[3][i] + b5 * k[4][i] +
                             b6 * k[5][i] + b7 * k[6][i]);
}

static int propagate_dopri5_ctx(const dynctx *D, const double s0[6], int n, const double *t,
                                const ora_dopri5_opts *o, double *out, long long *accepted,
                                long long *rejected);

int ora_propagate_dopri5(double mu, const double s0[6], int n, const double *t,
                         const ora_dopri5_opts *o, double *out, long long *accepted,
                         long long *rejected)
{
    const dynctx D = {mu, 0.0, 0.0, 0};
    return propagate_dopri5_ctx(&D, s0, n, t, o, out, accepted, rejected);
}

static int propagate_dopri5_ctx(const dynctx *D, const double s0[6], int n, const double *t,
                                const ora_dopri5_opts *o, double *out, long long *accepted,
                                long long *rejected)
{
    if (n < 1 || !(o->h0 > 0.0) || !(o->rtol > 0.0 || o->atol > 0.0)) return ORA_EINVAL;
    double s[6], s1[6], k1[6], k[7][6];
    memcpy(s, s0, sizeof s);
    double tc = 0.0, h = o->h0;
    const double tend = t[n - 1];
    int next = 0;
    long long acc = 0, rej = 0;
    while (next < n && t[next] <= tc) {        /* observations at the start time */
        memcpy(out + 6 * (size_t)next, s, sizeof s);
        ++next;
    }
    rhs_ctx(D, tc, s, k1);
    while (next < n) {
        if (acc + rej >= o->max_steps || !(h > 0.0) || !finite6(s)) return ORA_EDIVERGED;
        int last = 0;
        if (tc + h >= tend) {                  /* stop exactly at the last t_k */
            h = tend - tc;
            last = 1;
        }
        const double err = dopri5_attempt_ctx(D, tc, h, s, k1, s1, k, o->rtol, o->atol);
        if (!isfinite(err)) return ORA_EDIVERGED;
        double fac = 0.9 * pow(err, -0.2);
        if (err == 0.0 || fac > 5.0) fac = 5.0;
        if (fac < 0.2) fac = 0.2;
        if (err <= 1.0) {
            const double tn = last ? tend : tc + h;
            while (next < n && t[next] <= tn) {
                if (t[next] == tn) {
                    memcpy(out + 6 * (size_t)next, s1, sizeof s1);
                } else {
                    const double theta = (t[next] - tc) / h;
                    ora_dopri5_dense(h, s, k, theta, out + 6 * (size_t)next);
                }
                ++next;
            }
            memcpy(s, s1, sizeof s);
            memcpy(k1, k[6], sizeof k1);       /* FSAL */
            tc = tn;
            ++acc;
        } else {
            ++rej;
        }
        h = h * fac;
    }
    if (accepted) *accepted += acc;
    if (rejected) *rejected += rej;
    return finite6(s) ? ORA_OK : ORA_EDIVERGED;
}

/* ------------------------------------------------------------------------------
 * Measurement model, Eqs. 5-9: rho = r_d - r_c, L = rho/|rho|,
 * alpha = atan2(L_2, L_1) (Eq. 7 printed with one argument; read as the
 * two-argument arctangent of the y and x components), beta = asin(L_3), range |rho|.
 * ------------------------------------------------------------------------------ */
void ora_angles(const double rho[3], double *alpha, double *beta, double *range)
{
    const double r = sqrt(rho[0] * rho[0] + rho[1] * rho[1] + rho[2] * rho[2]);
    const double L[3] = {rho[0] / r, rho[1] / r, rho[2] / r};
    *alpha = atan2(L[1], L[0]);
    *beta = asin(L[2]);
    *range = r;
}

/* ER3BP: the observation times map to elapsed true anomaly f(t_k) - f0, which is the
   integrators' independent variable (the RK4 step bound dt then bounds steps in f) */
static double *er3bp_grid(double e, double f0, int n, const double *t)
{
    double *g = (double *)malloc(sizeof(double) * (size_t)n);
    if (!g) return NULL;
    for (int k = 0; k < n; ++k) g[k] = ora_er3bp_anomaly(e, f0, t[k]) - f0;
    return g;
}

int ora_propagate(const ora_problem *P, const double s0[6], double *out, long long *steps)
{
    const dynctx D = {P->mu, P->ecc, P->f0, P->dynamics == ORA_ER3BP};
    double *grid = NULL;
    const double *t = P->t;
    if (D.er) {
        grid = er3bp_grid(P->ecc, P->f0, P->n_obs, P->t);
        if (!grid) return ORA_EINVAL;
        t = grid;
    }
    int rc;
    if (P->integrator == ORA_RK4) {
        rc = propagate_rk4_ctx(&D, s0, P->n_obs, t, P->dt, out, steps);
    } else {
        long long acc = 0, rej = 0;
        rc = propagate_dopri5_ctx(&D, s0, P->n_obs, t, &P->dp, out, &acc, &rej);
        if (steps) *steps += acc + rej;
    }
    free(grid);
    return rc;
}

/* Eqs. 10-13.  b(t_k) = y~(t_k) - y(t_k), W = diag(1/sigma_rng^2, 1/sigma_ra^2,
   1/sigma_dec^2) (Eq. 12; w_1 = 0 for angles-only), J = sum_k b_k^T W b_k (CHI2) or
   J = b_total^T b_total = sum_k (b_k^T W b_k)^2 (QUARTIC, Eqs. 11 and 13 read
   literally).  The azimuth residual is wrapped to [-pi, pi] (paper silent).
   A degenerate line of sight (|rho| < 1e-15 LU) or any non-finite value gives
   J = +inf. */
double ora_cost_from_states(const ora_problem *P, const double *states)
{
    const double two_pi = 6.283185307179586; /* 2 pi rounded to double */
    const double w_ra = 1.0 / (P->sigma_ra * P->sigma_ra);
    const double w_dec = 1.0 / (P->sigma_dec * P->sigma_dec);
    const double w_rng = P->use_range ? 1.0 / (P->sigma_rng * P->sigma_rng) : 0.0;
    double J = 0.0;
    for (int k = 0; k < P->n_obs; ++k) {
        const double *rd = states + 6 * (size_t)k;
        const double rho[3] = {rd[0] - P->rc[3 * k + 0], rd[1] - P->rc[3 * k + 1],
                               rd[2] - P->rc[3 * k + 2]};                          /* Eq. 5 */
        const double rr = sqrt(rho[0] * rho[0] + rho[1] * rho[1] + rho[2] * rho[2]);
        if (!(rr >= 1e-15) || !isfinite(rr)) return INFINITY;
        double alpha, beta, range;
        ora_angles(rho, &alpha, &beta, &range);
        const double b_ra = remainder(P->ra[k] - alpha, two_pi);
        const double b_dec = P->dec[k] - beta;
        const double b_rng = P->use_range ? (P->rng[k] - range) : 0.0;
        const double Jk = b_rng * w_rng * b_rng + b_ra * w_ra * b_ra + b_dec * w_dec * b_dec;
        J += (P->cost_form == ORA_COST_QUARTIC) ? Jk * Jk : Jk;
    }
    return isfinite(J) ? J : INFINITY;
}

double ora_cost(const ora_problem *P, const double x[6], long long *steps)
{
    double *states = (double *)malloc(sizeof(double) * 6 * (size_t)P->n_obs);
    if (!states) return INFINITY;
    const int rc = ora_propagate(P, x, states, steps);
    const double J = (rc == ORA_OK) ? ora_cost_from_states(P, states) : INFINITY;
    free(states);
    return J;
}

/* a test objective for the swarm on its own: sum_d (x_d - c_d)^2 */
double ora_cost_sphere(const double *center, const double x[6])
{
    double J = 0.0;
    for (int d = 0; d < 6; ++d) J += (x[d] - center[d]) * (x[d] - center[d]);
    return J;
}

/* ------------------------------------------------------------------------------
 * Philox4x32-10 as defined by Salmon, Moraes, Dror & Shaw (SC'11): ten rounds of
 *   (c0, c1, c2, c3) <- (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
 * with M0 = 0xD2511F53, M1 = 0xCD9E8D57 and the key bumped by the Weyl constants
 * (0x9E3779B9, 0xBB67AE85) between rounds.
 * ------------------------------------------------------------------------------ */
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 53-bit double in [0, 1) from two words: ((a >> 5) 2^26 + (b >> 6)) 2^-53 */
double ora_u01(uint32_t hi_word, uint32_t lo_word)
{
    const double a = (double)(hi_word >> 5);
    const double b = (double)(lo_word >> 6);
    return (a * 67108864.0 + b) * (1.0 / 9007199254740992.0);
}

/* ------------------------------------------------------------------------------
 * Particle swarm, Algorithm 1.
 * Random numbers: key = (seed lo, seed hi); counter = (particle i, iteration n,
 * stream, block).  Stream 2 = initial positions (n = 0, blocks 0..2 give dims
 * (0,1), (2,3), (4,5)); stream 3 = the (r1, r2) pair of iteration n (block 0;
 * one scalar pair per particle per iteration, as Algorithm 1 draws "r1, r2").
 * Readings where the algorithm is silent: v_i = 0 at start; |v_d| clamped to
 * vmax_frac (hi_d - lo_d); a coordinate that leaves [lo_d, hi_d] is set to the bound
 * and its velocity to zero; ties in the argmin go to the lowest index; NaN costs
 * count as +inf.
 * ------------------------------------------------------------------------------ */
static void draw(uint64_t seed, uint32_t i, uint32_t n, uint32_t stream, uint32_t block,
                 double *u0, double *u1)
{
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    const uint32_t ctr[4] = {i, n, stream, block};
    uint32_t r[4];
    ora_philox4x32_10(ctr, key, r);
    *u0 = ora_u01(r[0], r[1]);
    *u1 = ora_u01(r[2], r[3]);
}

static double objective(const ora_pso *S, const double x[6], long long *steps)
{
    if (S->objective == ORA_OBJ_SPHERE) return ora_cost_sphere((const double *)S->ctx, x);
    const double J = ora_cost((const ora_problem *)S->ctx, x, steps);
    return isnan(J) ? INFINITY : J;
}

/* lowest-index argmin with NaN read as +inf */
static int argmin(const double *J, int m)
{
    int best = 0;
    for (int i = 1; i < m; ++i)
        if (J[i] < J[best]) best = i;
    return best;
}

/* Stratified ("grid-like", Sec. "Particle Swarm Optimization") initial position of
   particle i: per dimension d the m strata are visited in the order of the permutation
   pi_d(i) = (A_d i + B_d) mod m, A_d a prime above 2^31 (so coprime with m), B_d from
   Philox (stream 4, block d), and the particle sits at the uniform draw u inside its
   stratum: t = (pi_d(i) + u)/m in place of u, position lo + t (hi - lo). */
static const uint64_t GRID_A[6] = {2147483659ull, 2147483693ull, 2147483713ull,
                                   2147483743ull, 2147483777ull, 2147483783ull};

static double grid_t(const ora_pso *S, int m, int i, int d, double u)
{
    const uint32_t key[2] = {(uint32_t)S->seed, (uint32_t)(S->seed >> 32)};
    const uint32_t ctr[4] = {0u, 0u, 4u, (uint32_t)d};
    uint32_t r[4];
    ora_philox4x32_10(ctr, key, r);
    const uint64_t B = (uint64_t)r[0] % (uint64_t)m;
    const uint64_t pi = (GRID_A[d] * (uint64_t)i + B) % (uint64_t)m;
    return ((double)pi + u) / (double)m;
}

/* Sensor-feasible initial positions (the abstract's limit on starting positions from
   the known chief position and the sensor): at t_0 = 0 the deputy lies on the first
   observation's line of sight from the chief, r = r_c(0) + rho u(alpha_0, beta_0), with
   u = (cos b cos a, cos b sin a, sin b) the direction of Eqs. 7-8.  Reading: the range
   rho is drawn uniformly in [rho_min, rho_max] and the direction is tilted in the plane
   tangent to u along e_a = (-sin a, cos a, 0) and e_b = (-sin b cos a, -sin b sin a,
   cos b) by s_a, s_b uniform in +-k sigma_alpha cos b and +-k sigma_beta (the sensor's
   angular uncertainty), then renormalised; positions outside the box are clamped onto
   it.  The three position draws are the uniform initialisation's (or the stratified
   ones); velocities stay uniform in the box. */
static int cone_positions(const ora_pso *S, const double t[3], double x[3])
{
    const ora_problem *P = (const ora_problem *)S->ctx;
    const double a = P->ra[0], b = P->dec[0];
    const double ca = cos(a), sa = sin(a), cb = cos(b), sb = sin(b);
    const double u[3] = {cb * ca, cb * sa, sb};
    const double ea[3] = {-sa, ca, 0.0};
    const double eb[3] = {-sb * ca, -sb * sa, cb};
    const double smax_a = S->cone_sigmas * P->sigma_ra * cb, smax_b = S->cone_sigmas * P->sigma_dec;
    const double rho = S->cone_rho_min + t[0] * (S->cone_rho_max - S->cone_rho_min);
    const double s_a = (2.0 * t[1] - 1.0) * smax_a, s_b = (2.0 * t[2] - 1.0) * smax_b;
    double d[3];
    for (int j = 0; j < 3; ++j) d[j] = u[j] + s_a * ea[j] + s_b * eb[j];
    const double n = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int j = 0; j < 3; ++j) {
        double r = P->rc[3 * 0 + j] + rho * (d[j] / n);
        if (r < S->lo[j]) r = S->lo[j];
        if (r > S->hi[j]) r = S->hi[j];
        x[j] = r;
    }
    return ORA_OK;
}

int ora_pso_init(const ora_pso *S, ora_swarm *W)
{
    if (W->m < 1) return ORA_EINVAL;
    if (S->constriction && !(S->c1 + S->c2 > 4.0)) return ORA_EINVAL;     /* Eq. 4 needs phi > 4 */
    if (S->tol_tau > 0.0 && S->tol_window < 1) return ORA_EINVAL;
    if (S->init_cone) {
        const ora_problem *P = (const ora_problem *)S->ctx;
        if (S->objective != ORA_OBJ_IOD || P->t[0] != 0.0) return ORA_EINVAL;
        if (!(S->cone_rho_min >= 0.0) || !(S->cone_rho_max > S->cone_rho_min) || !(S->cone_sigmas > 0.0))
            return ORA_EINVAL;
    }
    for (int i = 0; i < W->m; ++i) {
        double *x = W->x + 6 * (size_t)i;
        double t[6];    /* the draws, uniform or stratified, in [0, 1) */
        for (int b = 0; b < 3; ++b) {
            double u0, u1;
            draw(S->seed, (uint32_t)i, 0u, 2u, (uint32_t)b, &u0, &u1);
            t[2 * b] = u0;
            t[2 * b + 1] = u1;
        }
        for (int d = 0; d < 6; ++d) {
            if (S->init_grid) t[d] = grid_t(S, W->m, i, d, t[d]);
            x[d] = S->lo[d] + t[d] * (S->hi[d] - S->lo[d]);
        }
        if (S->init_cone) cone_positions(S, t, x);
        /* initial velocity: zero (Algorithm 1 leaves it unspecified), or uniform within
           the velocity limits from Philox stream 5, block b giving dimensions 2b, 2b+1 */
        for (int d = 0; d < 6; ++d) W->v[6 * (size_t)i + d] = 0.0;
        if (S->velocity_init) {
            for (int b = 0; b < 3; ++b) {
                double u0, u1;
                draw(S->seed, (uint32_t)i, 0u, 5u, (uint32_t)b, &u0, &u1);
                const double m0 = S->vmax_frac * (S->hi[2 * b] - S->lo[2 * b]);
                const double m1 = S->vmax_frac * (S->hi[2 * b + 1] - S->lo[2 * b + 1]);
                W->v[6 * (size_t)i + 2 * b] = (2.0 * u0 - 1.0) * m0;
                W->v[6 * (size_t)i + 2 * b + 1] = (2.0 * u1 - 1.0) * m1;
            }
        }
        W->J[i] = objective(S, x, &W->steps);
        memcpy(W->p + 6 * (size_t)i, x, sizeof(double) * 6);   /* x_best <- x */
        W->pJ[i] = W->J[i];
    }
    W->gidx = argmin(W->J, W->m);                               /* g <- min J(x_i) */
    W->gJ = W->J[W->gidx];
    memcpy(W->g, W->x + 6 * (size_t)W->gidx, sizeof(double) * 6);
    return ORA_OK;
}

/* Eq. 4: kappa = 2/|2 - phi - sqrt(phi^2 - 4 phi)|, phi = c1 + c2 > 4.  Where kappa
   multiplies is not stated; reading (Clerc and Kennedy's form): the whole velocity
   update, v <- kappa (w v + c1 r1 (p - x) + c2 r2 (g - x)). */
double ora_constriction(double c1, double c2)
{
    const double phi = c1 + c2;
    return 2.0 / fabs(2.0 - phi - sqrt(phi * phi - 4.0 * phi));
}

static void move(const ora_pso *S, ora_swarm *W, int i, int n)
{
    double *x = W->x + 6 * (size_t)i, *v = W->v + 6 * (size_t)i;
    const double *p = W->p + 6 * (size_t)i;
    double r1, r2;
    draw(S->seed, (uint32_t)i, (uint32_t)n, 3u, 0u, &r1, &r2);
    const double kappa = S->constriction ? ora_constriction(S->c1, S->c2) : 1.0;
    for (int d = 0; d < 6; ++d) {
        /* one (r1, r2) pair per particle per iteration, as Algorithm 1 draws them, or one
           pair per dimension (block d of the same stream; block 0 is the shared pair) */
        if (S->per_dim_random && d > 0) draw(S->seed, (uint32_t)i, (uint32_t)n, 3u, (uint32_t)d, &r1, &r2);
        double vd = S->w * v[d] + S->c1 * r1 * (p[d] - x[d]) + S->c2 * r2 * (W->g[d] - x[d]);
        if (S->constriction) vd = kappa * vd;
        const double vmax = S->vmax_frac * (S->hi[d] - S->lo[d]);
        if (vd > vmax) vd = vmax;
        if (vd < -vmax) vd = -vmax;
        double xd = x[d] + vd;
        if (xd < S->lo[d]) { xd = S->lo[d]; vd = 0.0; }
        if (xd > S->hi[d]) { xd = S->hi[d]; vd = 0.0; }
        v[d] = vd;
        x[d] = xd;
    }
}

static void personal_best(ora_swarm *W, int i)
{
    if (W->J[i] < W->pJ[i]) {           /* strict decrease only */
        W->pJ[i] = W->J[i];
        memcpy(W->p + 6 * (size_t)i, W->x + 6 * (size_t)i, sizeof(double) * 6);
    }
}

int ora_pso_iterate(const ora_pso *S, ora_swarm *W, int n)
{
    if (S->gbest_order == ORA_GBEST_SYNC) {
        /* move with the current global best, evaluate, personal best, then the
           global best from this iteration's evaluated positions */
        for (int i = 0; i < W->m; ++i) {
            move(S, W, i, n);
            W->J[i] = objective(S, W->x + 6 * (size_t)i, &W->steps);
            personal_best(W, i);
        }
        const int b = argmin(W->J, W->m);
        if (W->J[b] < W->gJ) {
            W->gJ = W->J[b];
            W->gidx = b;
            memcpy(W->g, W->x + 6 * (size_t)b, sizeof(double) * 6);
        }
        return ORA_OK;
    }
    /* Algorithm 1 literally: per particle evaluate, personal best, move; after the
       particle loop the global best takes the best evaluated (pre-move) position. */
    double *xe = (double *)malloc(sizeof(double) * 6 * (size_t)W->m);
    if (!xe) return ORA_EINVAL;
    for (int i = 0; i < W->m; ++i) {
        W->J[i] = objective(S, W->x + 6 * (size_t)i, &W->steps);
        personal_best(W, i);
        memcpy(xe + 6 * (size_t)i, W->x + 6 * (size_t)i, sizeof(double) * 6);
        move(S, W, i, n);
    }
    const int b = argmin(W->J, W->m);
    if (W->J[b] < W->gJ) {
        W->gJ = W->J[b];
        W->gidx = b;
        memcpy(W->g, xe + 6 * (size_t)b, sizeof(double) * 6);
    }
    free(xe);
    return ORA_OK;
}

/* Algorithm 2: after iteration n > w, stop when |(J_n - J_{n-w})/J_n| < tau, with J_n
   the global best cost after iteration n (the listing's window w = 10; the prose's
   "three" is not used). */
int ora_pso_run(const ora_pso *S, ora_swarm *W, int iters, double *gJ_trace, int *gidx_trace)
{
    int rc = ora_pso_init(S, W);
    if (rc != ORA_OK) return rc;
    double *hist = (double *)malloc(sizeof(double) * (size_t)(iters + 1));
    if (!hist) return ORA_EINVAL;
    hist[0] = W->gJ;
    if (gJ_trace) gJ_trace[0] = W->gJ;
    if (gidx_trace) gidx_trace[0] = W->gidx;
    W->iters_done = 0;
    for (int n = 1; n <= iters; ++n) {
        rc = ora_pso_iterate(S, W, n);
        if (rc != ORA_OK) break;
        W->iters_done = n;
        hist[n] = W->gJ;
        if (gJ_trace) gJ_trace[n] = W->gJ;
        if (gidx_trace) gidx_trace[n] = W->gidx;
        if (S->tol_tau > 0.0 && n > S->tol_window) {
            const double K = fabs((hist[n] - hist[n - S->tol_window]) / hist[n]);
            if (K < S->tol_tau) break;
        }
    }
    free(hist);
    return rc;
}

/* ------------------------------------------------------------------------------
 * Levenberg-Marquardt refinement of a candidate initial state (Eqs. 14-16).  The paper
 * runs MATLAB's Levenberg-Marquardt on the vector F of per-epoch weighted residuals;
 * its settings are unstated.  Reading: minimise ||r||^2 where r is the weighted angle
 * residual vector (r_2k = wrap(a~ - a)/s_a, r_2k+1 = (b~ - b)/s_b; ||r||^2 is the CHI2
 * cost) or, as an option, F_k = b_k^T W b_k itself (Eq. 15 literally).  Jacobian by
 * central differences with step h_j = 1e-7 max(|x_j|, 0.1).  Each iteration solves
 * (J^T J + lam_i diag(J^T J)) d = -J^T r by Cholesky for the eight damping values
 * lam_i = lam 10^(i-3), i = 0..7, evaluates all eight trials, keeps the lowest cost
 * (lowest i on ties) if it is below the current cost and sets lam = lam_i/10; otherwise
 * lam *= 1e5.  Stops after max_iters iterations, when lam exceeds 1e16, or when the
 * relative cost decrease falls below 1e-10.  Starting lam = 1e-3.
 * ------------------------------------------------------------------------------ */
int ora_lm_residuals(const ora_problem *P, const double x[6], int form, double *r)
{
    const int K = P->n_obs;
    double *st = (double *)malloc(sizeof(double) * 6 * (size_t)K);
    if (!st) return ORA_EINVAL;
    int rc = ora_propagate(P, x, st, NULL);
    const double two_pi = 6.283185307179586;
    for (int k = 0; k < K; ++k) {
        const double *rd = st + 6 * (size_t)k;
        const double rho[3] = {rd[0] - P->rc[3 * k + 0], rd[1] - P->rc[3 * k + 1],
                               rd[2] - P->rc[3 * k + 2]};
        double a, b, rr;
        ora_angles(rho, &a, &b, &rr);
        const double ba = remainder(P->ra[k] - a, two_pi);
        const double bb = P->dec[k] - b;
        if (form == ORA_LM_RESIDUALS) {
            r[2 * k] = ba / P->sigma_ra;
            r[2 * k + 1] = bb / P->sigma_dec;
        } else {
            r[k] = ba * (1.0 / (P->sigma_ra * P->sigma_ra)) * ba + bb * (1.0 / (P->sigma_dec * P->sigma_dec)) * bb;
        }
    }
    free(st);
    const int n = form == ORA_LM_RESIDUALS ? 2 * K : K;
    for (int i = 0; i < n; ++i)
        if (!isfinite(r[i])) rc = ORA_EDIVERGED;
    return rc;
}

static double sumsq(const double *r, int n)
{
    double c = 0.0;
    for (int i = 0; i < n; ++i) c += r[i] * r[i];
    return c;
}

/* solve (A + lam diag(A)) d = -g for symmetric positive definite 6x6 A (Cholesky) */
static int damped_solve(const double A[36], const double g[6], double lam, double d[6])
{
    double M[36], L[36] = {0}, y[6];
    for (int i = 0; i < 36; ++i) M[i] = A[i];
    for (int i = 0; i < 6; ++i) M[7 * i] = A[7 * i] + lam * A[7 * i];
    for (int i = 0; i < 6; ++i) {
        for (int j = 0; j <= i; ++j) {
            double sum = M[6 * i + j];
            for (int k = 0; k < j; ++k) sum -= L[6 * i + k] * L[6 * j + k];
            if (i == j) {
                if (!(sum > 0.0)) return ORA_EDIVERGED;
                L[6 * i + i] = sqrt(sum);
            } else {
                L[6 * i + j] = sum / L[6 * j + j];
            }
        }
    }
    for (int i = 0; i < 6; ++i) {           /* L y = -g */
        double sum = -g[i];
        for (int k = 0; k < i; ++k) sum -= L[6 * i + k] * y[k];
        y[i] = sum / L[6 * i + i];
    }
    for (int i = 5; i >= 0; --i) {          /* L^T d = y */
        double sum = y[i];
        for (int k = i + 1; k < 6; ++k) sum -= L[6 * k + i] * d[k];
        d[i] = sum / L[6 * i + i];
    }
    return ORA_OK;
}

int ora_lm_refine(const ora_problem *P, const double x0[6], int max_iters, int form,
                  double x_out[6], double *cost_out, int *iters_out)
{
    const int n = form == ORA_LM_RESIDUALS ? 2 * P->n_obs : P->n_obs;
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *rp = (double *)malloc(sizeof(double) * (size_t)n);
    double *rm = (double *)malloc(sizeof(double) * (size_t)n);
    double *Jm = (double *)malloc(sizeof(double) * 6 * (size_t)n);
    double *rt = (double *)malloc(sizeof(double) * (size_t)n);
    if (!r || !rp || !rm || !Jm || !rt) {
        free(r); free(rp); free(rm); free(Jm); free(rt);
        return ORA_EINVAL;
    }
    double x[6];
    memcpy(x, x0, sizeof x);
    int rc = ora_lm_residuals(P, x, form, r);
    double c = rc == ORA_OK ? sumsq(r, n) : INFINITY;
    double lam = 1e-3;
    int it = 0;
    while (rc == ORA_OK && it < max_iters && lam <= 1e16) {
        ++it;
        for (int j = 0; j < 6; ++j) {      /* central-difference Jacobian, column j */
            const double h = 1e-7 * fmax(fabs(x[j]), 0.1);
            double xp[6], xm[6];
            memcpy(xp, x, sizeof xp);
            memcpy(xm, x, sizeof xm);
            xp[j] = x[j] + h;
            xm[j] = x[j] - h;
            ora_lm_residuals(P, xp, form, rp);
            ora_lm_residuals(P, xm, form, rm);
            for (int i = 0; i < n; ++i) Jm[6 * (size_t)i + j] = (rp[i] - rm[i]) / (2.0 * h);
        }
        double A[36], g[6];
        for (int a = 0; a < 6; ++a) {
            g[a] = 0.0;
            for (int i = 0; i < n; ++i) g[a] += Jm[6 * (size_t)i + a] * r[i];
            for (int b = 0; b < 6; ++b) {
                A[6 * a + b] = 0.0;
                for (int i = 0; i < n; ++i) A[6 * a + b] += Jm[6 * (size_t)i + a] * Jm[6 * (size_t)i + b];
            }
        }
        int best = -1;
        double best_c = c, best_x[6];
        for (int t = 0; t < 8; ++t) {
            const double lt = lam * pow(10.0, (double)(t - 3));
            double d[6], xt[6];
            if (damped_solve(A, g, lt, d) != ORA_OK) continue;
            for (int q = 0; q < 6; ++q) xt[q] = x[q] + d[q];
            if (ora_lm_residuals(P, xt, form, rt) != ORA_OK) continue;
            const double ct = sumsq(rt, n);
            if (ct < best_c) {
                best_c = ct;
                best = t;
                memcpy(best_x, xt, sizeof best_x);
            }
        }
        if (best < 0) {
            lam = lam * 1e5;
            continue;
        }
        const double dec = c - best_c;
        memcpy(x, best_x, sizeof x);
        lam = lam * pow(10.0, (double)(best - 3)) / 10.0;
        ora_lm_residuals(P, x, form, r);
        const double c_old = c;
        c = best_c;
        if (dec <= 1e-10 * c_old) break;
    }
    memcpy(x_out, x, sizeof x);
    if (cost_out) *cost_out = c;
    if (iters_out) *iters_out = it;
    free(r); free(rp); free(rm); free(Jm); free(rt);
    return rc;
}

/* ------------------------------------------------------------------------------
 * Scenario helpers.  Bounds: a box about the chief's known state, +-r_max per
 * position axis and +-v_max per velocity axis (the sensor-feasible region of the
 * abstract, read as a box).  Observations: both bodies propagated with DOPRI5,
 * angles from Eqs. 5-9, plus the given noise.
 * ------------------------------------------------------------------------------ */
void ora_bounds_from_chief(const double chief[6], double r_max_km, double v_max_ms,
                           double L_km, double TU_s, double lo[6], double hi[6])
{
    const double dr = r_max_km / L_km;
    const double dv = (v_max_ms / 1000.0) / (L_km / TU_s);
    for (int d = 0; d < 3; ++d) {
        lo[d] = chief[d] - dr;
        hi[d] = chief[d] + dr;
        lo[d + 3] = chief[d + 3] - dv;
        hi[d + 3] = chief[d + 3] + dv;
    }
}

static int simulate_ctx(const dynctx *D, const double chief0[6], const double deputy0[6], int n,
                        const double *t, const ora_dopri5_opts *o, const double *noise,
                        double *ra, double *dec, double *rng, double *rc);

int ora_simulate_obs(double mu, const double chief0[6], const double deputy0[6], int n,
                     const double *t, const ora_dopri5_opts *o, const double *noise,
                     double *ra, double *dec, double *rng, double *rc)
{
    const dynctx D = {mu, 0.0, 0.0, 0};
    return simulate_ctx(&D, chief0, deputy0, n, t, o, noise, ra, dec, rng, rc);
}

int ora_simulate_obs_er3bp(double mu, double ecc, double f0, const double chief0[6],
                           const double deputy0[6], int n, const double *t, const ora_dopri5_opts *o,
                           const double *noise, double *ra, double *dec, double *rng, double *rc)
{
    const dynctx D = {mu, ecc, f0, 1};
    double *g = er3bp_grid(ecc, f0, n, t);
    if (!g) return ORA_EINVAL;
    const int r = simulate_ctx(&D, chief0, deputy0, n, g, o, noise, ra, dec, rng, rc);
    free(g);
    return r;
}

static int simulate_ctx(const dynctx *D, const double chief0[6], const double deputy0[6], int n,
                        const double *t, const ora_dopri5_opts *o, const double *noise,
                        double *ra, double *dec, double *rng, double *rc)
{
    double *sc = (double *)malloc(sizeof(double) * 6 * (size_t)n);
    double *sd = (double *)malloc(sizeof(double) * 6 * (size_t)n);
    if (!sc || !sd) { free(sc); free(sd); return ORA_EINVAL; }
    int r1 = propagate_dopri5_ctx(D, chief0, n, t, o, sc, NULL, NULL);
    int r2 = propagate_dopri5_ctx(D, deputy0, n, t, o, sd, NULL, NULL);
    if (r1 != ORA_OK || r2 != ORA_OK) { free(sc); free(sd); return ORA_EDIVERGED; }
    for (int k = 0; k < n; ++k) {
        const double rho[3] = {sd[6 * k] - sc[6 * k], sd[6 * k + 1] - sc[6 * k + 1],
                               sd[6 * k + 2] - sc[6 * k + 2]};
        double a, b, r;
        ora_angles(rho, &a, &b, &r);
        ra[k] = a + (noise ? noise[2 * k] : 0.0);
        dec[k] = b + (noise ? noise[2 * k + 1] : 0.0);
        if (rng) rng[k] = r;
        if (rc) {
            rc[3 * k] = sc[6 * k];
            rc[3 * k + 1] = sc[6 * k + 1];
            rc[3 * k + 2] = sc[6 * k + 2];
        }
    }
    free(sc);
    free(sd);
    return ORA_OK;
}
