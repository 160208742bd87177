// iod_device.cuh -- device arithmetic of the PSO-IOD hot path (sm_103a, FP64).
//
// One thread owns one particle: its 6-D state, the Runge-Kutta stages and the
// running cost stay in registers; the observation table is read from shared memory
// (every thread reads the same entry at the same time, a broadcast).
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

namespace iod {
namespace dev {

// ---------------------------------------------------------------------------------
// CR3BP acceleration, Eqs. 1-3 (rotating barycentric frame, nondimensional).
// m / r^3 of each primary from m_over_r3.
// ---------------------------------------------------------------------------------
struct Dyn {
    double mu;          // mass parameter
    double omu;         // 1 - mu
    double e = 0.0;     // ER3BP: eccentricity of the primaries' orbit
    double f0 = 0.0;    // ER3BP: true anomaly where the independent variable is 0
    int er = 0;         // 1: elliptic problem (pulsating frame, independent variable f - f0)
};

// m / r^3 from s = r^2.  A hardware estimate y0 of s^(-1/2) (rsqrt.approx.ftz.f64;
// measured relative error below 2^-20 over s in [1e-5, 1e2]) is refined in one step by
// the binomial series (1 - e)^(-3/2) = 1 + 3e/2 + 15e^2/8 + 35e^3/16 + ..., with
// e = 1 - s y0^2 the estimate's defect: m / r^3 = m y0^3 (1 + e (3/2 + 15e/8)).  With
// |e| < 2^-18.9 the dropped terms stay below 1.4e-17 relative (an eighth of an FP64
// unit in the last place); measured during development against a quad-precision
// reference, the result is within 2 units of 2^-53 (the library's reciprocal square
// root, cubed: within 5).  Seven FP64 operations and one special-function instruction.
__device__ __forceinline__ double m_over_r3(double s, double m)
{
    double y0;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y0) : "d"(s));
    const double y2 = y0 * y0;
    const double e = fma(-s, y2, 1.0);
    const double p = fma(1.875, e, 1.5);
    const double c = m * (y2 * y0);
    return fma(c, e * p, c);
}

__device__ __forceinline__ void accel(const Dyn &D, double x, double y, double z, double vx,
                                      double vy, double &ax, double &ay, double &az)
{
    const double d1 = x + D.mu;          // x + mu
    const double d2 = x - D.omu;         // x - (1 - mu)
    const double yz = fma(y, y, z * z);
    const double r1s = fma(d1, d1, yz);
    const double r2s = fma(d2, d2, yz);
    const double g1 = m_over_r3(r1s, D.omu);    // (1 - mu) / r1^3
    const double g2 = m_over_r3(r2s, D.mu);     // mu / r2^3
    const double gs = g1 + g2;
    ax = fma(-g1, d1, fma(-g2, d2, fma(2.0, vy, x)));
    ay = fma(-gs, y, fma(-2.0, vx, y));
    az = -gs * z;
}

// ER3BP acceleration in the pulsating rotating frame with respect to the true anomaly f
// (Szebehely's form): a = Coriolis + grad(omega), omega = [(x^2 + y^2 - e z^2 cos f)/2 +
// (1-mu)/r1 + mu/r2] / (1 + e cos f).
// The same with e cos f and 1/(1 + e cos f) given.
__device__ __forceinline__ void accel_er_c(const Dyn &D, double ecf, double scale, double x, double y,
                                           double z, double vx, double vy, double &ax, double &ay,
                                           double &az)
{
    const double d1 = x + D.mu;
    const double d2 = x - D.omu;
    const double yz = fma(y, y, z * z);
    const double r1s = fma(d1, d1, yz);
    const double r2s = fma(d2, d2, yz);
    const double g1 = m_over_r3(r1s, D.omu);
    const double g2 = m_over_r3(r2s, D.mu);
    const double gs = g1 + g2;
    ax = fma(2.0, vy, fma(-g1, d1, fma(-g2, d2, x)) * scale);
    ay = fma(-2.0, vx, fma(-gs, y, y) * scale);
    az = -(ecf + gs) * z * scale;
}

__device__ __forceinline__ void accel_er(const Dyn &D, double f, double x, double y, double z,
                                         double vx, double vy, double &ax, double &ay, double &az)
{
    const double ecf = D.e * cos(f);
    const double scale = 1.0 / (1.0 + ecf);
    const double d1 = x + D.mu;
    const double d2 = x - D.omu;
    const double yz = fma(y, y, z * z);
    const double r1s = fma(d1, d1, yz);
    const double r2s = fma(d2, d2, yz);
    const double g1 = m_over_r3(r1s, D.omu);
    const double g2 = m_over_r3(r2s, D.mu);
    const double gs = g1 + g2;
    ax = fma(2.0, vy, fma(-g1, d1, fma(-g2, d2, x)) * scale);
    ay = fma(-2.0, vx, fma(-gs, y, y) * scale);
    az = -(ecf + gs) * z * scale;
}

// right-hand side at independent variable tv (read only by the elliptic problem,
// ER = 1, a compile-time choice)
template <int ER = 0>
__device__ __forceinline__ void rhs(const Dyn &D, double tv, const double s[6], double ds[6])
{
    ds[0] = s[3];
    ds[1] = s[4];
    ds[2] = s[5];
    if (ER)
        accel_er(D, D.f0 + tv, s[0], s[1], s[2], s[3], s[4], ds[3], ds[4], ds[5]);
    else
        accel(D, s[0], s[1], s[2], s[3], s[4], ds[3], ds[4], ds[5]);
}

__device__ __forceinline__ void rhs(const Dyn &D, const double s[6], double ds[6])
{
    rhs<0>(D, 0.0, s, ds);
}

// Step constants of RK4 with step h: h/2, h/6 and the products the folded z stages use.
struct RkH {
    double h, hh, h6, hq, hhh, h26;     // h, h/2, h/6, (h/2)^2, h^2/2, h^2/6
};

__device__ __forceinline__ RkH rk_h(double h)
{
    const double hh = 0.5 * h;
    return RkH{h, hh, h / 6.0, hh * hh, h * hh, (h * h) / 6.0};
}

// Classical RK4 step of the first-order system x' = v, v' = a(x, v).  The position
// stages are the velocity stages, so only accelerations are evaluated:
// acc(stage, x, y, z, vx, vy, ax, ay, az) at stages 0..3 (t, t + h/2 twice, t + h).
// The acceleration reads no z velocity, so z's stage velocities are folded into its
// positions: z + (h/2) v2z = z2 + (h/2)^2 a1z, z + h v3z = (z + h vz) + (h^2/2) a2z, and
// the 1-2-2-1 combination of the z velocities gives z + h vz + (h^2/6)(a1z + a2z +
// a3z); the same step in exact arithmetic, three FP64 operations fewer.
template <class Acc>
__device__ __forceinline__ void rk4_core(const RkH &C, double s[6], Acc &&acc)
{
    const double x = s[0], y = s[1], z = s[2], vx = s[3], vy = s[4], vz = s[5];
    double a1x, a1y, a1z, a2x, a2y, a2z, a3x, a3y, a3z, a4x, a4y, a4z;
    acc(0, x, y, z, vx, vy, a1x, a1y, a1z);
    const double v2x = fma(C.hh, a1x, vx), v2y = fma(C.hh, a1y, vy);
    const double z2 = fma(C.hh, vz, z);
    acc(1, fma(C.hh, vx, x), fma(C.hh, vy, y), z2, v2x, v2y, a2x, a2y, a2z);
    const double v3x = fma(C.hh, a2x, vx), v3y = fma(C.hh, a2y, vy);
    acc(2, fma(C.hh, v2x, x), fma(C.hh, v2y, y), fma(C.hq, a1z, z2), v3x, v3y, a3x, a3y, a3z);
    const double v4x = fma(C.h, a3x, vx), v4y = fma(C.h, a3y, vy);
    const double zh = fma(C.h, vz, z);
    acc(3, fma(C.h, v3x, x), fma(C.h, v3y, y), fma(C.hhh, a2z, zh), v4x, v4y, a4x, a4y, a4z);
    s[0] = fma(C.h6, fma(2.0, v2x + v3x, vx + v4x), x);
    s[1] = fma(C.h6, fma(2.0, v2y + v3y, vy + v4y), y);
    s[2] = fma(C.h26, a1z + a2z + a3z, zh);
    s[3] = fma(C.h6, fma(2.0, a2x + a3x, a1x + a4x), vx);
    s[4] = fma(C.h6, fma(2.0, a2y + a3y, a1y + a4y), vy);
    s[5] = fma(C.h6, fma(2.0, a2z + a3z, a1z + a4z), vz);
}

// RK4 step of the circular problem.
__device__ __forceinline__ void rk4_step(const Dyn &D, const RkH &C, double s[6])
{
    rk4_core(C, s, [&](int, double x, double y, double z, double vx, double vy, double &ax,
                       double &ay, double &az) { accel(D, x, y, z, vx, vy, ax, ay, az); });
}

// Two threads per particle: both lanes of a pair hold the particle's state, each
// evaluates one primary's attraction (even lane the Earth, odd lane the Moon) and they
// swap it; every lane then forms the acceleration exactly as accel() does, so the pair
// reproduces the one-thread result bit for bit.  mask: the lanes taking part in the
// exchange, the whole warp when every pair runs the same steps (RK4) or the pair alone
// when pairs follow different control flow (adaptive steps).
__device__ __forceinline__ void accel_pair(const Dyn &D, bool odd, double x, double y, double z,
                                           double vx, double vy, double &ax, double &ay, double &az,
                                           unsigned int mask = 0xffffffffu)
{
    const double dm = odd ? x - D.omu : x + D.mu;
    const double gm = odd ? D.mu : D.omu;
    const double yz = fma(y, y, z * z);
    const double rs = fma(dm, dm, yz);
    const double g = m_over_r3(rs, gm);
    const double go = __shfl_xor_sync(mask, g, 1);
    const double d1 = odd ? x + D.mu : dm;
    const double d2 = odd ? dm : x - D.omu;
    const double g1 = odd ? go : g, g2 = odd ? g : go;
    const double gs = g1 + g2;
    ax = fma(-g1, d1, fma(-g2, d2, fma(2.0, vy, x)));
    ay = fma(-gs, y, fma(-2.0, vx, y));
    az = -gs * z;
}

__device__ __forceinline__ void rk4_step_pair(const Dyn &D, bool odd, const RkH &C, double s[6],
                                              unsigned int mask = 0xffffffffu)
{
    rk4_core(C, s, [&](int, double x, double y, double z, double vx, double vy, double &ax,
                       double &ay, double &az) { accel_pair(D, odd, x, y, z, vx, vy, ax, ay, az, mask); });
}

// ER3BP step whose stages sit at true anomalies f, f + h/2 (twice) and f + h, given
// ca = cos f, cm = cos(f + h/2), ce = cos(f + h) (the same for every particle).
__device__ __forceinline__ void rk4_step_er(const Dyn &D, double ca, double cm, double ce, const RkH &C,
                                            double s[6])
{
    const double ea = D.e * ca, em = D.e * cm, ee = D.e * ce;
    const double sa = 1.0 / (1.0 + ea), sm = 1.0 / (1.0 + em), se = 1.0 / (1.0 + ee);
    rk4_core(C, s, [&](int st, double x, double y, double z, double vx, double vy, double &ax,
                       double &ay, double &az) {
        const double ec = st == 0 ? ea : (st == 3 ? ee : em);
        const double sc = st == 0 ? sa : (st == 3 ? se : sm);
        accel_er_c(D, ec, sc, x, y, z, vx, vy, ax, ay, az);
    });
}

// The same step as rk4_step (identical arithmetic), also reporting the four stage
// positions at which the acceleration was evaluated.
__device__ __forceinline__ void rk4_step_stages(const Dyn &D, const RkH &C, double s[6], double P[4][3])
{
    rk4_core(C, s, [&](int st, double x, double y, double z, double vx, double vy, double &ax,
                       double &ay, double &az) {
        P[st][0] = x;
        P[st][1] = y;
        P[st][2] = z;
        accel(D, x, y, z, vx, vy, ax, ay, az);
    });
}

// ---------------------------------------------------------------------------------
// Dormand-Prince 5(4): tableau of Dormand & Prince (1980); error weights E = b - bhat;
// continuous extension of Shampine (1986) as given in Hairer, Norsett & Wanner I, II.6.
// ---------------------------------------------------------------------------------
namespace dp {
constexpr double C2 = 1.0 / 5.0, C3 = 3.0 / 10.0, C4 = 4.0 / 5.0, C5 = 8.0 / 9.0;
constexpr double A21 = 1.0 / 5.0;
constexpr double A31 = 3.0 / 40.0, A32 = 9.0 / 40.0;
constexpr double A41 = 44.0 / 45.0, A42 = -56.0 / 15.0, A43 = 32.0 / 9.0;
constexpr double A51 = 19372.0 / 6561.0, A52 = -25360.0 / 2187.0, A53 = 64448.0 / 6561.0,
                 A54 = -212.0 / 729.0;
constexpr double A61 = 9017.0 / 3168.0, A62 = -355.0 / 33.0, A63 = 46732.0 / 5247.0,
                 A64 = 49.0 / 176.0, A65 = -5103.0 / 18656.0;
constexpr double B1 = 35.0 / 384.0, B3 = 500.0 / 1113.0, B4 = 125.0 / 192.0,
                 B5 = -2187.0 / 6784.0, B6 = 11.0 / 84.0;
constexpr double E1 = 71.0 / 57600.0, E3 = -71.0 / 16695.0, E4 = 71.0 / 1920.0,
                 E5 = -17253.0 / 339200.0, E6 = 22.0 / 525.0, E7 = -1.0 / 40.0;
}  // namespace dp

// Stage derivatives kept for the continuous extension (k2 is not needed there).
struct DpStages {
    double k1[6], k3[6], k4[6], k5[6], k6[6], k7[6];
};

// The right-hand side with the two primaries' attractions split over a lane pair
// (accel_pair; circular problem): the same values as rhs<0> in both lanes.
// Pairs may take different numbers of steps here, so the exchange names the pair alone.
__device__ __forceinline__ void rhs_pair(const Dyn &D, bool odd, const double s[6], double ds[6])
{
    ds[0] = s[3];
    ds[1] = s[4];
    ds[2] = s[5];
    const unsigned int pair_mask = 3u << ((threadIdx.x & 31u) & ~1u);
    accel_pair(D, odd, s[0], s[1], s[2], s[3], s[4], ds[3], ds[4], ds[5], pair_mask);
}

// rhs<ER> in one thread (PAIR = 0) or over a lane pair (PAIR = 1, circular problem).
template <int ER, int PAIR>
__device__ __forceinline__ void rhs_any(const Dyn &D, bool odd, double tv, const double s[6], double ds[6])
{
    if (PAIR)
        rhs_pair(D, odd, s, ds);
    else
        rhs<ER>(D, tv, s, ds);
}

// One attempt from s with step h; k1 = f(s) on entry (K.k1).  Writes s1 and the
// stages, returns the RMS error norm scaled by atol + rtol max(|y|, |y1|).
// tc: the independent variable at the start (stage i sits at tc + c_i h; only the
// elliptic problem reads it).  PAIR = 1: the right-hand sides over a lane pair.
template <int ER = 0, int PAIR = 0>
__device__ __forceinline__ double dopri5_attempt(const Dyn &D, double tc, double h, const double s[6],
                                                 DpStages &K, double s1[6], double rtol,
                                                 double atol, bool odd = false)
{
    using namespace dp;
    double t[6], k2[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) t[i] = fma(h, A21 * K.k1[i], s[i]);
    rhs_any<ER, PAIR>(D, odd, tc + C2 * h, t, k2);
#pragma unroll
    for (int i = 0; i < 6; ++i) t[i] = fma(h, fma(A31, K.k1[i], A32 * k2[i]), s[i]);
    rhs_any<ER, PAIR>(D, odd, tc + C3 * h, t, K.k3);
#pragma unroll
    for (int i = 0; i < 6; ++i)
        t[i] = fma(h, fma(A41, K.k1[i], fma(A42, k2[i], A43 * K.k3[i])), s[i]);
    rhs_any<ER, PAIR>(D, odd, tc + C4 * h, t, K.k4);
#pragma unroll
    for (int i = 0; i < 6; ++i)
        t[i] = fma(h, fma(A51, K.k1[i], fma(A52, k2[i], fma(A53, K.k3[i], A54 * K.k4[i]))), s[i]);
    rhs_any<ER, PAIR>(D, odd, tc + C5 * h, t, K.k5);
#pragma unroll
    for (int i = 0; i < 6; ++i)
        t[i] = fma(h, fma(A61, K.k1[i], fma(A62, k2[i], fma(A63, K.k3[i],
                   fma(A64, K.k4[i], A65 * K.k5[i])))), s[i]);
    rhs_any<ER, PAIR>(D, odd, tc + h, t, K.k6);
#pragma unroll
    for (int i = 0; i < 6; ++i)
        s1[i] = fma(h, fma(B1, K.k1[i], fma(B3, K.k3[i], fma(B4, K.k4[i],
                    fma(B5, K.k5[i], B6 * K.k6[i])))), s[i]);
    rhs_any<ER, PAIR>(D, odd, tc + h, s1, K.k7);
    // e_i / sc_i for the six components with one division: 1 / (sc_0 ... sc_5) times the
    // product of the other five scales (prefix and suffix products; every sc_i >= atol,
    // and the products stay far inside the double range for any finite state).  Each
    // quotient is then within a few units of the last place of e_i / sc_i, so the error
    // norm -- and the step's acceptance -- match the plain quotients except for a norm
    // within ~1e-15 of 1.
    double e[6], sc[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        e[i] = h * fma(E1, K.k1[i], fma(E3, K.k3[i], fma(E4, K.k4[i],
                   fma(E5, K.k5[i], fma(E6, K.k6[i], E7 * K.k7[i])))));
        sc[i] = fma(rtol, fmax(fabs(s[i]), fabs(s1[i])), atol);
    }
    const double p01 = sc[0] * sc[1], p012 = p01 * sc[2], p0123 = p012 * sc[3], p01234 = p0123 * sc[4];
    const double s45 = sc[4] * sc[5], s345 = sc[3] * s45, s2345 = sc[2] * s345, s12345 = sc[1] * s2345;
    const double inv = 1.0 / (p01234 * sc[5]);
    const double o[6] = {s12345, sc[0] * s2345, p01 * s345, p012 * s45, p0123 * sc[5], p01234};
    double sum = 0.0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const double q = e[i] * (inv * o[i]);
        sum = fma(q, q, sum);
    }
    return sqrt(sum * (1.0 / 6.0));
}

// Continuous extension: y(t + th h) = s + h sum_j b_j(th) k_j with Shampine's weights,
// expanded once into powers of th (exact rationals of the tableau's published form, each
// rounded once to double here) and evaluated by Horner's rule: b_1 = th + th^2 p_1(th),
// b_j = th^2 p_j(th) for j = 3..7 with cubic p_j.  The same interpolant as the factored
// form (weights within ~2e-15 of their magnitude), with no divisions.
namespace dpd {
constexpr double B12 = -4034104133.0 / 1410260304.0, B13 = 105330401.0 / 33982176.0,
                 B14 = -13107642775.0 / 11282082432.0, B15 = 6542295.0 / 470086768.0;
constexpr double B32 = 132343189600.0 / 32700410799.0, B33 = -833316000.0 / 131326951.0,
                 B34 = 91412856700.0 / 32700410799.0, B35 = -523383600.0 / 10900136933.0;
constexpr double B42 = -115792950.0 / 29380423.0, B43 = 185270875.0 / 16991088.0,
                 B44 = -12653452475.0 / 1880347072.0, B45 = 98134425.0 / 235043384.0;
constexpr double B52 = 70805911779.0 / 24914598704.0, B53 = -4531260609.0 / 600351776.0,
                 B54 = 988140236175.0 / 199316789632.0, B55 = -14307999165.0 / 24914598704.0;
constexpr double B62 = -331320693.0 / 205662961.0, B63 = 31361737.0 / 7433601.0,
                 B64 = -2426908385.0 / 822651844.0, B65 = 97305120.0 / 205662961.0;
constexpr double B72 = 44764047.0 / 29380423.0, B73 = -1532549.0 / 353981.0,
                 B74 = 90730570.0 / 29380423.0, B75 = -8293050.0 / 29380423.0;
}  // namespace dpd

__device__ __forceinline__ void dopri5_dense(double h, const double s[6], const DpStages &K,
                                             double th, double out[6])
{
    using namespace dpd;
    const double t2 = th * th;
    const double b1 = fma(t2, fma(th, fma(th, fma(th, B15, B14), B13), B12), th);
    const double b3 = t2 * fma(th, fma(th, fma(th, B35, B34), B33), B32);
    const double b4 = t2 * fma(th, fma(th, fma(th, B45, B44), B43), B42);
    const double b5 = t2 * fma(th, fma(th, fma(th, B55, B54), B53), B52);
    const double b6 = t2 * fma(th, fma(th, fma(th, B65, B64), B63), B62);
    const double b7 = t2 * fma(th, fma(th, fma(th, B75, B74), B73), B72);
#pragma unroll
    for (int i = 0; i < 6; ++i)
        out[i] = fma(h, fma(b1, K.k1[i], fma(b3, K.k3[i], fma(b4, K.k4[i],
                     fma(b5, K.k5[i], fma(b6, K.k6[i], b7 * K.k7[i]))))), s[i]);
}

// err^(-1/5) for the step-size controller: an FP32 estimate (__powf, relative error
// ~1e-6) refined by two Newton steps for y^-5 = err, y <- y + y (1 - err y^5) / 5, which
// converge quadratically to within ~2 units of the last place -- the accuracy of a
// library power function, at a fraction of its FP64 work.  err below 1e-30 gives +inf
// and above 1e30 gives 0 (the controller clamps both).
__device__ __forceinline__ double inv_fifth_root(double err)
{
    if (!(err >= 1e-30)) return CUDART_INF;
    if (err > 1e30) return 0.0;
    double y = (double)__powf((float)err, -0.2f);
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const double y2 = y * y;
        const double y5 = y2 * y2 * y;
        y = fma(0.2 * y, fma(-err, y5, 1.0), y);
    }
    return y;
}

// ---------------------------------------------------------------------------------
// Measurement residual and cost term of one epoch, Eqs. 5-13.
// ---------------------------------------------------------------------------------
struct CostW {
    double w_ra, w_dec, w_rng;   // 1/sigma^2 (w_rng = 0 for angles only)
    int quartic;                 // J_k squared before summing (Eqs. 11, 13 literal)
    int use_range;
};

// Adds epoch k's term to J; a degenerate line of sight or a non-finite value gives +inf.
__device__ __forceinline__ void add_epoch_cost(const CostW &W, double rx, double ry, double rz,
                                               double ra_obs, double dec_obs, double rng_obs,
                                               double &J)
{
    const double r = sqrt(fma(rx, rx, fma(ry, ry, rz * rz)));
    if (!(r >= 1e-15) || !isfinite(r)) {
        J = CUDART_INF;
        return;
    }
    // Eqs. 6-8: L = rho / |rho|, alpha = atan2(L_y, L_x), beta = asin(L_z); the two-argument
    // arctangent does not depend on the common scale of its arguments, so alpha is taken
    // from rho directly
    const double alpha = atan2(ry, rx);
    const double beta = asin(rz / r);
    // the azimuth residual reduced to [-pi, pi] (the IEEE remainder by 2 pi): for
    // pi < |b| < 3 pi that is b -/+ 2 pi, exact by Sterbenz's lemma, as the remainder is
    constexpr double kTwoPi = 6.283185307179586, kPi = 3.141592653589793;
    double b_ra = ra_obs - alpha;
    if (!(fabs(b_ra) <= kPi))
        b_ra = fabs(b_ra) < 3.0 * kPi ? b_ra - copysign(kTwoPi, b_ra) : remainder(b_ra, kTwoPi);
    const double b_dec = dec_obs - beta;
    double Jk = fma(b_ra * W.w_ra, b_ra, b_dec * W.w_dec * b_dec);
    if (W.use_range) {
        const double b_rng = rng_obs - r;
        Jk = fma(b_rng * W.w_rng, b_rng, Jk);
    }
    J += W.quartic ? Jk * Jk : Jk;
}

// ---------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) and the 53-bit uniform double.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// ((a >> 5) 2^26 + (b >> 6)) 2^-53: every operation is exact.
__device__ __forceinline__ double u01(uint32_t a, uint32_t b)
{
    return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) * (1.0 / 9007199254740992.0);
}

// ---------------------------------------------------------------------------------
// (cost, index) argmin with the lowest index winning ties; NaN is folded to +inf by
// the callers before they get here.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ bool better(double ja, int ia, double jb, int ib)
{
    return ja < jb || (ja == jb && ia < ib);
}

__device__ __forceinline__ void warp_argmin(double &j, int &i)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double oj = __shfl_xor_sync(0xffffffffu, j, off);
        const int oi = __shfl_xor_sync(0xffffffffu, i, off);
        if (better(oj, oi, j, i)) {
            j = oj;
            i = oi;
        }
    }
}

}  // namespace dev
}  // namespace iod
