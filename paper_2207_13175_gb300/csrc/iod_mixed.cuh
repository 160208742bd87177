// iod_mixed.cuh -- FP32 relative-state (Encke) propagation for the mixed-precision form.
//
// A particle is carried as its offset from the chief, delta = x_d - x_c, in FP32 with a
// compensated (Kahan) update.  RK4 is linear in its increments, so integrating delta with
// the stage-dependent right-hand side f(X_i + delta_i) - f(X_i), where X_i are the
// chief's own FP64 RK4 stage states, reproduces (up to rounding) the absolute RK4
// solution minus the chief's.  The gravity difference of each primary uses Encke's form
// (Battin, "An Introduction to the Mathematics and Methods of Astrodynamics", Encke's
// method):
//     (R + D)/|R + D|^3 - R/|R|^3 = [D - F(q) R] / |R + D|^3,
//     q = D.(2R + D)/|R|^2,  F(q) = (1 + q)^(3/2) - 1 = q (3 + 3q + q^2) / (1 + (1 + q)^(3/2)),
// which has no cancellation for |D| << |R|.  F is summed from its binomial series for
// |q| < 0.1 (truncation below 3e-9 relative) and from the closed ratio otherwise.  The
// Coriolis and centrifugal terms are linear in delta and exact.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>

namespace iod {
namespace mix {

// Chief data of one RK4 step: per stage i (0..3) and primary (E = Earth, M = Moon) the
// chief position relative to the primary R and |R|^2, plus 1/|R|^2.
struct __align__(16) Step {
    float4 e[4];    // (R_E, |R_E|^2) at stages 1..4
    float4 m[4];    // (R_M, |R_M|^2)
    float2 inv[4];  // (1/|R_E|^2, 1/|R_M|^2)
};
static_assert(sizeof(Step) == 160, "Step layout");

__device__ __forceinline__ float encke_F(float q)
{
    if (fabsf(q) < 0.1f) {
        // (1+q)^(3/2) - 1 = q (3/2 + 3/8 q - 1/16 q^2 + 3/128 q^3 - 3/256 q^4 + 7/1024 q^5 - 9/2048 q^6)
        float p = fmaf(q, -0.00439453125f, 0.0068359375f);
        p = fmaf(q, p, -0.01171875f);
        p = fmaf(q, p, 0.0234375f);
        p = fmaf(q, p, -0.0625f);
        p = fmaf(q, p, 0.375f);
        p = fmaf(q, p, 1.5f);
        return q * p;
    }
    const float opq = 1.0f + q;
    const float p32 = opq * sqrtf(opq);
    return q * fmaf(q, q + 3.0f, 3.0f) / (1.0f + p32);
}

// Gravity difference of one primary with gravitational parameter gm, accumulated into a.
__device__ __forceinline__ void grav_diff(float gm, float4 R, float iR2, float dx, float dy,
                                          float dz, float &ax, float &ay, float &az)
{
    const float s = fmaf(dx, fmaf(2.0f, R.x, dx), fmaf(dy, fmaf(2.0f, R.y, dy), dz * fmaf(2.0f, R.z, dz)));
    const float q = s * iR2;
    const float rho2 = R.w + s;                  // |R + D|^2
    const float ir = rsqrtf(rho2);
    const float c = gm * (ir * ir) * ir;         // gm / |R + D|^3
    const float F = encke_F(q);
    ax = fmaf(-c, fmaf(-F, R.x, dx), ax);
    ay = fmaf(-c, fmaf(-F, R.y, dy), ay);
    az = fmaf(-c, fmaf(-F, R.z, dz), az);
}

// Relative acceleration at one stage: linear rotating-frame terms plus both primaries.
__device__ __forceinline__ void rel_accel(float gmE, float gmM, float4 RE, float4 RM, float2 inv,
                                          float dx, float dy, float dz, float dvx, float dvy,
                                          float &ax, float &ay, float &az)
{
    ax = fmaf(2.0f, dvy, dx);
    ay = fmaf(-2.0f, dvx, dy);
    az = 0.0f;
    grav_diff(gmE, RE, inv.x, dx, dy, dz, ax, ay, az);
    grav_diff(gmM, RM, inv.y, dx, dy, dz, ax, ay, az);
}

// One RK4 step of delta (d: FP32 value, c: Kahan compensation, both [6]).  S points at
// the step's chief record in shared memory (every thread reads the same record, a
// broadcast); each stage reads its part just before use.
__device__ __forceinline__ void rk4_step_rel(float gmE, float gmM, const Step *__restrict__ S,
                                             float h, float hh, float h6, float d[6], float c[6])
{
    const float x = d[0], y = d[1], z = d[2], vx = d[3], vy = d[4], vz = d[5];
    float a1x, a1y, a1z, a2x, a2y, a2z, a3x, a3y, a3z, a4x, a4y, a4z;
    rel_accel(gmE, gmM, S->e[0], S->m[0], S->inv[0], x, y, z, vx, vy,
              a1x, a1y, a1z);
    const float v2x = fmaf(hh, a1x, vx), v2y = fmaf(hh, a1y, vy), v2z = fmaf(hh, a1z, vz);
    rel_accel(gmE, gmM, S->e[1], S->m[1], S->inv[1], fmaf(hh, vx, x),
              fmaf(hh, vy, y), fmaf(hh, vz, z), v2x, v2y, a2x, a2y, a2z);
    const float v3x = fmaf(hh, a2x, vx), v3y = fmaf(hh, a2y, vy), v3z = fmaf(hh, a2z, vz);
    rel_accel(gmE, gmM, S->e[2], S->m[2], S->inv[2], fmaf(hh, v2x, x),
              fmaf(hh, v2y, y), fmaf(hh, v2z, z), v3x, v3y, a3x, a3y, a3z);
    const float v4x = fmaf(h, a3x, vx), v4y = fmaf(h, a3y, vy), v4z = fmaf(h, a3z, vz);
    rel_accel(gmE, gmM, S->e[3], S->m[3], S->inv[3], fmaf(h, v3x, x),
              fmaf(h, v3y, y), fmaf(h, v3z, z), v4x, v4y, a4x, a4y, a4z);
    const float inc[6] = {h6 * fmaf(2.0f, v2x + v3x, vx + v4x), h6 * fmaf(2.0f, v2y + v3y, vy + v4y),
                          h6 * fmaf(2.0f, v2z + v3z, vz + v4z), h6 * fmaf(2.0f, a2x + a3x, a1x + a4x),
                          h6 * fmaf(2.0f, a2y + a3y, a1y + a4y), h6 * fmaf(2.0f, a2z + a3z, a1z + a4z)};
#pragma unroll
    for (int i = 0; i < 6; ++i) {   // Kahan: d carries the sum, c the lost low-order part
        const float yk = inc[i] - c[i];
        const float t = d[i] + yk;
        c[i] = (t - d[i]) - yk;
        d[i] = t;
    }
}

// Observed-direction constants of one epoch (FP32): sin/cos of the observed angles.
struct ObsDir {
    float sa, ca, sb, cb;
};

// Residuals of one epoch formed directly as small angles:
//   b_alpha = atan2(sin a~ rho_x - cos a~ rho_y, cos a~ rho_x + sin a~ rho_y)  (= wrap(a~ - a))
//   b_beta  = atan2(sin b~ rho_xy - cos b~ rho_z, cos b~ rho_xy + sin b~ rho_z) (= b~ - b)
// The epoch's weighted sum of squares is added to the FP64 total J.
__device__ __forceinline__ void add_epoch_cost_rel(float rx, float ry, float rz, const ObsDir &o,
                                                   float w_ra, float w_dec, int quartic,
                                                   int use_range, float rng_obs, float w_rng,
                                                   double &J)
{
    const float rxy2 = fmaf(rx, rx, ry * ry);
    const float r2 = fmaf(rz, rz, rxy2);
    if (!(r2 >= 1e-30f) || !isfinite(r2)) {
        J = CUDART_INF;
        return;
    }
    const float rxy = sqrtf(rxy2);
    const float ba = atan2f(fmaf(o.sa, rx, -o.ca * ry), fmaf(o.ca, rx, o.sa * ry));
    const float bb = atan2f(fmaf(o.sb, rxy, -o.cb * rz), fmaf(o.cb, rxy, o.sb * rz));
    float Jk = fmaf(ba * w_ra, ba, bb * w_dec * bb);
    if (use_range) {
        const float br = rng_obs - sqrtf(r2);
        Jk = fmaf(br * w_rng, br, Jk);
    }
    const double Jd = (double)Jk;
    J += quartic ? Jd * Jd : Jd;
}

}  // namespace mix
}  // namespace iod
