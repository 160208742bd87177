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

// Chief data of one RK4 step.  Per stage i (0..3) the chief position relative to the
// Earth and to the Moon, stored doubled (T = 2R, exact in binary), with |R|^2 and
// 1/|R|^2, laid out so that each quantity of the two primaries forms a float2 pair
// (Earth in .x, Moon in .y): the two gravity terms are evaluated together with packed
// FP32x2 instructions (FFMA2/FMUL2/FADD2, one issue slot for two lanes' worth of work).
struct __align__(16) Step {
    float4 txy[4];  // (2 R_E.x, 2 R_M.x, 2 R_E.y, 2 R_M.y)
    float4 tzr[4];  // (2 R_E.z, 2 R_M.z, |R_E|^2, |R_M|^2)
    float2 inv[4];  // (1/|R_E|^2, 1/|R_M|^2)
};
static_assert(sizeof(Step) == 160, "Step layout");

// the Moon's position relative to the chief at a step's first stage, R_M
__device__ __forceinline__ float3 moon_rel(const Step &S)
{
    return make_float3(0.5f * S.txy[0].y, 0.5f * S.txy[0].w, 0.5f * S.tzr[0].y);
}

// rsqrt.approx with denormals flushed: one special-function instruction (relative error
// below 2^-22; the arguments here are squared distances far from the denormal range)
__device__ __forceinline__ float rsqrt_ftz(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// F(q)/2 = ((1 + q)^(3/2) - 1)/2, closed ratio (no cancellation for any q > -1)
__device__ __forceinline__ float encke_F_half_closed(float q)
{
    const float opq = 1.0f + q;
    const float p32 = opq * sqrtf(opq);
    return 0.5f * q * fmaf(q, q + 3.0f, 3.0f) / (1.0f + p32);
}

// F(q)/2 for the (Earth, Moon) pair: its binomial series
//   q (3/2 + 3/8 q - 1/16 q^2 + 3/128 q^3 - 3/256 q^4 + 7/1024 q^5 - 9/2048 q^6) / 2
// (truncation below 3e-9 of F for |q| < 0.1) on both lanes at once while both |q| < 0.1,
// else lane by lane, the closed ratio where |q| >= 0.1.
__device__ __forceinline__ float2 encke_F_half2(float2 q)
{
    if (fabsf(q.x) < 0.1f && fabsf(q.y) < 0.1f) {
        float2 p = __ffma2_rn(q, f2(-0.002197265625f), f2(0.00341796875f));
        p = __ffma2_rn(q, p, f2(-0.005859375f));
        p = __ffma2_rn(q, p, f2(0.01171875f));
        p = __ffma2_rn(q, p, f2(-0.03125f));
        p = __ffma2_rn(q, p, f2(0.1875f));
        p = __ffma2_rn(q, p, f2(0.75f));
        return __fmul2_rn(q, p);
    }    float2 r;
    const float qq[2] = {q.x, q.y};
    float rr[2];
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        const float x = qq[l];
        if (fabsf(x) < 0.1f) {
            float p = fmaf(x, -0.002197265625f, 0.00341796875f);
            p = fmaf(x, p, -0.005859375f);
            p = fmaf(x, p, 0.01171875f);
            p = fmaf(x, p, -0.03125f);
            p = fmaf(x, p, 0.1875f);
            p = fmaf(x, p, 0.75f);
            rr[l] = x * p;
        } else {
            rr[l] = encke_F_half_closed(x);
        }
    }
    r.x = rr[0];
    r.y = rr[1];
    return r;
}

// Relative acceleration at one stage: linear rotating-frame terms plus the gravity
// differences of both primaries, [D - F R] gm/|R + D|^3 each, with
// s = 2 R.D + |D|^2 = |R + D|^2 - |R|^2 and q = s/|R|^2; gm = (gm_E, gm_M).
__device__ __forceinline__ void rel_accel(float2 gm, float4 txy, float4 tzr, float2 inv, float dx,
                                          float dy, float dz, float dvx, float dvy, float &ax,
                                          float &ay, float &az)
{
    const float2 TX = make_float2(txy.x, txy.y), TY = make_float2(txy.z, txy.w);
    const float2 TZ = make_float2(tzr.x, tzr.y), R2 = make_float2(tzr.z, tzr.w);
    const float D2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    float2 s = __ffma2_rn(TZ, f2(dz), f2(D2));
    s = __ffma2_rn(TY, f2(dy), s);
    s = __ffma2_rn(TX, f2(dx), s);
    const float2 q = __fmul2_rn(s, inv);
    const float2 rho2 = __fadd2_rn(R2, s);                    // |R + D|^2
    const float2 ir = make_float2(rsqrt_ftz(rho2.x), rsqrt_ftz(rho2.y));
    const float2 nc = __fmul2_rn(__fmul2_rn(gm, __fmul2_rn(ir, ir)), make_float2(-ir.x, -ir.y));
    const float2 Fh = encke_F_half2(q);                        // F/2, multiplies T = 2R
    const float2 nF = make_float2(-Fh.x, -Fh.y);
    const float2 wx = __ffma2_rn(nF, TX, f2(dx));              // D - F R, per primary
    const float2 wy = __ffma2_rn(nF, TY, f2(dy));
    const float2 wz = __ffma2_rn(nF, TZ, f2(dz));
    const float2 px = __ffma2_rn(nc, wx, make_float2(fmaf(2.0f, dvy, dx), 0.0f));
    const float2 py = __ffma2_rn(nc, wy, make_float2(fmaf(-2.0f, dvx, dy), 0.0f));
    const float2 pz = __fmul2_rn(nc, wz);
    ax = px.x + px.y;
    ay = py.x + py.y;
    az = pz.x + pz.y;
}

// One RK4 step of delta (d: FP32 value, c: Kahan compensation, both [6]).  S points at
// the step's chief record in shared memory (every thread reads the same record, a
// broadcast); each stage reads its part just before use.
__device__ __forceinline__ void rk4_step_rel(float2 gm, const Step *__restrict__ S, float h, float hh,
                                             float h6, float d[6], float c[6])
{
    const float x = d[0], y = d[1], z = d[2], vx = d[3], vy = d[4], vz = d[5];
    float a1x, a1y, a1z, a2x, a2y, a2z, a3x, a3y, a3z, a4x, a4y, a4z;
    rel_accel(gm, S->txy[0], S->tzr[0], S->inv[0], x, y, z, vx, vy, a1x, a1y, a1z);
    const float v2x = fmaf(hh, a1x, vx), v2y = fmaf(hh, a1y, vy), v2z = fmaf(hh, a1z, vz);
    rel_accel(gm, S->txy[1], S->tzr[1], S->inv[1], fmaf(hh, vx, x), fmaf(hh, vy, y), fmaf(hh, vz, z),
              v2x, v2y, a2x, a2y, a2z);
    const float v3x = fmaf(hh, a2x, vx), v3y = fmaf(hh, a2y, vy), v3z = fmaf(hh, a2z, vz);
    rel_accel(gm, S->txy[2], S->tzr[2], S->inv[2], fmaf(hh, v2x, x), fmaf(hh, v2y, y), fmaf(hh, v2z, z),
              v3x, v3y, a3x, a3y, a3z);
    const float v4x = fmaf(h, a3x, vx), v4y = fmaf(h, a3y, vy), v4z = fmaf(h, a3z, vz);
    rel_accel(gm, S->txy[3], S->tzr[3], S->inv[3], fmaf(h, v3x, x), fmaf(h, v3y, y), fmaf(h, v3z, z),
              v4x, v4y, a4x, a4y, a4z);
    // increments as three pairs: (x, y), (z, vx), (vy, vz)
    const float2 sA = __fadd2_rn(make_float2(v2x, v2y), make_float2(v3x, v3y));
    const float2 sB = __fadd2_rn(make_float2(v2z, a2x), make_float2(v3z, a3x));
    const float2 sC = __fadd2_rn(make_float2(a2y, a2z), make_float2(a3y, a3z));
    const float2 eA = __fadd2_rn(make_float2(vx, vy), make_float2(v4x, v4y));
    const float2 eB = __fadd2_rn(make_float2(vz, a1x), make_float2(v4z, a4x));
    const float2 eC = __fadd2_rn(make_float2(a1y, a1z), make_float2(a4y, a4z));
    const float2 iA = __fmul2_rn(f2(h6), __ffma2_rn(f2(2.0f), sA, eA));
    const float2 iB = __fmul2_rn(f2(h6), __ffma2_rn(f2(2.0f), sB, eB));
    const float2 iC = __fmul2_rn(f2(h6), __ffma2_rn(f2(2.0f), sC, eC));
    const float2 inc[3] = {iA, iB, iC};
#pragma unroll
    for (int i = 0; i < 3; ++i) {   // Kahan: d carries the sum, c the lost low-order part
        const float2 dd = make_float2(d[2 * i], d[2 * i + 1]);
        const float2 cc = make_float2(c[2 * i], c[2 * i + 1]);
        const float2 yk = __fadd2_rn(inc[i], make_float2(-cc.x, -cc.y));
        const float2 t = __fadd2_rn(dd, yk);
        const float2 lost = __fadd2_rn(__fadd2_rn(t, make_float2(-dd.x, -dd.y)), make_float2(-yk.x, -yk.y));
        d[2 * i] = t.x;
        d[2 * i + 1] = t.y;
        c[2 * i] = lost.x;
        c[2 * i + 1] = lost.y;
    }
}

// Observed-direction constants of one epoch (FP32): sin/cos of the observed angles.
struct ObsDir {
    float sa, ca, sb, cb;
};

// The exact product a b = p + e (the rounding error e by one FMA).  The double-float
// helpers below use the _rn intrinsics for every product and sum that is part of an
// error-free transformation: the compiler never fuses those into an FMA, which would
// change the rounding the transformation accounts for.
__device__ __forceinline__ float two_prod(float a, float b, float &e)
{
    const float p = __fmul_rn(a, b);
    e = fmaf(a, b, -p);
    return p;
}

// sn (u - uc) - cs (v - vc) for offsets carried as value u and compensation uc (the
// Kahan pair of the propagation), in double-float arithmetic: the two products are
// split exactly (two_prod), their leading parts differ by exactly their difference when
// they lie within a factor of two (Sterbenz), and the low-order terms are added after.
// The result is accurate to a few units in its own last place even when it is far
// smaller than either product -- the case of a small residual, b |rho| against |rho|.
__device__ __forceinline__ float cross_df(float sn, float cs, float u, float uc, float v, float vc)
{
    float e1, e2;
    const float p1 = two_prod(sn, u, e1);
    const float p2 = two_prod(cs, v, e2);
    return __fadd_rn(__fsub_rn(p1, p2), (e1 - e2) - fmaf(sn, uc, -cs * vc));
}

// sqrt((u - uc)^2 + (v - vc)^2) as hi + lo (double-float): the sum of squares with its
// rounding errors (two_prod, two-sum) and the compensation's first-order term, then one
// Newton correction of the FP32 square root.
__device__ __forceinline__ float hypot_df(float u, float uc, float v, float vc, float &lo)
{
    float eu, ev;
    const float su = two_prod(u, u, eu), sv = two_prod(v, v, ev);
    const float qh = __fadd_rn(su, sv);                       // two-sum: qh + qe = su + sv
    const float bv = __fsub_rn(qh, su);
    const float qe = __fadd_rn(__fsub_rn(su, __fsub_rn(qh, bv)), __fsub_rn(sv, bv));
    const float ql = ((qe + eu) + ev) - 2.0f * fmaf(u, uc, v * vc);
    const float r = __fsqrt_rn(qh);
    lo = (fmaf(-r, r, qh) + ql) * (0.5f / r);
    return r;
}

// Residuals of one epoch formed directly as small angles:
//   b_alpha = atan2(sin a~ rho_x - cos a~ rho_y, cos a~ rho_x + sin a~ rho_y)  (= wrap(a~ - a))
//   b_beta  = atan2(sin b~ rho_xy - cos b~ rho_z, cos b~ rho_xy + sin b~ rho_z) (= b~ - b)
// rho = d - c, the offset and its compensation.  The numerators cancel to b |rho|, so
// they (and rho_xy, which the second one needs to full accuracy) are formed in
// double-float arithmetic; an FP32 numerator would carry about 6e-8 |rho| of rounding,
// an error of about 6e-8 rad in every residual that differs from particle to particle
// (about 1% of a 1 arcsec sigma) and leaves false minima in the cost for the swarm to
// settle in.  The denominators (~|rho|) and the arctangents are plain FP32.  The epoch's
// weighted sum of squares is added to the FP64 total J.
__device__ __forceinline__ void add_epoch_cost_rel(const float d[3], const float c[3], const ObsDir &o,
                                                   float w_ra, float w_dec, int quartic,
                                                   int use_range, float rng_obs, float w_rng,
                                                   double &J)
{
    const float rx = d[0] - c[0], ry = d[1] - c[1], rz = d[2] - c[2];
    const float rxy2 = fmaf(rx, rx, ry * ry);
    const float r2 = fmaf(rz, rz, rxy2);
    if (!(r2 >= 1e-30f) || !isfinite(r2)) {
        J = CUDART_INF;
        return;
    }
    float rxy_lo;
    const float rxy = hypot_df(d[0], c[0], d[1], c[1], rxy_lo);
    const float na = cross_df(o.sa, o.ca, d[0], c[0], d[1], c[1]);
    const float nb = cross_df(o.sb, o.cb, rxy, -rxy_lo, d[2], c[2]);
    const float ba = atan2f(na, fmaf(o.ca, rx, o.sa * ry));
    const float bb = atan2f(nb, fmaf(o.cb, rxy, o.sb * rz));
    float Jk = fmaf(ba * w_ra, ba, bb * w_dec * bb);
    if (use_range) {
        // |rho| = hypot(rho_xy, rho_z) in double-float as well: the residual cancels too
        float r_lo;
        const float r = hypot_df(rxy, -rxy_lo, d[2], c[2], r_lo);
        const float br = (rng_obs - r) - r_lo;
        Jk = fmaf(br * w_rng, br, Jk);
    }
    const double Jd = (double)Jk;
    J += quartic ? Jd * Jd : Jd;
}

}  // namespace mix
}  // namespace iod
