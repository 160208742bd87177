// iod_kernels.cu -- CUDA kernels of the PSO-IOD hot path (sm_103a, FP64).
//
// One launch per swarm iteration does all of Algorithm 1's per-iteration work:
//   move (Philox r1, r2; bounded velocity/position update)  ->  propagate to every t_k
//   (RK4 on the interval table, or DOPRI5 with dense output)  ->  angles and weighted
//   residuals (Eqs. 5-13)  ->  personal best  ->  block argmin (warp shuffles)  ->
//   the last block to finish reduces the block winners into the global best.
// The last-block pattern needs no spin-wait: each block publishes its winner, fences,
// and bumps a counter; the block that sees the final count does the grid reduction.
#include "iod_device.cuh"
#include "iod_internal.h"
#include "iod_tma.cuh"

#include <climits>

namespace iod {

using namespace dev;

namespace {

constexpr int kRK4 = 0;
constexpr int kDOPRI5 = 1;
constexpr int kMaxThreads = 256;

// The problem's dynamics (CR3BP, or ER3BP about the true anomaly f0).
__device__ __forceinline__ Dyn make_dyn(const KParams &P)
{
    Dyn D{P.mu, 1.0 - P.mu};
    D.e = P.ecc;
    D.f0 = P.f0;
    D.er = P.dynamics;
    return D;
}

// Observation table view (shared memory in the swarm kernels, global elsewhere).
struct ObsView {
    const double *ra, *dec, *rng, *rcx, *rcy, *rcz, *t, *h;
    const int *ns;
    int n;
};

// Propagate s with fixed-step RK4 over the intervals ending at epochs ka..kb-1 (s is the
// state at t_{ka-1}, or at t = 0 for ka = 0); f(k, s) at each t_k.  ER = 1: the elliptic
// problem (a compile-time choice, so the circular problem's loop is unchanged).
template <int ER = 0, class F>
__device__ __forceinline__ long long propagate_rk4_epochs(const Dyn &D, double s[6], const ObsView &O,
                                                          int ka, int kb, F &&f)
{
    long long steps = 0;
    for (int k = ka; k < kb; ++k) {
        const int n = O.ns[k];
        const RkH C = rk_h(O.h[k]);
        if (ER) {
            // the interval starts at true anomaly f0 + t_{k-1}; cos f at the stages comes
            // from the angle-addition recurrence in steps of h/2 (restarted from sincos
            // at every interval), the same values for every particle
            double sf, cf, sh, ch;
            sincos(D.f0 + (k == 0 ? 0.0 : O.t[k - 1]), &sf, &cf);
            sincos(C.hh, &sh, &ch);
            for (int j = 0; j < n; ++j) {
                const double cm = fma(cf, ch, -sf * sh), sm = fma(sf, ch, cf * sh);
                const double ce = fma(cm, ch, -sm * sh), se = fma(sm, ch, cm * sh);
                rk4_step_er(D, cf, cm, ce, C, s);
                cf = ce;
                sf = se;
            }
        } else {
            for (int j = 0; j < n; ++j) rk4_step(D, C, s);
        }
        steps += n;
        f(k, s);
    }
    return steps;
}

// Propagate s through all epochs with fixed-step RK4; f(k, s) at each t_k.
template <int ER = 0, class F>
__device__ __forceinline__ long long propagate_rk4(const Dyn &D, double s[6], const ObsView &O, F &&f)
{
    return propagate_rk4_epochs<ER>(D, s, O, 0, O.n, f);
}

// RK4 propagation choosing the dynamics at run time (set-up, propagation and refinement
// kernels; the swarm kernels choose at compile time).
template <class F>
__device__ __forceinline__ long long propagate_rk4_any(const Dyn &D, double s[6], const ObsView &O, F &&f)
{
    return D.er ? propagate_rk4<1>(D, s, O, f) : propagate_rk4<0>(D, s, O, f);
}

// DOPRI5's whole loop state between attempts (the current state, its first stage --
// FSAL: the last step's seventh --, the next step size, the time, the next epoch to
// emit, the attempts taken, whether the solution is still finite and within budget).
// Continuing from a saved state repeats the uninterrupted sequence of attempts bit for
// bit, which is what lets the balanced schedule cut a particle's arc between warps.
struct DpState {
    double s[6], k1[6];
    double h, tc;
    int next;
    int ok;
    long long steps;
};

// Start: the state at t = 0, epochs at t <= 0 emitted, k1 = f(s).
template <int ER = 0, int PAIR = 0, class F>
__device__ __forceinline__ void dopri5_begin(const Dyn &D, DpState &st, const double s0[6], const ObsView &O,
                                             double h0, F &&f, bool odd = false)
{
#pragma unroll
    for (int i = 0; i < 6; ++i) st.s[i] = s0[i];
    st.tc = 0.0;
    st.h = h0;
    st.next = 0;
    st.ok = 1;
    st.steps = 0;
    while (st.next < O.n && O.t[st.next] <= st.tc) {
        f(st.next, st.s);
        ++st.next;
    }
    rhs_any<ER, PAIR>(D, odd, st.tc, st.s, st.k1);
}

// Attempt steps until the next epoch to emit is `stop` or later (O.n: the whole arc), the
// solution goes non-finite or the attempt budget runs out (ok = 0; later epochs are then
// not emitted); dense output at each epoch passed.
template <int ER = 0, int PAIR = 0, class F>
__device__ __forceinline__ void dopri5_advance(const Dyn &D, DpState &st, const ObsView &O, double rtol,
                                               double atol, long long max_steps, int stop, F &&f,
                                               bool odd = false)
{
    if (!st.ok) return;
    const double tend = O.t[O.n - 1];
    double tc = st.tc, h = st.h;
    int next = st.next;
    long long steps = st.steps;
    DpStages K;
    double s[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        s[i] = st.s[i];
        K.k1[i] = st.k1[i];
    }
    double s1[6], y[6];
    while (next < stop) {
        bool fin = true;
#pragma unroll
        for (int i = 0; i < 6; ++i) fin = fin && isfinite(s[i]);
        if (steps >= max_steps || !(h > 0.0) || !fin) {
            st.ok = 0;
            break;
        }
        bool last = false;
        if (tc + h >= tend) {
            h = tend - tc;
            last = true;
        }
        const double err = dopri5_attempt<ER, PAIR>(D, tc, h, s, K, s1, rtol, atol, odd);
        ++steps;
        if (!isfinite(err)) {
            st.ok = 0;
            break;
        }
        double fac = 0.9 * inv_fifth_root(err);
        if (err == 0.0 || fac > 5.0) fac = 5.0;
        if (fac < 0.2) fac = 0.2;
        if (err <= 1.0) {
            const double tn = last ? tend : tc + h;
            if (next < O.n && O.t[next] <= tn) {
                // epochs inside the step: theta = (t_k - t) / h from one reciprocal
                const double rh = 1.0 / h;
                do {
                    if (O.t[next] == tn) {
                        f(next, s1);
                    } else {
                        dopri5_dense(h, s, K, (O.t[next] - tc) * rh, y);
                        f(next, y);
                    }
                    ++next;
                } while (next < O.n && O.t[next] <= tn);
            }
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                s[i] = s1[i];
                K.k1[i] = K.k7[i];
            }
            tc = tn;
        }
        h = h * fac;
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        st.s[i] = s[i];
        st.k1[i] = K.k1[i];
    }
    st.tc = tc;
    st.h = h;
    st.next = next;
    st.steps = steps;
}

// Epoch positions waiting for their cost terms: a lane's FIFO of (epoch, position).
constexpr int kDpBufCap = 10, kDpFlushAt = 6;
struct DpEpochBuf {
    double y[kDpBufCap][3];
    int k[kDpBufCap];
    int head, count;
};

// The same integration as dopri5_advance, called by all 32 lanes of a warp together
// (act: the lane holds a particle) and with the epochs' cost terms taken out of the
// accepted-step branch.  An FP64 warp instruction costs its sub-partition 64 cycles however
// few lanes are active, and lanes cross different numbers of epochs per step, so the
// cost terms evaluated inside that branch ran with a few lanes at a time.  Here a lane
// only forms the dense-output position there and queues it; the warp, at the top of the
// step loop where its lanes are together, evaluates the queued terms of all lanes when any
// lane has kDpFlushAt of them (every lane its own, in epoch order), and the rest at the
// end.  Each lane adds its terms to J in epoch order as before, so the result is the same.
// cost(k, y): the cost term of epoch k at position y, added to the lane's running sum.
template <class C>
__device__ __forceinline__ void dopri5_advance_warp(const Dyn &D, DpState &st, const ObsView &O, double rtol,
                                                    double atol, long long max_steps, int stop, bool act,
                                                    DpEpochBuf &B, C &&cost)
{
    const double tend = O.t[O.n - 1];
    double tc = st.tc, h = st.h;
    int next = st.next, ok = st.ok;
    long long steps = st.steps;
    DpStages K;
    double s[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        s[i] = st.s[i];
        K.k1[i] = st.k1[i];
    }
    B.head = 0;
    B.count = 0;
    auto take = [&](int n_take) {     // the lane's n_take oldest queued terms, in order
        for (int j = 0; j < n_take; ++j) {
            const int e = B.head;
            cost(B.k[e], B.y[e]);
            B.head = e + 1 == kDpBufCap ? 0 : e + 1;
            --B.count;
        }
    };
    auto flush = [&]() {              // every lane its whole queue, the warp together
        const int mx = __reduce_max_sync(0xffffffffu, B.count);
        for (int j = 0; j < mx; ++j)
            if (B.count > 0) take(1);
    };
    auto queue = [&](int k, const double *y) {
        if (B.count == kDpBufCap) take(1);     // full: the oldest first
        int e = B.head + B.count;
        if (e >= kDpBufCap) e -= kDpBufCap;
        B.k[e] = k;
        B.y[e][0] = y[0];
        B.y[e][1] = y[1];
        B.y[e][2] = y[2];
        ++B.count;
    };
    bool run = act && ok && next < stop;
    double s1[6], y[6];
    while (__any_sync(0xffffffffu, run)) {
        if (__any_sync(0xffffffffu, B.count >= kDpFlushAt)) flush();
        if (!run) continue;
        bool fin = true;
#pragma unroll
        for (int i = 0; i < 6; ++i) fin = fin && isfinite(s[i]);
        if (steps >= max_steps || !(h > 0.0) || !fin) {
            ok = 0;
            run = false;
            continue;
        }
        bool last = false;
        if (tc + h >= tend) {
            h = tend - tc;
            last = true;
        }
        const double err = dopri5_attempt<0, 0>(D, tc, h, s, K, s1, rtol, atol, false);
        ++steps;
        if (!isfinite(err)) {
            ok = 0;
            run = false;
            continue;
        }
        double fac = 0.9 * inv_fifth_root(err);
        if (err == 0.0 || fac > 5.0) fac = 5.0;
        if (fac < 0.2) fac = 0.2;
        if (err <= 1.0) {
            const double tn = last ? tend : tc + h;
            if (next < O.n && O.t[next] <= tn) {
                const double rh = 1.0 / h;
                do {
                    if (O.t[next] == tn) {
                        queue(next, s1);
                    } else {
                        dopri5_dense(h, s, K, (O.t[next] - tc) * rh, y);
                        queue(next, y);
                    }
                    ++next;
                } while (next < O.n && O.t[next] <= tn);
            }
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                s[i] = s1[i];
                K.k1[i] = K.k7[i];
            }
            tc = tn;
        }
        h = h * fac;
        run = next < stop;
    }
    flush();
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        st.s[i] = s[i];
        st.k1[i] = K.k1[i];
    }
    st.tc = tc;
    st.h = h;
    st.next = next;
    st.ok = ok;
    st.steps = steps;
}

// Propagate s with DOPRI5 over the whole arc, emitting dense output at each t_k.  Returns
// attempts taken; sets ok = false if the solution goes non-finite or the step budget runs
// out (the remaining epochs are then not emitted).  PAIR = 1: the right-hand sides over a
// lane pair (both lanes carry the same state and take the same steps).
template <int ER = 0, int PAIR = 0, class F>
__device__ __forceinline__ long long propagate_dopri5(const Dyn &D, double s[6], const ObsView &O,
                                                      double rtol, double atol, double h0,
                                                      long long max_steps, bool &ok, F &&f,
                                                      bool odd = false)
{
    DpState st;
    dopri5_begin<ER, PAIR>(D, st, s, O, h0, f, odd);
    dopri5_advance<ER, PAIR>(D, st, O, rtol, atol, max_steps, O.n, f, odd);
#pragma unroll
    for (int i = 0; i < 6; ++i) s[i] = st.s[i];
    ok = st.ok != 0;
    return st.steps;
}

// Cost J(x) of one candidate; steps taken are added to *steps.
template <int INTEG, int ER = 0>
__device__ __forceinline__ double evaluate(const KParams &P, const Dyn &D, const CostW &W,
                                           const ObsView &O, const double x[6], long long &steps)
{
    double s[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) s[d] = x[d];
    double J = 0.0;
    auto epoch = [&](int k, const double *st) {
        add_epoch_cost(W, st[0] - O.rcx[k], st[1] - O.rcy[k], st[2] - O.rcz[k], O.ra[k],
                       O.dec[k], W.use_range ? O.rng[k] : 0.0, J);
    };
    if (INTEG == kRK4) {
        steps += propagate_rk4<ER>(D, s, O, epoch);
    } else {
        bool ok;
        steps += propagate_dopri5<ER>(D, s, O, P.rtol, P.atol, P.h0, P.max_steps, ok, epoch);
        if (!ok) J = CUDART_INF;
    }
    return (isnan(J) || !isfinite(J)) ? CUDART_INF : J;
}

// Stage the observation table into dynamic shared memory.
__device__ __forceinline__ ObsView stage_obs(const KParams &P, double *sm)
{
    const int K = P.n_obs;
    double *ra = sm, *dec = sm + K, *rng = sm + 2 * K, *rcx = sm + 3 * K, *rcy = sm + 4 * K,
           *rcz = sm + 5 * K, *t = sm + 6 * K, *h = sm + 7 * K;
    int *ns = reinterpret_cast<int *>(sm + 8 * K);
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        ra[k] = P.ra[k];
        dec[k] = P.dec[k];
        rng[k] = P.rng ? P.rng[k] : 0.0;
        rcx[k] = P.rc[k];
        rcy[k] = P.rc[K + k];
        rcz[k] = P.rc[2 * K + k];
        t[k] = P.t[k];
        h[k] = P.h[k];
        ns[k] = P.nsteps[k];
    }
    return ObsView{ra, dec, rng, rcx, rcy, rcz, t, h, ns, K};
}

__device__ __forceinline__ CostW load_weights(const KParams &P)
{
    CostW W;
    W.w_ra = P.cst->w_ra;
    W.w_dec = P.cst->w_dec;
    W.w_rng = P.cst->w_rng;
    W.quartic = P.cost_form == 1;
    W.use_range = P.use_range;
    return W;
}

// Sum per-thread step counts into the run's counter (one atomic per warp).
__device__ __forceinline__ void add_steps(GBest *gb, long long steps)
{
    unsigned long long s = (unsigned long long)steps;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(&gb->steps, s);
}

// Block argmin of (J, i) with the winner's state, then the last block to finish
// folds every block's winner into the global best.  `init`: take the winner
// unconditionally (initial evaluation) instead of on strict improvement.
// Returns true in every thread of the block that folded the global best (the problem's
// last block of this launch or round).
__device__ bool reduce_to_global_best(const KParams &P, double J, int i, const double xe[6],
                                      int n, bool init, int bidx, int nblk, int flags_or = 0)
{
    __shared__ double s_wj[32];
    __shared__ int s_wi[32];
    __shared__ int s_best;
    __shared__ bool s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    double bj = (i < P.m) ? J : CUDART_INF;
    int bi = (i < P.m) ? i : INT_MAX;
    warp_argmin(bj, bi);
    if (lane == 0) {
        s_wj[warp] = bj;
        s_wi[warp] = bi;
    }
    __syncthreads();
    if (warp == 0) {
        bj = lane < nwarps ? s_wj[lane] : CUDART_INF;
        bi = lane < nwarps ? s_wi[lane] : INT_MAX;
        warp_argmin(bj, bi);
        if (lane == 0) s_best = bi;
    }
    __syncthreads();
    if (i == s_best) {
        BlockBest &b = P.blk[bidx];
        b.J = J;
        b.idx = i;
#pragma unroll
        for (int d = 0; d < 6; ++d) b.x[d] = xe[d];
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int prev = atomicAdd(&P.gb->done_blocks, 1u);
        s_last = (prev == (unsigned int)nblk - 1);
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    // grid reduction over block winners (deterministic: a pure function of the slots)
    bj = CUDART_INF;
    bi = INT_MAX;
    int bslot = -1;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
        const double j = __ldcg(&P.blk[b].J);
        const int ix = __ldcg(&P.blk[b].idx);
        if (better(j, ix, bj, bi)) {
            bj = j;
            bi = ix;
            bslot = b;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double oj = __shfl_xor_sync(0xffffffffu, bj, off);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
        const int os = __shfl_xor_sync(0xffffffffu, bslot, off);
        if (better(oj, oi, bj, bi)) {
            bj = oj;
            bi = oi;
            bslot = os;
        }
    }
    __shared__ int s_slot[32];
    __syncthreads();
    if (lane == 0) {
        s_wj[warp] = bj;
        s_wi[warp] = bi;
        s_slot[warp] = bslot;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < nwarps; ++w)
            if (better(s_wj[w], s_wi[w], bj, bi)) {
                bj = s_wj[w];
                bi = s_wi[w];
                bslot = s_slot[w];
            }
        // the record may have been written by another SM earlier in this launch: read it
        // from L2
        GBest *gb = P.gb;
        double gJ = __ldcg(&gb->gJ);
        int gidx = __ldcg(&gb->gidx);
        if (bslot >= 0 && (init || bj < gJ)) {
            gJ = bj;
            gidx = bi + P.offset;   // index in the whole swarm
            gb->gJ = bj;
            gb->gidx = gidx;
#pragma unroll
            for (int d = 0; d < 6; ++d) gb->g[d] = __ldcg(&P.blk[bslot].x[d]);
        }
        gb->iter = n;
        int flags = __ldcg(&gb->flags) | flags_or;
        // Algorithm 2: after iteration n > w stop once |(J_n - J_{n-w}) / J_n| < tau
        if (!init && P.tol_tau > 0.0 && n > P.tol_window) {
            const double old = __ldcg(&gb->hist[(n - P.tol_window) % kTolHist]);
            const double K = fabs(__ddiv_rn(__dsub_rn(gJ, old), gJ));
            if (K < P.tol_tau) flags |= kFlagStopped;
        }
        gb->hist[n % kTolHist] = gJ;
        gb->flags = flags;
        if (P.trace_J && n < P.trace_cap) {
            P.trace_J[n] = gJ;
            P.trace_idx[n] = gidx;
        }
        gb->done_blocks = 0u;
        __threadfence();
    }
    __syncthreads();
    return true;
}

// Initial position of particle i: uniform in the box (Philox stream 2), or stratified
// ("grid-like" initialisation of the particle swarm section): per coordinate d the m
// strata of [lo_d, hi_d] are dealt out by the permutation (A_d i + B_d) mod m, A_d a
// prime above 2^31 and B_d a Philox draw (stream 4, block d), and the particle sits at
// the same uniform draw inside its stratum.  Every stratum of every coordinate holds
// exactly one particle.
//
// With the line-of-sight initialisation (the sensor-feasible starting positions of the
// abstract; first epoch at t = 0) the three position draws become a range rho in
// [rho_min, rho_max] and two tilts of the first observed direction u(alpha_0, beta_0)
// in its tangent plane; the position r_c(0) + rho (u + s_a e_a + s_b e_b)/|...| is
// clamped into the box.  Velocities stay uniform in the box.
__device__ __forceinline__ void initial_position(const KParams &P, int i, double x[6])
{
    constexpr unsigned long long kA[6] = {2147483659ull, 2147483693ull, 2147483713ull,
                                          2147483743ull, 2147483777ull, 2147483783ull};
    const uint2 key = make_uint2((uint32_t)P.seed, (uint32_t)(P.seed >> 32));
    double t[6];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const uint4 r = philox4x32_10(make_uint4((uint32_t)(i + P.offset), 0u, 2u, (uint32_t)b), key);
        t[2 * b] = u01(r.x, r.y);
        t[2 * b + 1] = u01(r.z, r.w);
    }
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        if (P.init_grid) {
            const uint4 q = philox4x32_10(make_uint4(0u, 0u, 4u, (uint32_t)d), key);
            const unsigned long long mm = (unsigned long long)P.m_total;
            const unsigned long long pi =
                (kA[d] * (unsigned long long)(i + P.offset) + (unsigned long long)q.x % mm) % mm;
            t[d] = __ddiv_rn(__dadd_rn((double)pi, t[d]), (double)P.m_total);
        }
        x[d] = __dadd_rn(P.lo[d], __dmul_rn(t[d], __dsub_rn(P.hi[d], P.lo[d])));
    }
    if (P.init_cone) {
        const ConeInit &C = P.cone;
        const double rho = __dadd_rn(C.rho[0], __dmul_rn(t[0], __dsub_rn(C.rho[1], C.rho[0])));
        const double sa = __dmul_rn(__dsub_rn(__dmul_rn(2.0, t[1]), 1.0), C.smax[0]);
        const double sb = __dmul_rn(__dsub_rn(__dmul_rn(2.0, t[2]), 1.0), C.smax[1]);
        double dir[3];
#pragma unroll
        for (int j = 0; j < 3; ++j)
            dir[j] = __dadd_rn(__dadd_rn(C.u[j], __dmul_rn(sa, C.ea[j])), __dmul_rn(sb, C.eb[j]));
        const double n = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dir[0], dir[0]), __dmul_rn(dir[1], dir[1])),
                                              __dmul_rn(dir[2], dir[2])));
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double r = __dadd_rn(P.rc[j * P.n_obs], __dmul_rn(rho, __ddiv_rn(dir[j], n)));
            if (r < P.lo[j]) r = P.lo[j];
            if (r > P.hi[j]) r = P.hi[j];
            x[j] = r;
        }
    }
}

// Initial velocity: zero (Algorithm 1 leaves it unspecified), or with velocity_init
// uniform within the velocity limits, v_d = (2u - 1) vmax_d, u from Philox stream 5
// (block b gives dimensions 2b, 2b+1).
__device__ __forceinline__ void initial_velocity(const KParams &P, int i, double v[6])
{
#pragma unroll
    for (int d = 0; d < 6; ++d) v[d] = 0.0;
    if (!P.velocity_init) return;
    const uint2 key = make_uint2((uint32_t)P.seed, (uint32_t)(P.seed >> 32));
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const uint4 r = philox4x32_10(make_uint4((uint32_t)(i + P.offset), 0u, 5u, (uint32_t)b), key);
        v[2 * b] = __dmul_rn(__dsub_rn(__dmul_rn(2.0, u01(r.x, r.y)), 1.0), P.cst->vmax[2 * b]);
        v[2 * b + 1] = __dmul_rn(__dsub_rn(__dmul_rn(2.0, u01(r.z, r.w)), 1.0), P.cst->vmax[2 * b + 1]);
    }
}

// Bounded velocity/position update of Algorithm 1 in the oracle's exact rounding
// order (no contraction), so that positions agree bit for bit given the same bests.
// r1, r2 come from Philox stream 3 at counter (i, n): one pair per particle per iteration
// (block 0), or with per_dim_random one pair per dimension (block d).  i is the particle's
// index in the whole swarm (P.offset + the local index: a swarm sharded over problems
// draws the numbers the unsharded swarm draws).
__device__ __forceinline__ void move(const KParams &P, const double g[6], int i, int n,
                                     double x[6], double v[6], const double p[6])
{
    const uint2 key = make_uint2((uint32_t)P.seed, (uint32_t)(P.seed >> 32));
    const uint32_t gi = (uint32_t)(i + P.offset);      // the particle's index in the whole swarm
    uint4 r = philox4x32_10(make_uint4(gi, (uint32_t)n, 3u, 0u), key);
    double a1 = __dmul_rn(P.c1, u01(r.x, r.y)), a2 = __dmul_rn(P.c2, u01(r.z, r.w));
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        if (P.per_dim_random && d > 0) {
            r = philox4x32_10(make_uint4(gi, (uint32_t)n, 3u, (uint32_t)d), key);
            a1 = __dmul_rn(P.c1, u01(r.x, r.y));
            a2 = __dmul_rn(P.c2, u01(r.z, r.w));
        }
        double vd = __dadd_rn(__dadd_rn(__dmul_rn(P.w, v[d]), __dmul_rn(a1, __dsub_rn(p[d], x[d]))),
                              __dmul_rn(a2, __dsub_rn(g[d], x[d])));
        if (P.constriction) vd = __dmul_rn(P.kappa, vd);   // Eq. 4, kappa formed on the host
        const double vmax = P.cst->vmax[d];
        if (vd > vmax) vd = vmax;
        if (vd < -vmax) vd = -vmax;
        double xd = __dadd_rn(x[d], vd);
        if (xd < P.lo[d]) {
            xd = P.lo[d];
            vd = 0.0;
        }
        if (xd > P.hi[d]) {
            xd = P.hi[d];
            vd = 0.0;
        }
        v[d] = vd;
        x[d] = xd;
    }
}

// ------------------------------------------------------------------ kernels
// Interval table, weights, velocity limits, run counters and the chief trajectory of one
// problem (one thread).  Returns the number of RK4 steps per propagation.
// The RK4 interval rule: the interval from t_prev to t_k (t_prev = 0 before the first
// epoch) takes n_k = max(1, ceil(span/dt - 1e-9)) equal steps of span/n_k, none for an
// empty span.  Every kernel that builds an interval table calls this one rule.
__device__ __forceinline__ void interval_rule(double t_prev, double t_k, double dt, int &n, double &h)
{
    const double span = t_k - t_prev;
    if (span == 0.0) {
        n = 0;
        h = 0.0;
    } else {
        double q = ceil(__dsub_rn(__ddiv_rn(span, dt), 1e-9));
        if (q < 1.0) q = 1.0;
        n = (int)q;
        h = __ddiv_rn(span, q);
    }
}

// Interval k of the problem's RK4 table.
__device__ __forceinline__ void interval_steps(const KParams &P, int k, int &n, double &h)
{
    interval_rule(k == 0 ? 0.0 : P.t[k - 1], P.t[k], P.dt, n, h);
}

// Problem set-up.  One thread, or (pair = true: RK4, circular problem) lanes 0 and 1 of a
// warp, which propagate the chief together on a lane pair (rk4_step_pair, the same values
// as one thread); lane 0 writes every output.  cs (pair form only; null when unused): the
// chief's state at every RK4 step boundary, [S+1][6], which the mixed-precision table is
// built from in parallel (setup_mixed_body).
__device__ long long setup_body(const KParams &P, double vmax_frac, double sig_ra, double sig_dec,
                                double sig_rng, const double *__restrict__ chief, double *rc,
                                int *nsteps, double *hs, Consts *cst, GBest *gb, int lane = 0,
                                bool pair = false, double *cs = nullptr)
{
    const int K = P.n_obs;
    if (pair) {
        const Dyn D = make_dyn(P);
        double s[6];
        for (int d = 0; d < 6; ++d) s[d] = chief[d];
        if (cs && lane == 0)
            for (int d = 0; d < 6; ++d) cs[d] = s[d];
        long long g = 0;
        for (int k = 0; k < K; ++k) {
            int n;
            double h;
            interval_steps(P, k, n, h);
            const RkH C = rk_h(h);
            for (int j = 0; j < n; ++j) {
                rk4_step_pair(D, lane == 1, C, s, 0x3u);
                ++g;
                if (cs && lane == 0)
                    for (int d = 0; d < 6; ++d) cs[6 * g + d] = s[d];
            }
            if (lane == 0) {
                nsteps[k] = n;
                hs[k] = h;
                rc[k] = s[0];
                rc[K + k] = s[1];
                rc[2 * K + k] = s[2];
            }
        }
        if (lane != 0) return 0;
    } else {
        for (int k = 0; k < K; ++k) interval_steps(P, k, nsteps[k], hs[k]);
    }
    cst->w_ra = 1.0 / (sig_ra * sig_ra);
    cst->w_dec = 1.0 / (sig_dec * sig_dec);
    cst->w_rng = P.use_range ? 1.0 / (sig_rng * sig_rng) : 0.0;
    for (int d = 0; d < 6; ++d) cst->vmax[d] = __dmul_rn(vmax_frac, __dsub_rn(P.hi[d], P.lo[d]));
    cst->tend = P.t[K - 1];
    gb->done_blocks = 0u;
    gb->status = 0;
    gb->steps = 0ull;
    gb->iter = -1;
    // chief trajectory with the problem's integrator and grid (already done on a pair)
    const Dyn D = make_dyn(P);
    ObsView O{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, P.t, hs, nsteps, K};
    double s[6];
    for (int d = 0; d < 6; ++d) s[d] = chief[d];
    bool ok = true;
    auto store = [&](int k, const double *st) {
        rc[k] = st[0];
        rc[K + k] = st[1];
        rc[2 * K + k] = st[2];
    };
    if (pair) {
    } else if (P.integrator == kRK4) {
        propagate_rk4_any(D, s, O, store);
    } else {
        if (D.er)
            propagate_dopri5<1>(D, s, O, P.rtol, P.atol, P.h0, P.max_steps, ok, store);
        else
            propagate_dopri5<0>(D, s, O, P.rtol, P.atol, P.h0, P.max_steps, ok, store);
    }
    for (int k = 0; k < 3 * K; ++k) ok = ok && isfinite(rc[k]);
    if (!ok) gb->status |= kStatusChiefDiverged;
    long long S = 0;
    for (int k = 0; k < K; ++k) S += nsteps[k];
    return S;
}

__global__ void setup_kernel(KParams P, double vmax_frac, double sig_ra, double sig_dec,
                             double sig_rng, const double *__restrict__ chief, double *rc,
                             int *nsteps, double *hs, Consts *cst, GBest *gb, double *cs)
{
    const bool pair = P.integrator == kRK4 && !P.dynamics;
    if (blockIdx.x != 0 || threadIdx.x >= (pair ? 2u : 1u)) return;
    setup_body(P, vmax_frac, sig_ra, sig_dec, sig_rng, chief, rc, nsteps, hs, cst, gb, threadIdx.x, pair,
               pair ? cs : nullptr);
}

// Argument checks of the IOD_CHECK build (a stand-in for a memory checker, which this
// GPU's tooling does not offer here): at the entry of every swarm body, the swarm and
// observation-table pointers are present and 8-byte aligned, the stride covers the
// swarm, the launch's tiles cover every particle (threads_per_particle lanes each), the
// block index lies among them, the dynamic shared memory holds the observation table
// (mixed: its own layout, checked where its copies are issued) and the interval table
// sums to the step count.  A failed check sets kStatusCheck and the whole tile returns
// before touching memory; the host reports it.  Compiled out of the normal build.
__device__ __forceinline__ bool params_ok(const KParams &P, int bidx, int nblk, int lanes, bool fp64_table)
{
#ifdef IOD_CHECK
    const auto al8 = [](const void *q) { return q && (reinterpret_cast<uintptr_t>(q) & 7u) == 0u; };
    bool ok = P.m >= 1 && P.stride >= P.m && P.n_obs >= 1 && bidx >= 0 && bidx < nblk && P.offset >= 0 &&
              (long long)P.offset + P.m <= (long long)P.m_total &&
              (long long)nblk * blockDim.x >= (long long)P.m * lanes && al8(P.x) && al8(P.v) &&
              al8(P.p) && al8(P.pJ) && al8(P.J) && al8(P.gb) && al8(P.blk) && al8(P.t) && al8(P.ra) &&
              al8(P.dec) && al8(P.rc) && al8(P.h) && P.nsteps && P.cst;
    if (ok && fp64_table) {
        unsigned int dyn;
        asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
        ok = (size_t)dyn >= (size_t)P.n_obs * (8 * sizeof(double) + sizeof(int));
    }
    if (ok && P.integrator == kRK4 && P.total_steps > 0) {
        long long S = 0;
        for (int k = 0; k < P.n_obs; ++k) S += P.nsteps[k];
        ok = S == P.total_steps;
    }
    if (!ok && threadIdx.x == 0 && P.gb) atomicOr(&P.gb->status, kStatusCheck);
    return ok;
#else
    (void)P, (void)bidx, (void)nblk, (void)lanes, (void)fp64_table;
    return true;
#endif
}

template <int INTEG, int ER = 0>
__device__ __forceinline__ bool init_body(const KParams &P, int bidx, int nblk)
{
    if (!params_ok(P, bidx, nblk, 1, true)) return false;
    extern __shared__ double sm[];
    const ObsView O = stage_obs(P, sm);
    const CostW W = load_weights(P);
    const Dyn D = make_dyn(P);
    __syncthreads();
    const int i = bidx * blockDim.x + threadIdx.x;
    double x[6] = {0, 0, 0, 0, 0, 0};
    double J = CUDART_INF;
    long long steps = 0;
    if (i < P.m) {
        initial_position(P, i, x);
        J = evaluate<INTEG, ER>(P, D, W, O, x, steps);
        double v0[6];
        initial_velocity(P, i, v0);
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            P.x[d * P.stride + i] = x[d];
            P.v[d * P.stride + i] = v0[d];
            P.p[d * P.stride + i] = x[d];
        }
        P.pJ[i] = J;
        P.J[i] = J;
    }
    add_steps(P.gb, steps);
    return reduce_to_global_best(P, J, i, x, 0, true, bidx, nblk, kFlagStarted);
}

template <int INTEG, int LAGGED, int ER = 0>
__device__ __forceinline__ bool iter_body(const KParams &P, int bidx, int nblk)
{
    if (!params_ok(P, bidx, nblk, 1, true)) return false;
    extern __shared__ double sm[];
    const ObsView O = stage_obs(P, sm);
    const CostW W = load_weights(P);
    const Dyn D = make_dyn(P);
    __shared__ double s_g[6];
    __shared__ int s_n;
    if (threadIdx.x < 6) s_g[threadIdx.x] = __ldcg(&P.gb->g[threadIdx.x]);
    __shared__ int s_stop;
    if (threadIdx.x == 0) {
        s_n = __ldcg(&P.gb->iter) + 1;
        s_stop = __ldcg(&P.gb->flags) & kFlagStopped;
    }
    __syncthreads();
    if (s_stop) return false;     // Algorithm 2 ended the run: nothing more to do
    const int n = s_n;
    const int i = bidx * blockDim.x + threadIdx.x;
    double xe[6] = {0, 0, 0, 0, 0, 0};
    double J = CUDART_INF;
    long long steps = 0;
    if (i < P.m) {
        double x[6], v[6], p[6], g[6];
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            x[d] = __ldcg(&P.x[d * P.stride + i]);
            v[d] = __ldcg(&P.v[d * P.stride + i]);
            p[d] = __ldcg(&P.p[d * P.stride + i]);
            g[d] = s_g[d];
        }
        double pJ = __ldcg(&P.pJ[i]);
        if (!LAGGED) {
            move(P, g, i, n, x, v, p);
#pragma unroll
            for (int d = 0; d < 6; ++d) xe[d] = x[d];
            J = evaluate<INTEG, ER>(P, D, W, O, xe, steps);
            if (J < pJ) {
                pJ = J;
#pragma unroll
                for (int d = 0; d < 6; ++d) p[d] = xe[d];
            }
        } else {
#pragma unroll
            for (int d = 0; d < 6; ++d) xe[d] = x[d];
            J = evaluate<INTEG, ER>(P, D, W, O, xe, steps);
            if (J < pJ) {
                pJ = J;
#pragma unroll
                for (int d = 0; d < 6; ++d) p[d] = xe[d];
            }
            move(P, g, i, n, x, v, p);
        }
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            P.x[d * P.stride + i] = x[d];
            P.v[d * P.stride + i] = v[d];
            P.p[d * P.stride + i] = p[d];
        }
        P.pJ[i] = pJ;
        P.J[i] = J;
    }
    add_steps(P.gb, steps);
    return reduce_to_global_best(P, J, i, xe, n, false, bidx, nblk);
}

template <int INTEG>
__global__ void __launch_bounds__(kMaxThreads) eval_kernel(KParams P, const double *__restrict__ X,
                                                           int m, double *__restrict__ Jout)
{
    extern __shared__ double sm[];
    const ObsView O = stage_obs(P, sm);
    const CostW W = load_weights(P);
    const Dyn D = make_dyn(P);
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    double x[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) x[d] = X[(size_t)d * m + i];
    long long steps = 0;
    Jout[i] = P.dynamics ? evaluate<INTEG, 1>(P, D, W, O, x, steps) : evaluate<INTEG, 0>(P, D, W, O, x, steps);
}

template <int INTEG>
__global__ void __launch_bounds__(kMaxThreads) propagate_kernel(KParams P, const double *__restrict__ X,
                                                                int m, double *__restrict__ out)
{
    extern __shared__ double sm[];
    const ObsView O = stage_obs(P, sm);
    const Dyn D = make_dyn(P);
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    double s[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) s[d] = X[(size_t)d * m + i];
    auto store = [&](int k, const double *st) {
#pragma unroll
        for (int d = 0; d < 6; ++d) out[((size_t)k * 6 + d) * m + i] = st[d];
    };
    if (INTEG == kRK4) {
        propagate_rk4_any(D, s, O, store);
    } else {
        bool ok;
        if (D.er)
            propagate_dopri5<1>(D, s, O, P.rtol, P.atol, P.h0, P.max_steps, ok, store);
        else
            propagate_dopri5<0>(D, s, O, P.rtol, P.atol, P.h0, P.max_steps, ok, store);
        if (!ok)
            for (int k = 0; k < O.n; ++k)
                for (int d = 0; d < 6; ++d) out[((size_t)k * 6 + d) * m + i] = CUDART_NAN;
    }
}

// Observation synthesis: thread 0 propagates the chief (positions to chief_pos), then
// the deputy, forming angles (and range) at each epoch plus the given noise.
// ER = 1: the elliptic problem (t then holds elapsed true anomaly).
template <int ER>
__global__ void simulate_kernel(double mu, double ecc, double f0, const double *__restrict__ chief,
                                const double *__restrict__ deputy, int n, const double *__restrict__ t,
                                double rtol, double atol, double h0, const double *__restrict__ noise,
                                double *angles, double *ranges, double *chief_pos, int *status)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    Dyn D{mu, 1.0 - mu};
    D.e = ecc;
    D.f0 = f0;
    D.er = ER;
    ObsView O{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, t, nullptr, nullptr, n};
    double s[6];
    for (int d = 0; d < 6; ++d) s[d] = chief[d];
    bool ok1, ok2;
    propagate_dopri5<ER>(D, s, O, rtol, atol, h0, 100000000LL, ok1, [&](int k, const double *st) {
        chief_pos[3 * k] = st[0];
        chief_pos[3 * k + 1] = st[1];
        chief_pos[3 * k + 2] = st[2];
    });
    for (int d = 0; d < 6; ++d) s[d] = deputy[d];
    propagate_dopri5<ER>(D, s, O, rtol, atol, h0, 100000000LL, ok2, [&](int k, const double *st) {
        const double rx = st[0] - chief_pos[3 * k], ry = st[1] - chief_pos[3 * k + 1],
                     rz = st[2] - chief_pos[3 * k + 2];
        const double r = sqrt(fma(rx, rx, fma(ry, ry, rz * rz)));
        const double a = atan2(ry / r, rx / r), b = asin(rz / r);
        angles[2 * k] = a + (noise ? noise[2 * k] : 0.0);
        angles[2 * k + 1] = b + (noise ? noise[2 * k + 1] : 0.0);
        if (ranges) ranges[k] = r;
    });
    *status = (ok1 && ok2) ? 0 : 1;
}

// ------------------------------------------------------------------ mixed precision
constexpr int kChunk = 32;                  // chief RK4 steps per shared-memory buffer
constexpr unsigned long long kWaitLimitNs = 1000000000ull;   // a copy wait gives up after 1 s

// Set-up of the mixed-precision tables from the chief's states at the RK4 step boundaries
// (cs, written by the set-up kernel): per step its four stage positions relative to each
// primary (FP32), recomputed from the step's start state by the set-up's own RK4
// arithmetic (rk4_step_stages, the same values as rk4_step and rk4_step_pair); per chunk of
// kChunk steps its duration (FP32, summed in step order); per epoch the observed
// direction's sines and cosines.  Every step is independent, so the work is spread over
// threads tid = 0..nthreads-1 (a block, or a grid).
__device__ void setup_mixed_body(const KParams &P, mix::Step *steps, const double *__restrict__ cs,
                                 mix::ObsDir *obsdir, float *chunk_time, int tid, int nthreads)
{
    for (int k = tid; k < P.n_obs; k += nthreads) {
        double sa, ca, sb, cb;
        sincos(P.ra[k], &sa, &ca);
        sincos(P.dec[k], &sb, &cb);
        obsdir[k] = mix::ObsDir{(float)sa, (float)ca, (float)sb, (float)cb};
    }
    const Dyn D = make_dyn(P);
    long long g0 = 0;             // first step of interval k
    for (int k = 0; k < P.n_obs; ++k) {
        const int n = P.nsteps[k];
        const RkH C = rk_h(P.h[k]);
        for (int j = tid; j < n; j += nthreads) {
            const long long g = g0 + j;
            double s[6], St[4][3];
            for (int d = 0; d < 6; ++d) s[d] = cs[6 * g + d];
            rk4_step_stages(D, C, s, St);
            mix::Step M;
            for (int i = 0; i < 4; ++i) {
                const double ex = St[i][0] + D.mu, mx = St[i][0] - D.omu, y = St[i][1], z = St[i][2];
                const double e2 = ex * ex + y * y + z * z, m2 = mx * mx + y * y + z * z;
                M.txy[i] = make_float4(2.0f * (float)ex, 2.0f * (float)mx, 2.0f * (float)y, 2.0f * (float)y);
                M.tzr[i] = make_float4(2.0f * (float)z, 2.0f * (float)z, (float)e2, (float)m2);
                M.inv[i] = make_float2((float)(1.0 / e2), (float)(1.0 / m2));
            }
            steps[g] = M;
        }
        g0 += n;
    }
    // chunk durations: each thread walks the interval table to its chunks' steps
    const long long S = g0;
    const long long nch = (S + kChunk - 1) / kChunk;
    int k = 0;
    long long kstart = 0;          // first step of interval k
    for (long long c = tid; c < nch; c += nthreads) {
        float acc = 0.0f;
        const long long ge = (c + 1) * kChunk < S ? (c + 1) * kChunk : S;
        for (long long g = c * kChunk; g < ge; ++g) {
            while (g >= kstart + P.nsteps[k]) kstart += P.nsteps[k++];
            acc += (float)P.h[k];
        }
        chunk_time[c] = acc;
    }
}

__global__ void setup_mixed_kernel(KParams P, mix::Step *steps, const double *cs, mix::ObsDir *obsdir,
                                   float *chunk_time)
{
    setup_mixed_body(P, steps, cs, obsdir, chunk_time, blockIdx.x * blockDim.x + threadIdx.x,
                     gridDim.x * blockDim.x);
}

// Mixed-precision shared memory: two chief-table buffers filled by bulk asynchronous
// copies, then per epoch the step count, FP32 step sizes (h, h/2, h/6), observed range
// and observed-direction constants.

struct MixView {
    mix::Step *buf;              // 2 x kChunk steps
    const float *chunk_time;     // duration of each chunk of kChunk steps (TU)
    const int *ns;
    const float *hf, *hh, *h6, *rng;
    const mix::ObsDir *od;
    int n;
};

__device__ __forceinline__ MixView stage_mixed(const KParams &P, unsigned char *sm)
{
    const int K = P.n_obs;
    mix::Step *b0 = reinterpret_cast<mix::Step *>(sm);
    int *ns = reinterpret_cast<int *>(sm + 2 * kChunk * sizeof(mix::Step));
    float *hf = reinterpret_cast<float *>(ns + K), *hh = hf + K, *h6 = hh + K, *rng = h6 + K;
    mix::ObsDir *od = reinterpret_cast<mix::ObsDir *>(rng + K);
    float *ct = reinterpret_cast<float *>(od + K);
    const int nch = (int)((P.total_steps + kChunk - 1) / kChunk);
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const double h = P.h[k];
        ns[k] = P.nsteps[k];
        hf[k] = (float)h;
        hh[k] = (float)(0.5 * h);
        h6[k] = (float)(h / 6.0);
        rng[k] = P.rng ? (float)P.rng[k] : 0.0f;
        od[k] = P.obsdir[k];
    }
    for (int ch = threadIdx.x; ch < nch; ch += blockDim.x) ct[ch] = P.chunk_time[ch];
    return MixView{b0, ct, ns, hf, hh, h6, rng, od, K};
}

// One FP64 RK4 step of the absolute state x_c(step start) + delta, returned as the new
// offset from the chief's state at the step's end.  Rare (only near the Moon), so it is
// kept out of line and takes and returns the offset by value.
struct RelState {
    float d[6], c[6];
};

__device__ __noinline__ RelState moon_step(Dyn D, double h, const double *c0, RelState r)
{
    double xa[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) xa[q] = c0[q] + ((double)r.d[q] - (double)r.c[q]);
    rk4_step(D, rk_h(h), xa);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const double d0 = xa[q] - c0[6 + q];
        r.d[q] = (float)d0;
        r.c[q] = -(float)(d0 - (double)r.d[q]);
    }
    return r;
}

// Dynamic shared memory the mixed evaluation lays out (stage_mixed): two chief-table
// buffers of kChunk steps, the per-epoch tables and one duration per chunk.
__host__ __device__ __forceinline__ size_t mixed_smem_layout_bytes(int n_obs, long long total_steps)
{
    const long long nch = (total_steps + kChunk - 1) / kChunk;
    return 2 * kChunk * sizeof(mix::Step) +
           (size_t)n_obs * (sizeof(int) + 4 * sizeof(float) + sizeof(mix::ObsDir)) +
           (size_t)nch * sizeof(float);
}

__device__ __forceinline__ unsigned int dynamic_smem_size()
{
    unsigned int v;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(v));
    return v;
}

// Block-wide record that a bulk copy of the mixed evaluation had still not landed after
// a second bounded wait.  Such a copy may yet write this block's shared memory, so the
// block must not use its buffers again in this launch: the kernels that run several
// mixed ranges per block (the balanced mixed iteration and both batch schedulers) clear
// the flag at entry and stop using the block once it is set; the others never read it.
__device__ __forceinline__ int &mixed_copy_lost()
{
    __shared__ int s_lost;
    return s_lost;
}

// The mixed form over the epochs [ka, kb) (block-collective).  Every thread of the block
// must call this together: the chief's stage table streams through shared memory in
// chunks of kChunk steps (one bulk copy per chunk, issued a chunk ahead by thread 0), so
// all threads walk the same step sequence.  (d, c): each thread's offset delta = x - x_c
// in FP32 and its Kahan compensation at the start of interval ka; steps that start within
// sqrt(moon_r2) of the Moon run in FP64 on the absolute state; epoch terms are added to J
// in FP64.  With out != nullptr the absolute state at each epoch is stored there
// (out[(k*6+d)*m + i], when `active`) instead of forming the cost.  Adds the steps taken
// to steps (and the FP64 ones to steps64); returns false if a copy wait gave up or a
// copy failed its checks (the problem's status says which).
__device__ bool mixed_epochs(const KParams &P, const Dyn &D, const MixView &V, int ka, int kb,
                             float d[6], float c[6], double &J, bool active, long long &steps,
                             long long &steps64, double *out = nullptr, int m = 0, int i = 0)
{
    __shared__ uint64_t bars[2];
    const long long S = P.total_steps;
    // Checks before any copy is issued (the same in every thread): the chief table is
    // 16-byte aligned (every copy starts at a multiple of sizeof(Step) = 160 B from it),
    // and the launch's dynamic shared memory holds the buffers and tables stage_mixed
    // lays out.  A failure marks the problem and issues nothing.
    if ((reinterpret_cast<uintptr_t>(P.mix) & 15u) != 0u || (sizeof(mix::Step) & 15u) != 0u ||
        mixed_smem_layout_bytes(P.n_obs, S) > (size_t)dynamic_smem_size()) {
        if (threadIdx.x == 0) atomicOr(&P.gb->status, kStatusCopyCheck);
        return false;
    }
    // the step range [g0, g1) of the epochs [ka, kb)
    long long g0 = 0, g1;
    for (int k = 0; k < ka; ++k) g0 += V.ns[k];
    g1 = g0;
    for (int k = ka; k < kb; ++k) g1 += V.ns[k];
    const int ch0 = (int)(g0 / kChunk);
    const int ch1 = g1 > g0 ? (int)((g1 - 1) / kChunk) + 1 : ch0;   // chunks [ch0, ch1)
    if (threadIdx.x == 0) {
        tma::mbar_init(&bars[0], 1);
        tma::mbar_init(&bars[1], 1);
        tma::mbar_init_fence();
    }
    __syncthreads();
    // chunk ch goes to buffer and barrier (ch - ch0) & 1
    auto issue = [&](int ch) {
        const int lc = ch - ch0;
        const long long first = (long long)ch * kChunk;
        const int n = (int)((S - first) < kChunk ? (S - first) : kChunk);
        const uint32_t bytes = (uint32_t)n * (uint32_t)sizeof(mix::Step);
        tma::mbar_arrive_expect_tx(&bars[lc & 1], bytes);
        tma::bulk_g2s(V.buf + (lc & 1) * kChunk, P.mix + first, bytes, &bars[lc & 1]);
    };
    // the buffers may hold generic-proxy writes of an earlier tile of this block (its
    // observation table): order them before the first bulk copy
    if (threadIdx.x == 0 && ch1 > ch0) {
        tma::fence_proxy_async();
        issue(ch0);
    }

    const float2 gm2 = make_float2((float)(1.0 - P.mu), (float)P.mu);   // (gm_E, gm_M)
    const float w_ra = (float)P.cst->w_ra, w_dec = (float)P.cst->w_dec, w_rng = (float)P.cst->w_rng;
    const float moon_r2 = (float)P.moon_r2;
    const int quartic = P.cost_form == 1, use_range = P.use_range;
    auto epoch = [&](int k, long long g) {
        if (out) {
            if (active) {
                const double *cg = P.chief_cs + 6 * g;
#pragma unroll
                for (int q = 0; q < 6; ++q)
                    out[((size_t)k * 6 + q) * m + i] = cg[q] + ((double)d[q] - (double)c[q]);
            }
        } else {
            mix::add_epoch_cost_rel(d, c, V.od[k], w_ra, w_dec,
                                    quartic, use_range, V.rng[k], w_rng, J);
        }
    };
    int k = ka;
    while (k < kb && V.ns[k] == 0) epoch(k++, g0);
    int rem = k < kb ? V.ns[k] : 0;
    // step sizes of the current interval, kept in registers between epochs
    float fh = 0.0f, fhh = 0.0f, fh6 = 0.0f;
    auto load_h = [&]() {
        if (k < kb) {
            fh = V.hf[k];
            fhh = V.hh[k];
            fh6 = V.h6[k];
        }
    };
    load_h();
    bool ok = true;
    long long g = g0;
    for (int ch = ch0; ch < ch1; ++ch) {
        const int lc = ch - ch0;
        if (threadIdx.x == 0 && ch + 1 < ch1) {
            tma::fence_proxy_async();
            issue(ch + 1);
        }
        // every thread waits for the chunk; if any wait gave up the whole block stops.
        // Thread 0 then waits once more (bounded) for both copies that may be in flight,
        // this chunk's and the next one's: if both land, the buffers and barriers are
        // quiet and can be retired; if not, the block is marked (mixed_copy_lost) so that
        // it touches these buffers no more in this launch.
        const bool got = tma::mbar_wait(&bars[lc & 1], (lc >> 1) & 1, kWaitLimitNs);
        if (__syncthreads_or(!got)) {
            if (threadIdx.x == 0) {
                bool landed = tma::mbar_wait(&bars[lc & 1], (lc >> 1) & 1, kWaitLimitNs);
                if (ch + 1 < ch1)
                    landed = tma::mbar_wait(&bars[(lc + 1) & 1], ((lc + 1) >> 1) & 1, kWaitLimitNs) && landed;
                if (landed) {
                    tma::mbar_inval(&bars[0]);
                    tma::mbar_inval(&bars[1]);
                } else {
                    mixed_copy_lost() = 1;
                }
            }
            __syncthreads();
            ok = false;
            break;
        }
        const mix::Step *B = V.buf + (lc & 1) * kChunk;
        const long long cs = (long long)ch * kChunk;
        const int j0 = (int)(g - cs);                                    // first step of the range in this chunk
        const int jn = (int)((g1 - cs) < kChunk ? (g1 - cs) : kChunk);   // one past its last
        // Can any lane of this warp start a step within the Moon radius during the chunk?
        // Bound the motion over the chunk by (|v_chief| + |delta v| + 1) x its duration
        // (speeds in these units stay below 1 away from the primaries; the +1 covers the
        // growth of speed near the Moon), against the distance at the range's first step
        // in the chunk.
        const float3 Rm0 = mix::moon_rel(B[j0]);
        const double *cv = P.chief_cs + 6 * g + 3;
        const float vc = sqrtf((float)(cv[0] * cv[0] + cv[1] * cv[1] + cv[2] * cv[2]));
        const float vd = sqrtf(fmaf(d[3], d[3], fmaf(d[4], d[4], d[5] * d[5])));
        const float dist = sqrtf(fmaf(Rm0.x + d[0], Rm0.x + d[0],
                                      fmaf(Rm0.y + d[1], Rm0.y + d[1], (Rm0.z + d[2]) * (Rm0.z + d[2]))));
        const float reach = (vc + vd + 1.0f) * V.chunk_time[ch];
        const bool near = __any_sync(0xffffffffu, dist - reach < sqrtf(moon_r2));
        if (!near) {
            for (int j = j0; j < jn; ++j, ++g) {
                mix::rk4_step_rel(gm2, &B[j], fh, fhh, fh6, d, c);
                if (--rem == 0) {
                    epoch(k++, g + 1);
                    while (k < kb && V.ns[k] == 0) epoch(k++, g + 1);
                    rem = k < kb ? V.ns[k] : 0;
                    load_h();
                }
            }
        } else {
            for (int j = j0; j < jn; ++j, ++g) {
                const mix::Step &St = B[j];
                const float3 Rm = mix::moon_rel(St);
                const float mx = Rm.x + d[0], my = Rm.y + d[1], mz = Rm.z + d[2];
                if (fmaf(mx, mx, fmaf(my, my, mz * mz)) < moon_r2) {
                    RelState r;
#pragma unroll
                    for (int q = 0; q < 6; ++q) {
                        r.d[q] = d[q];
                        r.c[q] = c[q];
                    }
                    r = moon_step(D, P.h[k], P.chief_cs + 6 * g, r);   // near the Moon: FP64
#pragma unroll
                    for (int q = 0; q < 6; ++q) {
                        d[q] = r.d[q];
                        c[q] = r.c[q];
                    }
                    ++steps64;
                } else {
                    mix::rk4_step_rel(gm2, &St, fh, fhh, fh6, d, c);
                }
                if (--rem == 0) {
                    epoch(k++, g + 1);
                    while (k < kb && V.ns[k] == 0) epoch(k++, g + 1);
                    rem = k < kb ? V.ns[k] : 0;
                    load_h();
                }
            }
        }
        __syncthreads();
    }
    steps += g1 - g0;
    // every copy has landed and every thread is past its last wait: retire the barriers
    // (a block initialises them again for its next range)
    if (ok && threadIdx.x == 0) {
        tma::mbar_inval(&bars[0]);
        tma::mbar_inval(&bars[1]);
    }
    if (!ok && threadIdx.x == 0) atomicOr(&P.gb->status, kStatusCopyTimeout);
    return ok;
}

// The offset of x from the chief's initial state, split into FP32 value and compensation.
__device__ __forceinline__ void mixed_offset(const KParams &P, const double x[6], float d[6], float c[6])
{
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const double d0 = x[q] - P.chief_cs[q];
        d[q] = (float)d0;
        c[q] = -(float)(d0 - (double)d[q]);
    }
}

// Cost of each thread's candidate x in the mixed form over the whole arc (block-collective).
__device__ double evaluate_mixed_block(const KParams &P, const Dyn &D, const MixView &V,
                                       const double x[6], bool active, long long &steps,
                                       long long &steps64, double *out = nullptr, int m = 0,
                                       int i = 0)
{
    float d[6], c[6];
    mixed_offset(P, x, d, c);
    double J = 0.0;
    if (!mixed_epochs(P, D, V, 0, V.n, d, c, J, active, steps, steps64, out, m, i)) return CUDART_INF;
    return (isnan(J) || !isfinite(J)) ? CUDART_INF : J;
}

__device__ __forceinline__ void add_steps64(GBest *gb, long long steps64)
{
    unsigned long long s = (unsigned long long)steps64;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(&gb->steps64, s);
}

__device__ __forceinline__ bool init_mixed_body(const KParams &P, int bidx, int nblk)
{
    if (!params_ok(P, bidx, nblk, 1, false)) return false;
    extern __shared__ __align__(128) unsigned char smb[];
    const MixView V = stage_mixed(P, smb);
    const Dyn D = make_dyn(P);
    __syncthreads();
    const int i = bidx * blockDim.x + threadIdx.x;
    const bool active = i < P.m;
    double x[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) x[d] = P.chief_cs[d];      // idle lanes follow the chief
    long long steps = 0, steps64 = 0;
    if (active) initial_position(P, i, x);
    double J = evaluate_mixed_block(P, D, V, x, active, steps, steps64);
    if (active) {
        double v0[6];
        initial_velocity(P, i, v0);
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            P.x[d * P.stride + i] = x[d];
            P.v[d * P.stride + i] = v0[d];
            P.p[d * P.stride + i] = x[d];
        }
        P.pJ[i] = J;
        P.J[i] = J;
    } else {
        J = CUDART_INF;
        steps = 0;
    }
    add_steps(P.gb, steps);
    add_steps64(P.gb, active ? steps64 : 0);
    return reduce_to_global_best(P, J, i, x, 0, true, bidx, nblk, kFlagStarted);
}

template <int LAGGED>
__device__ __forceinline__ bool iter_mixed_body(const KParams &P, int bidx, int nblk)
{
    if (!params_ok(P, bidx, nblk, 1, false)) return false;
    extern __shared__ __align__(128) unsigned char smb[];
    const MixView V = stage_mixed(P, smb);
    const Dyn D = make_dyn(P);
    __shared__ double s_g[6];
    __shared__ int s_n;
    if (threadIdx.x < 6) s_g[threadIdx.x] = __ldcg(&P.gb->g[threadIdx.x]);
    __shared__ int s_stop;
    if (threadIdx.x == 0) {
        s_n = __ldcg(&P.gb->iter) + 1;
        s_stop = __ldcg(&P.gb->flags) & kFlagStopped;
    }
    __syncthreads();
    if (s_stop) return false;     // Algorithm 2 ended the run: nothing more to do
    const int n = s_n;
    const int i = bidx * blockDim.x + threadIdx.x;
    const bool active = i < P.m;
    double x[6], v[6], p[6], xe[6];
    double pJ = CUDART_INF;
#pragma unroll
    for (int d = 0; d < 6; ++d) x[d] = P.chief_cs[d];
    if (active) {
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            x[d] = __ldcg(&P.x[d * P.stride + i]);
            v[d] = __ldcg(&P.v[d * P.stride + i]);
            p[d] = __ldcg(&P.p[d * P.stride + i]);
        }
        pJ = __ldcg(&P.pJ[i]);
        if (!LAGGED) move(P, s_g, i, n, x, v, p);
    }
#pragma unroll
    for (int d = 0; d < 6; ++d) xe[d] = x[d];
    long long steps = 0, steps64 = 0;
    double J = evaluate_mixed_block(P, D, V, xe, active, steps, steps64);
    if (active) {
        if (J < pJ) {
            pJ = J;
#pragma unroll
            for (int d = 0; d < 6; ++d) p[d] = xe[d];
        }
        if (LAGGED) move(P, s_g, i, n, x, v, p);
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            P.x[d * P.stride + i] = x[d];
            P.v[d * P.stride + i] = v[d];
            P.p[d * P.stride + i] = p[d];
        }
        P.pJ[i] = pJ;
        P.J[i] = J;
    } else {
        J = CUDART_INF;
        steps = 0;
        steps64 = 0;
    }
    add_steps(P.gb, steps);
    add_steps64(P.gb, steps64);
    return reduce_to_global_best(P, J, i, xe, n, false, bidx, nblk);
}

// FP64 re-evaluation of every personal best and of the global best: the switch from
// the mixed exploration phase to the FP64 refinement phase.
__device__ __forceinline__ bool rescore_body(const KParams &P, int bidx, int nblk)
{
    if (!params_ok(P, bidx, nblk, 1, true)) return false;
    extern __shared__ double sm[];
    const ObsView O = stage_obs(P, sm);
    const CostW W = load_weights(P);
    const Dyn D = make_dyn(P);
    __shared__ int s_n;
    if (threadIdx.x == 0) s_n = __ldcg(&P.gb->iter);
    __syncthreads();
    const int i = bidx * blockDim.x + threadIdx.x;
    double p[6] = {0, 0, 0, 0, 0, 0};
    double J = CUDART_INF;
    long long steps = 0;
    if (i < P.m) {
#pragma unroll
        for (int d = 0; d < 6; ++d) p[d] = __ldcg(&P.p[d * P.stride + i]);
        J = evaluate<kRK4>(P, D, W, O, p, steps);
        P.pJ[i] = J;
    }
    add_steps(P.gb, steps);
    return reduce_to_global_best(P, J, i, p, s_n, true, bidx, nblk, kFlagRescored);
}


// ------------------------------------------------------------------ two threads per particle
// The FP64 swarm step of the circular problem with each particle on a lane pair
// (accel_pair), RK4 or DOPRI5.  Both lanes carry the particle; the even lane writes it
// back and takes part in the global best.  Both lanes of a pair run the whole
// propagation (pairs past the swarm's end follow particle 0 and are discarded).  RK4:
// for swarms too small to fill the GPU; DOPRI5, whose iteration is latency-bound: twice
// the threads to hide the latency of its long per-step chains.
template <int INTEG>
__device__ __forceinline__ double evaluate_pair(const KParams &P, const Dyn &D, const CostW &W,
                                                const ObsView &O, bool odd, const double x[6],
                                                long long &steps)
{
    double s[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) s[d] = x[d];
    double J = 0.0;
    if (INTEG == kRK4) {
        for (int k = 0; k < O.n; ++k) {
            const int n = O.ns[k];
            const RkH C = rk_h(O.h[k]);
            for (int j = 0; j < n; ++j) rk4_step_pair(D, odd, C, s);
            steps += n;
            add_epoch_cost(W, s[0] - O.rcx[k], s[1] - O.rcy[k], s[2] - O.rcz[k], O.ra[k], O.dec[k],
                           W.use_range ? O.rng[k] : 0.0, J);
        }
    } else {
        auto epoch = [&](int k, const double *st) {
            add_epoch_cost(W, st[0] - O.rcx[k], st[1] - O.rcy[k], st[2] - O.rcz[k], O.ra[k],
                           O.dec[k], W.use_range ? O.rng[k] : 0.0, J);
        };
        bool ok;
        steps += propagate_dopri5<0, 1>(D, s, O, P.rtol, P.atol, P.h0, P.max_steps, ok, epoch, odd);
        if (!ok) J = CUDART_INF;
    }
    return (isnan(J) || !isfinite(J)) ? CUDART_INF : J;
}

template <int INTEG>
__device__ __forceinline__ bool init_body_pair(const KParams &P, int bidx, int nblk)
{
    if (!params_ok(P, bidx, nblk, 2, true)) return false;
    extern __shared__ double sm[];
    const ObsView O = stage_obs(P, sm);
    const CostW W = load_weights(P);
    const Dyn D = make_dyn(P);
    __syncthreads();
    const int gt = bidx * blockDim.x + threadIdx.x;
    const int i = gt >> 1;
    const bool odd = gt & 1, lead = !odd && i < P.m;
    const int ii = i < P.m ? i : 0;
    double x[6];
    initial_position(P, ii, x);
    long long steps = 0;
    double J = evaluate_pair<INTEG>(P, D, W, O, odd, x, steps);
    if (lead) {
        double v0[6];
        initial_velocity(P, i, v0);
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            P.x[d * P.stride + i] = x[d];
            P.v[d * P.stride + i] = v0[d];
            P.p[d * P.stride + i] = x[d];
        }
        P.pJ[i] = J;
        P.J[i] = J;
    }
    add_steps(P.gb, lead ? steps : 0);
    return reduce_to_global_best(P, lead ? J : CUDART_INF, lead ? i : P.m, x, 0, true, bidx, nblk,
                                 kFlagStarted);
}

template <int INTEG, int LAGGED>
__device__ __forceinline__ bool iter_body_pair(const KParams &P, int bidx, int nblk)
{
    if (!params_ok(P, bidx, nblk, 2, true)) return false;
    extern __shared__ double sm[];
    const ObsView O = stage_obs(P, sm);
    const CostW W = load_weights(P);
    const Dyn D = make_dyn(P);
    __shared__ double s_g[6];
    __shared__ int s_n;
    if (threadIdx.x < 6) s_g[threadIdx.x] = __ldcg(&P.gb->g[threadIdx.x]);
    __shared__ int s_stop;
    if (threadIdx.x == 0) {
        s_n = __ldcg(&P.gb->iter) + 1;
        s_stop = __ldcg(&P.gb->flags) & kFlagStopped;
    }
    __syncthreads();
    if (s_stop) return false;     // Algorithm 2 ended the run: nothing more to do
    const int n = s_n;
    const int gt = bidx * blockDim.x + threadIdx.x;
    const int i = gt >> 1;
    const bool odd = gt & 1, lead = !odd && i < P.m;
    const int ii = i < P.m ? i : 0;
    double x[6], v[6], p[6], g[6], xe[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        x[d] = __ldcg(&P.x[d * P.stride + ii]);
        v[d] = __ldcg(&P.v[d * P.stride + ii]);
        p[d] = __ldcg(&P.p[d * P.stride + ii]);
        g[d] = s_g[d];
    }
    double pJ = __ldcg(&P.pJ[ii]);
    long long steps = 0;
    if (!LAGGED) move(P, g, ii, n, x, v, p);
#pragma unroll
    for (int d = 0; d < 6; ++d) xe[d] = x[d];
    const double J = evaluate_pair<INTEG>(P, D, W, O, odd, xe, steps);
    if (J < pJ) {
        pJ = J;
#pragma unroll
        for (int d = 0; d < 6; ++d) p[d] = xe[d];
    }
    if (LAGGED) move(P, g, ii, n, x, v, p);
    if (lead) {
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            P.x[d * P.stride + i] = x[d];
            P.v[d * P.stride + i] = v[d];
            P.p[d * P.stride + i] = p[d];
        }
        P.pJ[i] = pJ;
        P.J[i] = J;
    }
    add_steps(P.gb, lead ? steps : 0);
    return reduce_to_global_best(P, lead ? J : CUDART_INF, lead ? i : P.m, xe, n, false, bidx, nblk);
}

// ------------------------------------------------------------------ balanced FP64 iteration
// The FP64 pipe belongs to a sub-partition (4 per SM) and a warp costs it the same whether
// its 32 lanes are busy or not, so a swarm of G 32-particle groups run one warp per group
// takes as many group-times as its busiest sub-partition holds warps.  The balanced form
// keeps one to three warps resident per sub-partition (one block of 4, 8 or 12 warps per
// SM, cooperative launch) and gives every warp G / (its warps) group-times: the groups'
// work is laid end to end (epoch k weighs its RK4 steps plus kBalancedEpochWeight) and cut
// into equal shares at epoch boundaries.  A cut group is propagated up to the cut by the warp whose
// share ends in it, as that warp's first job, and finished by the next warp, as its last
// job, from the state and partial cost handed over through global memory; a share that
// lies inside one group (a middle piece: only when there are fewer groups than warps,
// which the host does not plan) takes the hand-off and passes it on.  Every particle's
// arithmetic is exactly that of iter_body, so the results are identical.

constexpr unsigned long long kHandoffWaitLimitNs = 20000000000ull;   // a hand-off wait gives up after 20 s

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned int *p, unsigned int v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Plan: G groups of gsize particles (32 for the FP64 warps, 384 for the mixed blocks);
// boundary j (j = 0..nw) at j G / nw groups of work, moved to the nearest epoch
// boundary of its group (a boundary at the group's end becomes the next group's start).
// One block; each thread computes every blockDim.x-th boundary.
// The plan's work line: group after group, epoch k of a group weighing wk(k); cut into nw
// equal shares at epoch boundaries (each cut at the boundary nearest its ideal place).
template <class W>
__device__ void plan_cuts(SplitCtl *S, int nw, int G, int K, W &&wk)
{
    double T = 0.0;
    for (int k = 0; k < K; ++k) T += wk(k);
    for (int j = threadIdx.x; j <= nw; j += blockDim.x) {
        const double B = (double)j * (double)G / (double)nw;
        int c = (int)floor(B);
        const double o = (B - (double)c) * T;
        int e = 0;
        double acc = 0.0;
        while (e < K) {
            const double w = wk(e);
            if (acc + 0.5 * w > o) break;
            acc += w;
            ++e;
        }
        if (e == K) {
            ++c;
            e = 0;
        }
        if (c >= G || j == nw) {
            c = G;
            e = 0;
        }
        if (j < nw) {
            S->seg[j].c0 = c;
            S->seg[j].e0 = e;
        }
        if (j > 0) {
            S->seg[j - 1].c1 = c;
            S->seg[j - 1].e1 = e;
        }
    }
}

// RK4: epoch k weighs its steps plus kBalancedEpochWeight.  DOPRI5: the chief's own
// attempts in interval k (thread 0 propagates it once; particles near the chief take
// about the same steps) plus kBalancedDpEpochWeight; the weights sit in dynamic shared
// memory (K floats).
__global__ void __launch_bounds__(256) split_plan_kernel(KParams P, int nw, int gsize)
{
    SplitCtl *S = P.split;
    const int K = P.n_obs, G = (P.m + gsize - 1) / gsize;
    if (threadIdx.x == 0) S->nw = nw;
    if (P.integrator == kDOPRI5) {
        extern __shared__ float s_w[];
        if (threadIdx.x == 0) {
            const Dyn D = make_dyn(P);
            const ObsView O{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, P.t, P.h, P.nsteps, K};
            auto none = [](int, const double *) {};
            DpState st;
            dopri5_begin<0>(D, st, P.chief0, O, P.h0, none);
            long long before = 0;
            for (int k = 0; k < K; ++k) {
                dopri5_advance<0>(D, st, O, P.rtol, P.atol, P.max_steps, k + 1, none);
                s_w[k] = (float)(st.steps - before) + kBalancedDpEpochWeight;
                before = st.steps;
            }
        }
        __syncthreads();
        plan_cuts(S, nw, G, K, [&](int k) { return (double)s_w[k]; });
    } else {
        plan_cuts(S, nw, G, K, [&](int k) { return (double)P.nsteps[k] + kBalancedEpochWeight; });
    }
}

// Waits (lane 0 of the warp) until flag holds stamp; false once limit_ns have passed.
__device__ __forceinline__ bool wait_handoff(const unsigned int *flag, unsigned int stamp,
                                             unsigned long long limit_ns = kHandoffWaitLimitNs)
{
    const unsigned long long t0 = tma::globaltimer_ns();
    for (;;) {
        if (ld_acquire_u32(flag) == stamp) return true;
        if (tma::globaltimer_ns() - t0 > limit_ns) return false;
        __nanosleep(256);
    }
}

// Diagnostic of the hand-off wait: one thread waits on *flag for stamp with limit_ns;
// writes whether it gave up and how long it waited.
__global__ void wait_probe_kernel(const unsigned int *flag, unsigned int stamp,
                                  unsigned long long limit_ns, int *timed_out,
                                  unsigned long long *waited_ns)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const unsigned long long t0 = tma::globaltimer_ns();
    const bool ok = wait_handoff(flag, stamp, limit_ns);
    *waited_ns = tma::globaltimer_ns() - t0;
    *timed_out = ok ? 0 : 1;
}

// Diagnostic of the FP64 pipe: in one block of `warps` warps, lanes [0, lanes) of every
// warp run a dependent chain of n FP64 FMAs; each warp's lane 0 writes the SM cycles the
// chain took.  sink[threadIdx.x] keeps the chain's value (so that it is computed).
__global__ void __launch_bounds__(1024) fp64_issue_probe_kernel(int lanes, int n, long long *cycles, double *sink)
{
    double a = 1.0 + 1e-3 * (double)threadIdx.x;
    const double b = 1.0000001, c = 1e-9;
    __syncthreads();
    const long long t0 = clock64();
    if ((int)(threadIdx.x & 31u) < lanes)
        for (int i = 0; i < n; ++i) a = fma(a, b, c);
    const long long t1 = clock64();
    sink[threadIdx.x] = a;
    if ((threadIdx.x & 31u) == 0u) cycles[threadIdx.x >> 5] = t1 - t0;
}

// MODE 0: an iteration, synchronous global best; 1: Algorithm 1's lagged order; 2: the
// initial evaluation (init_body's work: initial positions and velocities, first bests).
// ER = 1: the elliptic problem.
template <int MODE, int ER>
__global__ void __launch_bounds__(32 * kBalancedMaxWarpsPerSm, 1) iter_kernel_balanced(KParams P)
{
    if (!params_ok(P, blockIdx.x, gridDim.x, 0, true)) return;
    constexpr bool LAGGED = MODE == 1, INIT = MODE == 2;
    extern __shared__ double sm[];
    const ObsView O = stage_obs(P, sm);
    const CostW W = load_weights(P);
    const Dyn D = make_dyn(P);
    SplitCtl *S = P.split;
    __shared__ double s_g[6];
    __shared__ int s_n, s_stop;
    __shared__ unsigned int s_stamp;
    if (threadIdx.x < 6) s_g[threadIdx.x] = INIT ? 0.0 : __ldcg(&P.gb->g[threadIdx.x]);
    if (threadIdx.x == 0) {
        s_n = INIT ? 0 : __ldcg(&P.gb->iter) + 1;
        s_stop = INIT ? 0 : (__ldcg(&P.gb->flags) & kFlagStopped);
        s_stamp = __ldcg(&S->stamp) + 1u;
    }
    __syncthreads();
    if (s_stop) return;     // Algorithm 2 ended the run: nothing more to do
    const int n = s_n;
    const unsigned int stamp = s_stamp;
    const int lane = threadIdx.x & 31;
    const int wj = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int G = (P.m + 31) >> 5;
    const SplitSeg sg = S->seg[wj];
    double g[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) g[d] = s_g[d];
    // this lane's best among the particles it finished
    double bJ = CUDART_INF, bx[6] = {0, 0, 0, 0, 0, 0};
    int bI = INT_MAX;
    long long steps = 0;

    // Group c over epochs [ea, eb).  in: take over the previous warp's hand-off; out: hand
    // this warp's state on to the next warp instead of finishing the particles.
    auto part = [&](int c, int ea, int eb, bool in, bool out) {
        const int i = c * 32 + lane;
        const bool act = i < P.m;
        double s[6], J = 0.0;
        if (in) {
            int ok = 1;
            if (lane == 0) ok = wait_handoff(&S->flag[wj - 1], stamp);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                if (lane == 0) atomicOr(&P.gb->status, kStatusHandoffTimeout);
                return;
            }
            __threadfence();
            const double *h = S->hand + (size_t)(wj - 1) * 7 * 32;
#pragma unroll
            for (int d = 0; d < 6; ++d) s[d] = __ldcg(&h[d * 32 + lane]);
            J = __ldcg(&h[6 * 32 + lane]);
        }
        double x[6], v[6], p[6], xe[6], pJ = CUDART_INF;
        if (act) {
            if (INIT) {
                // a pure function of i: the group's second warp recomputes it
                initial_position(P, i, x);
            } else {
#pragma unroll
                for (int d = 0; d < 6; ++d) {
                    x[d] = __ldcg(&P.x[d * P.stride + i]);
                    v[d] = __ldcg(&P.v[d * P.stride + i]);
                    p[d] = __ldcg(&P.p[d * P.stride + i]);
                }
                pJ = __ldcg(&P.pJ[i]);
            }
            // synchronous order: the group's first warp moves the particle (and stores the
            // moved state before any hand-off); the evaluated position is x either way
            if (!INIT && !LAGGED && !in) move(P, g, i, n, x, v, p);
#pragma unroll
            for (int d = 0; d < 6; ++d) xe[d] = x[d];
            if (!in) {
#pragma unroll
                for (int d = 0; d < 6; ++d) s[d] = x[d];
            }
            auto epoch = [&](int k, const double *st) {
                add_epoch_cost(W, st[0] - O.rcx[k], st[1] - O.rcy[k], st[2] - O.rcz[k], O.ra[k],
                               O.dec[k], W.use_range ? O.rng[k] : 0.0, J);
            };
            steps += propagate_rk4_epochs<ER>(D, s, O, ea, eb, epoch);
        }
        if (out) {
            double *h = S->hand + (size_t)wj * 7 * 32;
#pragma unroll
            for (int d = 0; d < 6; ++d) h[d * 32 + lane] = s[d];
            h[6 * 32 + lane] = J;
            if (act && !INIT && !LAGGED && !in) {
#pragma unroll
                for (int d = 0; d < 6; ++d) {
                    P.x[d * P.stride + i] = x[d];
                    P.v[d * P.stride + i] = v[d];
                }
            }
            __threadfence();
            __syncwarp();
            if (lane == 0) st_release_u32(&S->flag[wj], stamp);
            return;
        }
        if (!act) return;
        J = (isnan(J) || !isfinite(J)) ? CUDART_INF : J;
        if (INIT) {
            initial_velocity(P, i, v);
#pragma unroll
            for (int d = 0; d < 6; ++d) p[d] = xe[d];
            pJ = J;
        } else if (J < pJ) {
            pJ = J;
#pragma unroll
            for (int d = 0; d < 6; ++d) p[d] = xe[d];
        }
        if (LAGGED) move(P, g, i, n, x, v, p);
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            P.x[d * P.stride + i] = x[d];
            P.v[d * P.stride + i] = v[d];
            P.p[d * P.stride + i] = p[d];
        }
        P.pJ[i] = pJ;
        P.J[i] = J;
        if (better(J, i, bJ, bI)) {
            bJ = J;
            bI = i;
#pragma unroll
            for (int d = 0; d < 6; ++d) bx[d] = xe[d];
        }
    };

    // the warp's jobs, in order: the head it hands on (first), its whole groups, the tail
    // it takes over (last); one call site, so the propagation is compiled once
    const bool has_in = sg.e0 > 0;
    const bool has_out = sg.e1 > 0 && sg.c1 < G;
    const bool middle = has_in && has_out && sg.c0 == sg.c1;
    const int head = (has_out && !middle) ? 1 : 0;
    const int cf = has_in ? sg.c0 + 1 : sg.c0;
    const int nfull = sg.c1 > cf ? sg.c1 - cf : 0;
    const int njobs = head + nfull + (has_in ? 1 : 0);
    for (int q = 0; q < njobs; ++q) {
        int c = cf + (q - head), ea = 0, eb = O.n;
        bool in = false, out = false;
        if (q < head) {
            c = sg.c1;
            eb = sg.e1;
            out = true;
        } else if (q >= head + nfull) {
            c = sg.c0;
            ea = sg.e0;
            eb = middle ? sg.e1 : O.n;
            in = true;
            out = middle;
        }
        part(c, ea, eb, in, out);
    }
    add_steps(P.gb, steps);
    const bool last = reduce_to_global_best(P, bJ, bI, bx, n, INIT, blockIdx.x, gridDim.x,
                                            INIT ? kFlagStarted : 0);
    if (last && threadIdx.x == 0) {
        S->stamp = stamp;
        __threadfence();
    }
}

// Balanced FP64 DOPRI5 iteration (circular problem), the RK4 balanced kernel's schedule
// for adaptive steps: a group cut at epoch e is propagated by the first warp until its next
// epoch to emit is e or later, and the second warp resumes from the integrator's whole loop
// state (DpState: state, FSAL stage, step size, time, next epoch, attempts, validity) and
// the partial cost, so every particle takes the attempts of an uncut propagation, bit for
// bit.  The plan weighs each interval by the chief's own attempts.
template <int MODE>
__global__ void __launch_bounds__(32 * kBalancedDpMaxWarpsPerSm, 1) iter_kernel_balanced_dp(KParams P)
{
    if (!params_ok(P, blockIdx.x, gridDim.x, 0, true)) return;
    constexpr bool LAGGED = MODE == 1, INIT = MODE == 2;
    extern __shared__ double sm[];
    const ObsView O = stage_obs(P, sm);
    const CostW W = load_weights(P);
    const Dyn D = make_dyn(P);
    SplitCtl *S = P.split;
    __shared__ double s_g[6];
    __shared__ int s_n, s_stop;
    __shared__ unsigned int s_stamp;
    if (threadIdx.x < 6) s_g[threadIdx.x] = INIT ? 0.0 : __ldcg(&P.gb->g[threadIdx.x]);
    if (threadIdx.x == 0) {
        s_n = INIT ? 0 : __ldcg(&P.gb->iter) + 1;
        s_stop = INIT ? 0 : (__ldcg(&P.gb->flags) & kFlagStopped);
        s_stamp = __ldcg(&S->stamp) + 1u;
    }
    __syncthreads();
    if (s_stop) return;     // Algorithm 2 ended the run: nothing more to do
    const int n = s_n;
    const unsigned int stamp = s_stamp;
    const int lane = threadIdx.x & 31;
    const int wj = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int G = (P.m + 31) >> 5;
    const SplitSeg sg = S->seg[wj];
    double g[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) g[d] = s_g[d];
    double bJ = CUDART_INF, bx[6] = {0, 0, 0, 0, 0, 0};
    int bI = INT_MAX;
    long long steps = 0;

    // Group c up to the epoch `stop_at` (out) or to the end.  in: resume from the previous
    // warp's hand-off; out: hand this warp's integrator state on instead of finishing.
    auto part = [&](int c, int stop_at, bool in, bool out) {
        const int i = c * 32 + lane;
        const bool act = i < P.m;
        DpState st;
        double J = 0.0;
        long long st0 = 0;
        if (in) {
            int ok = 1;
            if (lane == 0) ok = wait_handoff(&S->flag[wj - 1], stamp);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                if (lane == 0) atomicOr(&P.gb->status, kStatusHandoffTimeout);
                return;
            }
            __threadfence();
            const double *h = S->hand + (size_t)(wj - 1) * kDpHandRows * 32;
#pragma unroll
            for (int d = 0; d < 6; ++d) {
                st.s[d] = __ldcg(&h[d * 32 + lane]);
                st.k1[d] = __ldcg(&h[(6 + d) * 32 + lane]);
            }
            st.h = __ldcg(&h[12 * 32 + lane]);
            st.tc = __ldcg(&h[13 * 32 + lane]);
            J = __ldcg(&h[14 * 32 + lane]);
            st.next = (int)__ldcg(&h[15 * 32 + lane]);
            st.ok = (int)__ldcg(&h[16 * 32 + lane]);
            st.steps = (long long)__ldcg(&h[17 * 32 + lane]);
            st0 = st.steps;
        }
        double x[6], v[6], p[6], xe[6], pJ = CUDART_INF;
        if (act) {
            if (INIT) {
                initial_position(P, i, x);      // a pure function of i
            } else {
#pragma unroll
                for (int d = 0; d < 6; ++d) {
                    x[d] = __ldcg(&P.x[d * P.stride + i]);
                    v[d] = __ldcg(&P.v[d * P.stride + i]);
                    p[d] = __ldcg(&P.p[d * P.stride + i]);
                }
                pJ = __ldcg(&P.pJ[i]);
            }
            if (!INIT && !LAGGED && !in) move(P, g, i, n, x, v, p);
#pragma unroll
            for (int d = 0; d < 6; ++d) xe[d] = x[d];
        }
        auto epoch = [&](int k, const double *y) {
            add_epoch_cost(W, y[0] - O.rcx[k], y[1] - O.rcy[k], y[2] - O.rcz[k], O.ra[k],
                           O.dec[k], W.use_range ? O.rng[k] : 0.0, J);
        };
        if (act && !in) dopri5_begin<0>(D, st, x, O, P.h0, epoch);
        {   // the whole warp: lanes without a particle only take part in the warp's steps
            DpEpochBuf buf;
            dopri5_advance_warp(D, st, O, P.rtol, P.atol, P.max_steps, out ? stop_at : O.n, act, buf, epoch);
        }
        if (act) steps += st.steps - st0;
        if (out) {
            double *h = S->hand + (size_t)wj * kDpHandRows * 32;
            if (act) {
#pragma unroll
                for (int d = 0; d < 6; ++d) {
                    h[d * 32 + lane] = st.s[d];
                    h[(6 + d) * 32 + lane] = st.k1[d];
                }
                h[12 * 32 + lane] = st.h;
                h[13 * 32 + lane] = st.tc;
                h[14 * 32 + lane] = J;
                h[15 * 32 + lane] = (double)st.next;
                h[16 * 32 + lane] = (double)st.ok;
                h[17 * 32 + lane] = (double)st.steps;
            }
            if (act && !INIT && !LAGGED && !in) {
#pragma unroll
                for (int d = 0; d < 6; ++d) {
                    P.x[d * P.stride + i] = x[d];
                    P.v[d * P.stride + i] = v[d];
                }
            }
            __threadfence();
            __syncwarp();
            if (lane == 0) st_release_u32(&S->flag[wj], stamp);
            return;
        }
        if (!act) return;
        J = (!st.ok || isnan(J) || !isfinite(J)) ? CUDART_INF : J;
        if (INIT) {
            initial_velocity(P, i, v);
#pragma unroll
            for (int d = 0; d < 6; ++d) p[d] = xe[d];
            pJ = J;
        } else if (J < pJ) {
            pJ = J;
#pragma unroll
            for (int d = 0; d < 6; ++d) p[d] = xe[d];
        }
        if (LAGGED) move(P, g, i, n, x, v, p);
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            P.x[d * P.stride + i] = x[d];
            P.v[d * P.stride + i] = v[d];
            P.p[d * P.stride + i] = p[d];
        }
        P.pJ[i] = pJ;
        P.J[i] = J;
        if (better(J, i, bJ, bI)) {
            bJ = J;
            bI = i;
#pragma unroll
            for (int d = 0; d < 6; ++d) bx[d] = xe[d];
        }
    };

    // the warp's jobs, in order: the head it hands on (first), its whole groups, the tail
    // it takes over (last)
    const bool has_in = sg.e0 > 0;
    const bool has_out = sg.e1 > 0 && sg.c1 < G;
    const bool middle = has_in && has_out && sg.c0 == sg.c1;
    const int head = (has_out && !middle) ? 1 : 0;
    const int cf = has_in ? sg.c0 + 1 : sg.c0;
    const int nfull = sg.c1 > cf ? sg.c1 - cf : 0;
    const int njobs = head + nfull + (has_in ? 1 : 0);
    for (int q = 0; q < njobs; ++q) {
        int c = cf + (q - head), stop_at = O.n;
        bool in = false, out = false;
        if (q < head) {
            c = sg.c1;
            stop_at = sg.e1;
            out = true;
        } else if (q >= head + nfull) {
            c = sg.c0;
            stop_at = middle ? sg.e1 : O.n;
            in = true;
            out = middle;
        }
        part(c, stop_at, in, out);
    }
    add_steps(P.gb, steps);
    const bool last = reduce_to_global_best(P, bJ, bI, bx, n, INIT, blockIdx.x, gridDim.x,
                                            INIT ? kFlagStarted : 0);
    if (last && threadIdx.x == 0) {
        S->stamp = stamp;
        __threadfence();
    }
}

// Balanced mixed-precision iteration.  The mixed evaluation is block-synchronous (the
// chief-table chunks a block stages in shared memory serve all its warps), so the unit
// cut at epoch boundaries is a super-group of 384 particles: one 384-thread block per SM
// (twelve warps, three per sub-partition) takes an equal share of the super-groups laid
// end to end, every warp the same epochs of its own 32 particles.  A cut super-group's
// FP32 offsets, their compensations and the partial costs are handed from one block to
// the next through global memory, as in iter_kernel_balanced.  Each particle's arithmetic
// is that of iter_mixed_body.
template <int LAGGED>
__global__ void __launch_bounds__(kMixedBalancedThreads, 1) iter_mixed_balanced(KParams P)
{
    if (!params_ok(P, blockIdx.x, gridDim.x, 0, false)) return;
    extern __shared__ __align__(128) unsigned char smb[];
    const MixView V = stage_mixed(P, smb);
    const Dyn D = make_dyn(P);
    SplitCtl *S = P.split;
    __shared__ double s_g[6];
    __shared__ int s_n, s_stop, s_ok;
    __shared__ unsigned int s_stamp;
    if (threadIdx.x < 6) s_g[threadIdx.x] = __ldcg(&P.gb->g[threadIdx.x]);
    if (threadIdx.x == 0) {
        s_n = __ldcg(&P.gb->iter) + 1;
        s_stop = __ldcg(&P.gb->flags) & kFlagStopped;
        s_stamp = __ldcg(&S->stamp) + 1u;
        mixed_copy_lost() = 0;
    }
    __syncthreads();
    if (s_stop) return;     // Algorithm 2 ended the run: nothing more to do
    const int n = s_n;
    const unsigned int stamp = s_stamp;
    const int b = blockIdx.x, t = threadIdx.x, NT = blockDim.x;
    const int G = (P.m + NT - 1) / NT;
    const SplitSeg sg = S->seg[b];
    double bJ = CUDART_INF, bx[6] = {0, 0, 0, 0, 0, 0};
    int bI = INT_MAX;
    long long steps = 0, steps64 = 0;

    // Super-group cg over epochs [ea, eb) (block-collective).  in: take over the previous
    // block's hand-off; out: hand this block's offsets on instead of finishing.
    auto part = [&](int cg, int ea, int eb, bool in, bool out) {
        const int i = cg * NT + t;
        const bool act = i < P.m;
        float d[6], c[6];
        double J = 0.0;
        if (in) {
            if (t == 0) s_ok = wait_handoff(&S->flag[b - 1], stamp);
            __syncthreads();
            if (!s_ok) {
                if (t == 0) atomicOr(&P.gb->status, kStatusHandoffTimeout);
                return;
            }
            __threadfence();
            const double *h = S->hand + (size_t)(b - 1) * 13 * NT;
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                d[q] = (float)__ldcg(&h[q * NT + t]);
                c[q] = (float)__ldcg(&h[(6 + q) * NT + t]);
            }
            J = __ldcg(&h[12 * NT + t]);
        }
        double x[6], v[6], p[6], xe[6], pJ = CUDART_INF;
#pragma unroll
        for (int q = 0; q < 6; ++q) x[q] = P.chief_cs[q];   // lanes past the swarm: the chief
        if (act) {
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                x[q] = __ldcg(&P.x[q * P.stride + i]);
                v[q] = __ldcg(&P.v[q * P.stride + i]);
                p[q] = __ldcg(&P.p[q * P.stride + i]);
            }
            pJ = __ldcg(&P.pJ[i]);
            if (!LAGGED && !in) move(P, s_g, i, n, x, v, p);
        }
#pragma unroll
        for (int q = 0; q < 6; ++q) xe[q] = x[q];
        if (!in) mixed_offset(P, xe, d, c);
        long long st = 0, st64 = 0;
        // after a copy that never landed this block's buffers are not used again (the
        // problem already carries the failure status)
        const bool ok = !mixed_copy_lost() && mixed_epochs(P, D, V, ea, eb, d, c, J, act, st, st64);
        if (act) {
            steps += st;
            steps64 += st64;
        }
        if (out) {
            double *h = S->hand + (size_t)b * 13 * NT;
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                h[q * NT + t] = (double)d[q];
                h[(6 + q) * NT + t] = (double)c[q];
            }
            h[12 * NT + t] = J;
            if (act && !LAGGED && !in) {
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    P.x[q * P.stride + i] = x[q];
                    P.v[q * P.stride + i] = v[q];
                }
            }
            __threadfence();
            __syncthreads();
            if (t == 0) st_release_u32(&S->flag[b], stamp);
            return;
        }
        if (!act) return;
        J = (!ok || isnan(J) || !isfinite(J)) ? CUDART_INF : J;
        if (J < pJ) {
            pJ = J;
#pragma unroll
            for (int q = 0; q < 6; ++q) p[q] = xe[q];
        }
        if (LAGGED) move(P, s_g, i, n, x, v, p);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            P.x[q * P.stride + i] = x[q];
            P.v[q * P.stride + i] = v[q];
            P.p[q * P.stride + i] = p[q];
        }
        P.pJ[i] = pJ;
        P.J[i] = J;
        if (better(J, i, bJ, bI)) {
            bJ = J;
            bI = i;
#pragma unroll
            for (int q = 0; q < 6; ++q) bx[q] = xe[q];
        }
    };

    const bool has_in = sg.e0 > 0;
    const bool has_out = sg.e1 > 0 && sg.c1 < G;
    const bool middle = has_in && has_out && sg.c0 == sg.c1;
    const int head = (has_out && !middle) ? 1 : 0;
    const int cf = has_in ? sg.c0 + 1 : sg.c0;
    const int nfull = sg.c1 > cf ? sg.c1 - cf : 0;
    const int njobs = head + nfull + (has_in ? 1 : 0);
    for (int q = 0; q < njobs; ++q) {
        int cg = cf + (q - head), ea = 0, eb = V.n;
        bool in = false, out = false;
        if (q < head) {
            cg = sg.c1;
            eb = sg.e1;
            out = true;
        } else if (q >= head + nfull) {
            cg = sg.c0;
            ea = sg.e0;
            eb = middle ? sg.e1 : V.n;
            in = true;
            out = middle;
        }
        part(cg, ea, eb, in, out);
    }
    add_steps(P.gb, steps);
    add_steps64(P.gb, steps64);
    const bool last = reduce_to_global_best(P, bJ, bI, bx, n, false, b, gridDim.x);
    if (last && t == 0) {
        S->stamp = stamp;
        __threadfence();
    }
}

// ------------------------------------------------------------------ single-problem kernels
template <int INTEG>
__global__ void __launch_bounds__(kMaxThreads) init_kernel(KParams P)
{
    if (INTEG == kDOPRI5 && P.dynamics)
        init_body<INTEG, 1>(P, blockIdx.x, gridDim.x);
    else
        init_body<INTEG, 0>(P, blockIdx.x, gridDim.x);
}

template <int INTEG>
__global__ void __launch_bounds__(kMaxThreads) init_kernel_pair(KParams P)
{
    init_body_pair<INTEG>(P, blockIdx.x, gridDim.x);
}

template <int INTEG, int LAGGED>
__global__ void __launch_bounds__(kMaxThreads) iter_kernel_pair(KParams P)
{
    iter_body_pair<INTEG, LAGGED>(P, blockIdx.x, gridDim.x);
}

// the same kernels for the elliptic problem with RK4 (separate instantiations, so the
// circular problem's kernels are compiled exactly as without them); held to 128
// registers, so sixteen one-warp blocks stay resident per SM as in the circular kernels
__global__ void __launch_bounds__(kMaxThreads, 2) init_kernel_er(KParams P) { init_body<kRK4, 1>(P, blockIdx.x, gridDim.x); }

template <int LAGGED>
__global__ void __launch_bounds__(kMaxThreads, 2) iter_kernel_er(KParams P)
{
    iter_body<kRK4, LAGGED, 1>(P, blockIdx.x, gridDim.x);
}

template <int INTEG, int LAGGED>
__global__ void __launch_bounds__(kMaxThreads) iter_kernel(KParams P)
{
    if (INTEG == kDOPRI5 && P.dynamics)
        iter_body<INTEG, LAGGED, 1>(P, blockIdx.x, gridDim.x);
    else
        iter_body<INTEG, LAGGED, 0>(P, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(kMaxThreads, 2) init_mixed_kernel(KParams P) { init_mixed_body(P, blockIdx.x, gridDim.x); }

template <int LAGGED>
__global__ void __launch_bounds__(kMaxThreads, 2) iter_mixed_kernel(KParams P)
{
    iter_mixed_body<LAGGED>(P, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(kMaxThreads) rescore_kernel(KParams P) { rescore_body(P, blockIdx.x, gridDim.x); }

__global__ void __launch_bounds__(kMaxThreads, 2) eval_mixed_kernel(KParams P, const double *__restrict__ X,
                                                                    int m, double *__restrict__ Jout,
                                                                    double *__restrict__ states)
{
    extern __shared__ __align__(128) unsigned char smb[];
    const MixView V = stage_mixed(P, smb);
    const Dyn D = make_dyn(P);
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = i < m;
    double x[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) x[d] = active ? X[(size_t)d * m + i] : P.chief_cs[d];
    long long steps = 0, steps64 = 0;
    const double J = evaluate_mixed_block(P, D, V, x, active, steps, steps64, states, m, i);
    if (active && !states) Jout[i] = J;
}


// ------------------------------------------------------------------ batches
// Set-up of newly admitted problems, one block each: the FP64 set-up (interval table,
// weights, chief trajectory), then the mixed-precision tables (all threads of the block).  The step count per
// propagation is written back into the slot's descriptor.
__global__ void batch_setup_kernel(BatchSlot *slots, const int *__restrict__ ids, int n)
{
    if (blockIdx.x >= n) return;
    BatchSlot &B = slots[ids[blockIdx.x]];
    // the FP64 set-up on a lane pair (batches run the circular problem with RK4), which
    // also records the chief's step-boundary states for the mixed-precision table
    if (threadIdx.x < 2) {
        const long long S = setup_body(B.P, B.vmax_frac, B.sig_ra, B.sig_dec, B.sig_rng, B.chief, B.rc_w,
                                       B.ns_w, B.h_w, B.cst_w, B.P.gb, threadIdx.x, true,
                                       B.n_mixed >= 0 ? B.cs_w : nullptr);
        if (threadIdx.x == 0) B.P.total_steps = S;
    }
    __syncthreads();
    if (B.n_mixed >= 0) setup_mixed_body(B.P, B.mix_w, B.cs_w, B.od_w, B.ct_w, threadIdx.x, blockDim.x);
}

__device__ bool refine_body(const KParams &P, int max_iters, double sig_ra, double sig_dec, double *R);

// The refinement gate's restart: the request's record cleared for an FP64 solve from the
// start (kFlagFallback set; the step counters keep counting), so that the next action is
// the FP64 initialisation of the same initial swarm.  Returns true in every thread.
__device__ bool restart_body(const KParams &P)
{
    if (threadIdx.x == 0) {
        GBest *gb = P.gb;
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            gb->g[d] = 0.0;
            gb->g_pso[d] = 0.0;
        }
        gb->gJ = 0.0;
        gb->gidx = 0;
        gb->iter = 0;
        gb->done_blocks = 0u;
        for (int q = 0; q < kTolHist; ++q) gb->hist[q] = 0.0;
        gb->gJ_pso = 0.0;
        gb->lm_iters = 0;
        gb->lm_status = 0;
        gb->lm_lam = 0.0;
        gb->flags = kFlagFallback;
        __threadfence();
    }
    __syncthreads();
    return true;
}

// A resident problem's next action, from its device state (read from L2: the state may
// have been written by another SM in the same launch).
__device__ __forceinline__ int decide_action(const BatchSlot &B)
{
    if (!__ldcg(&B.active)) return kActNone;
    const GBest *gb = B.P.gb;
    const int it = __ldcg(&gb->iter), fl = __ldcg(&gb->flags);
    if (__ldcg(&gb->status)) return kActNone;
    const bool fallback = fl & kFlagFallback;              // the FP64 solve of the gate
    const int n_mixed = fallback ? -1 : B.n_mixed;
    if (!(fl & kFlagStarted)) return n_mixed >= 0 ? kActInitMixed : kActInitFP64;
    const bool stopped = fl & kFlagStopped;    // Algorithm 2 ended the iterations
    if (n_mixed >= 0 && it < n_mixed && !stopped) return kActIterMixed;
    if (n_mixed >= 0 && !(fl & kFlagRescored)) return kActRescore;
    if (it < B.n_iters && !stopped) return kActIterFP64;
    const bool gated = B.gate_cost > 0.0 && !fallback && !(__ldcg(&gb->gJ) <= B.gate_cost);
    if (B.refine_iters > 0 && !(fl & kFlagRefined)) {
        // a refinement still above the gate after kLmGateIters iterations gives up
        if (gated && (fl & kFlagLmStarted) && __ldcg(&gb->lm_iters) >= kLmGateIters) return kActRestart;
        return kActRefine;
    }
    if (gated) return kActRestart;
    return kActNone;
}

// Tiles of an action: the swarm actions cover the swarm; the refinement is one block.
__device__ __forceinline__ int action_tiles(const BatchSlot &B, int act)
{
    return (act == kActRefine || act == kActRestart) ? 1 : B.n_tiles;
}

// One action per resident problem for the coming round.
__global__ void batch_plan_kernel(BatchSlot *slots, int n_slots)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_slots) return;
    slots[s].action = decide_action(slots[s]);
}

// Run one tile of a problem's current action; true in the block that folded the
// problem's global best (its last tile of the action).
__device__ __forceinline__ bool run_action(const BatchSlot &B, int act, int tile)
{
    switch (act) {
    case kActInitMixed: return init_mixed_body(B.P, tile, B.n_tiles);
    case kActIterMixed: return iter_mixed_body<0>(B.P, tile, B.n_tiles);
    case kActInitFP64: return init_body<kRK4>(B.P, tile, B.n_tiles);
    case kActIterFP64: return iter_body<kRK4, 0>(B.P, tile, B.n_tiles);
    case kActRescore: return rescore_body(B.P, tile, B.n_tiles);
    case kActRefine: return tile == 0 ? refine_body(B.P, B.refine_iters, B.sig_ra, B.sig_dec, B.lm_R) : false;
    case kActRestart: return tile == 0 ? restart_body(B.P) : false;
    default: return false;
    }
}

// One round over tiles (slot, block of that slot): blocks pull tiles from an atomic
// queue until it is empty (grid sized to the resident capacity), run that slot's action
// on the tile -- FP32 and FP64 actions alike, so one launch covers every resident
// problem -- and the slot's last tile folds its global best.  The last block out resets
// the queue for the next launch.
__global__ void __launch_bounds__(kMaxThreads, 2) batch_round_kernel(BatchSlot *slots, const int2 *__restrict__ tiles,
                                                                     int n_tiles, BatchQueue *q)
{
    __shared__ int s_t;
    __shared__ bool s_last;
    if (threadIdx.x == 0) mixed_copy_lost() = 0;
    for (;;) {
        if (threadIdx.x == 0) s_t = (int)atomicAdd(&q->next, 1u);
        __syncthreads();
        const int t = s_t;
        __syncthreads();
        if (t >= n_tiles) break;
        const int2 tl = tiles[t];
        const BatchSlot &B = slots[tl.x];
        run_action(B, B.action, tl.y);
        __syncthreads();
        // a chief-table copy of this block never landed: its shared memory may still be
        // written, so it takes no further tile (the others take them)
        if (mixed_copy_lost()) break;
    }
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&q->done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        q->next = 0u;
        q->done = 0u;
        __threadfence();
    }
}


// ------------------------------------------------------------------ dependency-driven scheduler
constexpr unsigned long long kWqWaitLimitNs = 20000000000ull;   // a claim wait gives up after 20 s

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_acquire_s32(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Publish the n tiles of slot s's next action (all threads of the block call this).
__device__ __forceinline__ void wq_push(WorkQueue *q, int2 *ring, unsigned long long *seq,
                                        unsigned long long cap, int s, int n)
{
    __shared__ unsigned long long s_base;
    if (threadIdx.x == 0) s_base = atomicAdd(&q->tail, (unsigned long long)n);
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const unsigned long long c = s_base + (unsigned long long)j;
        ring[c % cap] = make_int2(s, j);
        st_release_u64(&seq[c % cap], c);   // orders the item (and the slot's state) before it
    }
}

// Start of a launch: move both indices past everything earlier, then publish every
// resident problem's next action.  One block.
__global__ void wq_seed_kernel(BatchSlot *slots, int n_slots, WorkQueue *q, int2 *ring,
                               unsigned long long *seq, unsigned long long cap)
{
    if (threadIdx.x == 0) {
        const unsigned long long base = q->head > q->tail ? q->head : q->tail;
        q->head = base;
        q->tail = base;
        q->active = 0;
        q->status = 0;
        q->t0 = 0ull;
        __threadfence();
    }
    __syncthreads();
    for (int s = threadIdx.x; s < n_slots; s += blockDim.x) {
        BatchSlot &B = slots[s];
        const int act = decide_action(B);
        B.action = act;
        if (act == kActNone) continue;
        const int nt = action_tiles(B, act);
        const unsigned long long base = atomicAdd(&q->tail, (unsigned long long)nt);
        for (int j = 0; j < nt; ++j) {
            ring[(base + j) % cap] = make_int2(s, j);
            seq[(base + j) % cap] = base + j;
        }
        atomicAdd(&q->active, 1);
    }
}

// The persistent scheduler: blocks (all co-resident: cooperative launch) claim item
// indices in order and wait for them to be published; a problem's last tile of an
// action publishes its next action at once (until the device-time budget is spent),
// so problems advance independently.  Blocks leave when no problem has work left in
// this launch, or when one wait has lasted kWqWaitLimitNs (status kWqTimeout).
// MINB resident blocks of 256 threads per SM at least: 2 (128 registers, no spills) keeps
// each block's chains fastest, the latency form for a few requests; 3 (80 registers, the
// bodies spilling about a kilobyte per thread to local memory) runs a full batch 5%
// faster (64 registers: 16% slower), the throughput form.
template <int MINB>
__global__ void __launch_bounds__(kMaxThreads, MINB) wq_kernel(BatchSlot *slots, WorkQueue *q, int2 *ring,
                                                            unsigned long long *seq, unsigned long long cap,
                                                            unsigned long long budget_ns)
{
    __shared__ int2 s_item;
    __shared__ int s_exit;
    __shared__ unsigned long long s_deadline;
    if (threadIdx.x == 0) {
        const unsigned long long now = globaltimer();
        const unsigned long long old = atomicCAS(&q->t0, 0ull, now);
        const unsigned long long t0 = old ? old : now;
        s_deadline = budget_ns ? t0 + budget_ns : ~0ull;
        mixed_copy_lost() = 0;
    }
    __syncthreads();
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned long long c = atomicAdd(&q->head, 1ull);
            int ex = 0;
            unsigned int ns = 32;
            const unsigned long long w0 = globaltimer();
            for (;;) {
                if (ld_acquire_s32(&q->status) & kWqCopyLost) {
                    ex = 1;
                    break;
                }
                if (ld_acquire_u64(&seq[c % cap]) == c) break;
                if (ld_acquire_s32(&q->active) == 0) {
                    // nothing will be published any more (re-check once: ordering)
                    if (ld_acquire_u64(&seq[c % cap]) != c) ex = 1;
                    break;
                }
                if (globaltimer() - w0 > kWqWaitLimitNs) {
                    atomicOr(&q->status, kWqTimeout);
                    ex = 1;
                    break;
                }
                __nanosleep(ns);
                if (ns < 1024) ns *= 2;
            }
            if (!ex) s_item = __ldcg(&ring[c % cap]);
            s_exit = ex;
        }
        __syncthreads();
        if (s_exit) break;
        const int2 it = s_item;
        BatchSlot &B = slots[it.x];
        const int act = __ldcg(&B.action);
        __syncthreads();
        const bool last = run_action(B, act, it.y);
        if (last) {
            __shared__ int s_next;
            if (threadIdx.x == 0) {
                int nxt = decide_action(B);
                if (nxt != kActNone && globaltimer() >= s_deadline) nxt = kActNone;   // pause
                if (nxt != kActNone) {
                    B.action = nxt;
                    __threadfence();
                } else {
                    __threadfence();
                    atomicSub(&q->active, 1);
                }
                s_next = nxt;
            }
            __syncthreads();
            if (s_next != kActNone) wq_push(q, ring, seq, cap, it.x, action_tiles(B, s_next));
        }
        __syncthreads();
        // a chief-table copy of this block never landed: its shared memory may still be
        // written, so it claims nothing more, and the launch is marked so that the other
        // blocks stop at their next claim and the host fails every problem that did not
        // finish (as after a claim timeout)
        if (mixed_copy_lost()) {
            if (threadIdx.x == 0) atomicOr(&q->status, kWqCopyLost);
            break;
        }
    }
}


// ------------------------------------------------------------------ Levenberg-Marquardt
// Refinement of one candidate state (Eqs. 14-16), one block.  Residual vector: weighted
// angle residuals (form 0, 2K entries) or the per-epoch chi-squares b_k^T W b_k (form 1, K
// entries).  Per iteration: the centre's residuals and x +- h_j e_j (central-difference
// Jacobian, h_j = 1e-7 max(|x_j|, 0.1)) are propagated (threads 0-12, unless the previous
// iteration's speculative columns already hold them); threads 0-26 form J^T J and J^T r;
// threads 0-7 each solve (J^T J + lam_t diag(J^T J)) d = -J^T r (Cholesky) for lam_t =
// lam 10^(t-3) and propagate their trial; thread 0 keeps the lowest improving trial (lam =
// lam_t/10) or raises lam by 1e5, and stops on a relative decrease below 1e-10, lam > 1e16
// or max_iters.  R: global scratch of kLmVecs residual vectors and kLmTail doubles.
__device__ bool lm_residuals(const Dyn &D, const ObsView &O, const double x[6], int form,
                             double sig_ra, double sig_dec, double *r, double &cost)
{
    double s[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) s[d] = x[d];
    const double w_ra = 1.0 / (sig_ra * sig_ra), w_dec = 1.0 / (sig_dec * sig_dec);
    const double i_ra = 1.0 / sig_ra, i_dec = 1.0 / sig_dec;
    double c = 0.0;
    bool ok = true;
    propagate_rk4_any(D, s, O, [&](int k, const double *st) {
        // Eqs. 6-8 as the swarm's FP64 cost forms them: the azimuth from rho itself (the
        // two-argument arctangent does not depend on the common scale), its residual
        // reduced to [-pi, pi] (exactly b -/+ 2 pi for pi < |b| < 3 pi), the elevation
        // from rho_z / |rho|; every FP64 instruction costs a propagating lane alike, and
        // the unit vector's three divisions and the general remainder are not needed
        constexpr double kTwoPi = 6.283185307179586, kPi = 3.141592653589793;
        const double rx = st[0] - O.rcx[k], ry = st[1] - O.rcy[k], rz = st[2] - O.rcz[k];
        const double rr = sqrt(fma(rx, rx, fma(ry, ry, rz * rz)));
        double ba = O.ra[k] - atan2(ry, rx);
        if (!(fabs(ba) <= kPi)) ba = fabs(ba) < 3.0 * kPi ? ba - copysign(kTwoPi, ba) : remainder(ba, kTwoPi);
        const double bb = O.dec[k] - asin(rz / rr);
        if (form == 0) {
            const double a = ba * i_ra, b = bb * i_dec;
            r[2 * k] = a;
            r[2 * k + 1] = b;
            c = fma(a, a, c);
            c = fma(b, b, c);
        } else {
            const double f = fma(ba * w_ra, ba, bb * w_dec * bb);
            r[k] = f;
            c = fma(f, f, c);
        }
        ok = ok && isfinite(rr) && rr >= 1e-15;
    });
    cost = (ok && isfinite(c)) ? c : CUDART_INF;
    return ok;
}

__device__ bool chol_solve6(const double *A, const double *g, double lam, double *d)
{
    double L[36], y[6];
    for (int i = 0; i < 6; ++i) {
        for (int j = 0; j <= i; ++j) {
            double sum = (i == j) ? fma(lam, A[7 * i], A[7 * i]) : A[6 * i + j];
            for (int k = 0; k < j; ++k) sum -= L[6 * i + k] * L[6 * j + k];
            if (i == j) {
                if (!(sum > 0.0)) return false;
                L[7 * i] = sqrt(sum);
            } else {
                L[6 * i + j] = sum / L[7 * j];
            }
        }
    }
    for (int i = 0; i < 6; ++i) {
        double sum = -g[i];
        for (int k = 0; k < i; ++k) sum -= L[6 * i + k] * y[k];
        y[i] = sum / L[7 * i];
    }
    for (int i = 5; i >= 0; --i) {
        double sum = y[i];
        for (int k = i + 1; k < 6; ++k) sum -= L[6 * k + i] * d[k];
        d[i] = sum / L[7 * i];
    }
    return true;
}

// The refinement itself (block-collective: every thread of a block of at least 32 calls
// it; threads 0-26 work).  O: the observation table, staged and synchronised by the
// caller.  out[0..5] the refined state, out[6] its cost, out[7] iterations, out[8] the
// stop reason (0 iteration limit or damping bound, 1 converged, 2 start not evaluable).
// Levenberg-Marquardt state of one block: the estimate, its cost, the damping, the
// iterations taken and the stop reason (0 running or iteration limit, 1 converged, 2 start
// not evaluable), and where the Jacobian of the estimate stands: jac 0 = its columns are
// still to be propagated, 1 = its central-difference residual vectors are in the scratch
// (plus columns from vector col, minus columns from col + 6, the estimate's own residuals
// at vector ctr), 2 = J^T J (A) and J^T r (g) are formed.  tprev: the damping index of the
// last accepted trial (the first point the speculative columns are propagated about).
struct LmState {
    double x[6];
    double c, lam;
    int it, stop;
    int jac, col, ctr, tprev;
    double A[36], g[6];
};

// The start: the estimate x0 and its cost; damping 1e-3.
__device__ void lm_start(const Dyn &D, const ObsView &O, LmState &S, const double *x0, int form, double sig_ra,
                         double sig_dec, double *R)
{
    const int t = threadIdx.x;
    if (t < 6) S.x[t] = x0[t];
    __syncthreads();
    if (t == 0) {
        double c = 0.0;
        lm_residuals(D, O, S.x, form, sig_ra, sig_dec, R, c);
        S.c = c;
        S.lam = 1e-3;
        S.it = 0;
        S.stop = isfinite(c) ? 0 : 2;
        S.jac = 0;
        S.col = 1;
        S.ctr = 0;
        S.tprev = 3;
    }
    __syncthreads();
}

// Whether the iteration has ended: a stop reason, the iteration limit or a damping that
// no longer moves the estimate.
__device__ __forceinline__ bool lm_finished(const LmState &S, int max_iters)
{
    return S.stop != 0 || S.it >= max_iters || S.lam > 1e16;
}

// Finite-difference step of component j about x
__device__ __forceinline__ double lm_step(const double *x, int j)
{
    return 1e-7 * fmax(fabs(x[j]), 0.1);
}

// Iterations until the iteration has ended or `until` iterations have been taken in all
// (the state carries everything an iteration reads, so stopping and resuming between
// iterations gives the same result as one run).
//
// An FP64 instruction of a warp occupies its sub-partition's FP64 pipe for 64 cycles
// however few of its lanes are active, and a propagation is one lane's long chain of
// them, so the eight trials (threads 0-7) leave the other lanes idle at no gain.  Those
// lanes (threads 8 and up, twelve per point, up to eight points) propagate the
// central-difference columns about the trial points, in the order tprev, 0, 1, ..., in the
// same pass: when the accepted trial is one of them, the next iteration's Jacobian needs
// no propagation of its own (its columns and the estimate's residuals are those vectors).
// An iteration without improvement keeps the estimate, and with it A and g.  The values
// are those of the plain order (each column is the same propagation of the same state),
// so the result does not depend on the block size.
__device__ void lm_iterate(const Dyn &D, const ObsView &O, LmState &S, int max_iters, int until, int form,
                           double sig_ra, double sig_dec, double *R, int n_obs)
{
    const int n = form == 0 ? 2 * n_obs : n_obs;
    __shared__ double s_h[6], s_tc[8], s_tx[8][6];
    __shared__ int s_ok[8], s_pt[8];
    const int t = threadIdx.x;
    const int nspec = min(8, ((int)blockDim.x - 8) / 12);
    while (!lm_finished(S, max_iters) && S.it < until) {
        if (S.jac == 0) {   // the estimate's residuals and its twelve columns
            if (t < 6) s_h[t] = lm_step(S.x, t);
            __syncthreads();
            if (t < 13) {
                double xs[6];
#pragma unroll
                for (int d = 0; d < 6; ++d) xs[d] = S.x[d];
                if (t >= 1 && t <= 6) xs[t - 1] = S.x[t - 1] + s_h[t - 1];
                if (t >= 7) xs[t - 7] = S.x[t - 7] - s_h[t - 7];
                double c;
                lm_residuals(D, O, xs, form, sig_ra, sig_dec, R + (size_t)t * n, c);
            }
            __syncthreads();
            if (t == 0) {
                S.col = 1;
                S.ctr = 0;
                S.jac = 1;
            }
            __syncthreads();
        }
        if (S.jac == 1) {   // J^T J (21 entries) and J^T r (6)
            if (t < 6) s_h[t] = lm_step(S.x, t);
            __syncthreads();
            // the Jacobian's columns (r(x + h_a e_a) - r(x - h_a e_a)) / (2 h_a), every
            // element once, spread over the block (the residual vectors may have been
            // written by another block, a batch refinement resumed on another SM, and the
            // columns by other threads: both are read from L2)
            double *Jc = R + (size_t)kLmJac * n;
            for (int e = t; e < 6 * n; e += blockDim.x) {
                const int a = e / n, i = e - a * n;
                Jc[e] = (__ldcg(&R[(size_t)(S.col + a) * n + i]) - __ldcg(&R[(size_t)(S.col + 6 + a) * n + i])) /
                        (2.0 * s_h[a]);
            }
            __syncthreads();
            if (t < 27) {   // each entry one sequential sum over the residuals
                int a, b = -1;
                if (t < 21) {
                    int k = t;
                    a = 0;
                    while (k >= 6 - a) {
                        k -= 6 - a;
                        ++a;
                    }
                    b = a + k;
                } else {
                    a = t - 21;
                }
                const double *ja = Jc + (size_t)a * n;
                const double *jb = b >= 0 ? Jc + (size_t)b * n : R + (size_t)S.ctr * n;
                double sum = 0.0;
                for (int i = 0; i < n; ++i) sum = fma(__ldcg(&ja[i]), __ldcg(&jb[i]), sum);
                if (b >= 0) {
                    S.A[6 * a + b] = sum;
                    S.A[6 * b + a] = sum;
                } else {
                    S.g[a] = sum;
                }
            }
            __syncthreads();
            if (t == 0) S.jac = 2;
            __syncthreads();
        }
        if (t < 8) {    // eight damping values: the steps
            const double lt = S.lam * pow(10.0, (double)(t - 3));
            double d[6];
            s_ok[t] = chol_solve6(S.A, S.g, lt, d);
            if (s_ok[t]) {
#pragma unroll
                for (int q = 0; q < 6; ++q) s_tx[t][q] = S.x[q] + d[q];
            }
        }
        if (t == 0) {   // speculation order: the last accepted damping index, then 0, 1, ...
            s_pt[0] = S.tprev;
            for (int q = 0, k = 1; q < 8; ++q)
                if (q != S.tprev) s_pt[k++] = q;
        }
        __syncthreads();
        {   // the trials' residuals and costs; the columns about the first nspec points
            const double *xb = nullptr;
            double *out = nullptr;
            int pj = -1;
            double xs[6];
            if (t < 8) {
                if (s_ok[t]) {
                    xb = s_tx[t];
                    out = R + (size_t)(13 + t) * n;
                }
            } else {
                const int slot = t - 8, ps = slot / 12, cc = slot % 12;
                if (ps < nspec && s_ok[s_pt[ps]]) {
                    xb = s_tx[s_pt[ps]];
                    out = R + (size_t)(21 + 12 * ps + cc) * n;
                    pj = cc;
                }
            }
            double c = CUDART_INF;
            if (xb) {
#pragma unroll
                for (int d = 0; d < 6; ++d) xs[d] = xb[d];
                if (pj >= 0 && pj < 6) xs[pj] = xb[pj] + lm_step(xb, pj);
                if (pj >= 6) xs[pj - 6] = xb[pj - 6] - lm_step(xb, pj - 6);
                lm_residuals(D, O, xs, form, sig_ra, sig_dec, out, c);
            }
            if (t < 8) s_tc[t] = s_ok[t] ? c : CUDART_INF;
        }
        __syncthreads();
        if (t == 0) {
            int best = -1;
            double bc = S.c;
            for (int q = 0; q < 8; ++q)
                if (s_tc[q] < bc) {
                    bc = s_tc[q];
                    best = q;
                }
            ++S.it;
            if (best < 0) {
                S.lam = S.lam * 1e5;   // the estimate stays: so do A and g
            } else {
                const double dec = S.c - bc;
                for (int q = 0; q < 6; ++q) S.x[q] = s_tx[best][q];
                S.lam = S.lam * pow(10.0, (double)(best - 3)) / 10.0;
                const double c_old = S.c;
                S.c = bc;
                if (dec <= 1e-10 * c_old) S.stop = 1;
                S.tprev = best;
                S.jac = 0;
                for (int ps = 0; ps < nspec; ++ps)
                    if (s_pt[ps] == best) {   // its columns are ready
                        S.col = 21 + 12 * ps;
                        S.ctr = 13 + best;
                        S.jac = 1;
                    }
            }
        }
        __syncthreads();
    }
}

__device__ void lm_body(const KParams &P, const ObsView &O, const double *x0, int max_iters, int form,
                        double sig_ra, double sig_dec, double *R, double *out)
{
    const Dyn D = make_dyn(P);
    __shared__ LmState S;
    lm_start(D, O, S, x0, form, sig_ra, sig_dec, R);
    lm_iterate(D, O, S, max_iters, max_iters, form, sig_ra, sig_dec, R, P.n_obs);
    if (threadIdx.x == 0) {
        for (int q = 0; q < 6; ++q) out[q] = S.x[q];
        out[6] = S.c;
        out[7] = (double)S.it;
        out[8] = (double)S.stop;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(128) lm_kernel(KParams P, const double *__restrict__ x0, int max_iters,
                                                int form, double sig_ra, double sig_dec, double *R,
                                                double *out)
{
    extern __shared__ double sm[];
    const ObsView O = stage_obs(P, sm);
    __syncthreads();
    lm_body(P, O, x0, max_iters, form, sig_ra, sig_dec, R, out);
}

// A batch request's closing step: Levenberg-Marquardt from its global best (the form of
// its cost: CHI2 residuals or the per-epoch chi-squares of QUARTIC), kLmItersPerAction
// iterations per action.  The first action keeps the swarm's best (g_pso, gJ_pso) and
// takes the start; from then on g and gJ hold the current estimate and its cost (the
// estimate only ever moves to a lower cost, so it stays evaluable), with the damping,
// iteration count and stop reason beside them.  The last action sets kFlagRefined; a
// start that is not evaluable ends at once and keeps the swarm's best.  Returns true in
// every thread (the action's only tile).
__device__ bool refine_body(const KParams &P, int max_iters, double sig_ra, double sig_dec, double *R)
{
    extern __shared__ double sm[];
    const ObsView O = stage_obs(P, sm);
    const Dyn D = make_dyn(P);
    const int form = P.cost_form == 1 ? 1 : 0;
    GBest *gb = P.gb;
    __shared__ LmState S;
    __shared__ double s_x0[6];
    __shared__ int s_started;
    if (threadIdx.x == 0) s_started = (__ldcg(&gb->flags) & kFlagLmStarted) != 0;
    if (threadIdx.x < 6) s_x0[threadIdx.x] = __ldcg(&gb->g[threadIdx.x]);
    __syncthreads();
    if (!s_started) {
        lm_start(D, O, S, s_x0, form, sig_ra, sig_dec, R);
        if (threadIdx.x == 0) {
            for (int q = 0; q < 6; ++q) gb->g_pso[q] = s_x0[q];
            gb->gJ_pso = __ldcg(&gb->gJ);
        }
    } else {
        const int n = form == 0 ? 2 * P.n_obs : P.n_obs;
        const double *tail = R + (size_t)kLmVecs * n;
        if (threadIdx.x < 36) S.A[threadIdx.x] = __ldcg(&tail[threadIdx.x]);
        if (threadIdx.x < 6) S.g[threadIdx.x] = __ldcg(&tail[36 + threadIdx.x]);
        if (threadIdx.x == 0) {
            for (int q = 0; q < 6; ++q) S.x[q] = s_x0[q];
            S.c = __ldcg(&gb->gJ);
            S.lam = __ldcg(&gb->lm_lam);
            S.it = __ldcg(&gb->lm_iters);
            S.stop = __ldcg(&gb->lm_status);
            S.jac = (int)__ldcg(&tail[42]);
            S.col = (int)__ldcg(&tail[43]);
            S.ctr = (int)__ldcg(&tail[44]);
            S.tprev = (int)__ldcg(&tail[45]);
        }
    }
    __syncthreads();
    lm_iterate(D, O, S, max_iters, S.it + kLmItersPerAction, form, sig_ra, sig_dec, R, P.n_obs);
    {   // the carried part of the state, for the next action
        const int n = form == 0 ? 2 * P.n_obs : P.n_obs;
        double *tail = R + (size_t)kLmVecs * n;
        if (threadIdx.x < 36) tail[threadIdx.x] = S.A[threadIdx.x];
        if (threadIdx.x < 6) tail[36 + threadIdx.x] = S.g[threadIdx.x];
        if (threadIdx.x == 0) {
            tail[42] = (double)S.jac;
            tail[43] = (double)S.col;
            tail[44] = (double)S.ctr;
            tail[45] = (double)S.tprev;
        }
    }
    __syncthreads();   // the block's writes before thread 0's fence and flags
    if (threadIdx.x == 0) {
        if (S.stop != 2) {   // an evaluable start: the current estimate is the result so far
            for (int q = 0; q < 6; ++q) gb->g[q] = S.x[q];
            gb->gJ = S.c;
        }
        gb->lm_lam = S.lam;
        gb->lm_iters = S.it;
        gb->lm_status = S.stop;
        int fl = __ldcg(&gb->flags) | kFlagLmStarted;
        if (lm_finished(S, max_iters)) fl |= kFlagRefined;
        gb->flags = fl;
        __threadfence();
    }
    __syncthreads();
    return true;
}

int grid_for(int m, int block) { return (m + block - 1) / block; }

template <class K>
cudaError_t prepare(K kernel, size_t smem)
{
    if (smem > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaSuccess;
}

}  // namespace

size_t swarm_smem_bytes(int n_obs, int /*integrator*/)
{
    return (size_t)n_obs * (8 * sizeof(double) + sizeof(int));
}

int max_block_threads() { return kMaxThreads; }

cudaError_t launch_setup(const KParams &P, double vmax_frac, double sigma_ra, double sigma_dec,
                         double sigma_rng, const double *chief, double *rc_out, int *nsteps_out,
                         double *h_out, Consts *cst_out, GBest *gb, cudaStream_t st, double *chief_cs)
{
    setup_kernel<<<1, 32, 0, st>>>(P, vmax_frac, sigma_ra, sigma_dec, sigma_rng, chief, rc_out,
                                   nsteps_out, h_out, cst_out, gb, chief_cs);
    return cudaGetLastError();
}

size_t mixed_smem_bytes(int n_obs, long long total_steps)
{
    return mixed_smem_layout_bytes(n_obs, total_steps);
}

int mixed_chunk_steps() { return kChunk; }

cudaError_t launch_setup_mixed(const KParams &P, mix::Step *steps, const double *chief_cs,
                               mix::ObsDir *obsdir, float *chunk_time, cudaStream_t st)
{
    const long long work = P.total_steps > P.n_obs ? P.total_steps : P.n_obs;
    const int grid = (int)((work + 127) / 128 < 1024 ? (work + 127) / 128 : 1024);
    setup_mixed_kernel<<<grid, 128, 0, st>>>(P, steps, chief_cs, obsdir, chunk_time);
    return cudaGetLastError();
}

cudaError_t launch_init_mixed(const KParams &P, int block, cudaStream_t st)
{
    const size_t smem = mixed_smem_bytes(P.n_obs, P.total_steps);
    cudaError_t e;
    if ((e = prepare(init_mixed_kernel, smem)) != cudaSuccess) return e;
    init_mixed_kernel<<<grid_for(P.m, block), block, smem, st>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_iter_mixed(const KParams &P, int block, int gbest_order, cudaStream_t st)
{
    const size_t smem = mixed_smem_bytes(P.n_obs, P.total_steps);
    cudaError_t e;
    if (gbest_order) {
        if ((e = prepare(iter_mixed_kernel<1>, smem)) != cudaSuccess) return e;
        iter_mixed_kernel<1><<<grid_for(P.m, block), block, smem, st>>>(P);
    } else {
        if ((e = prepare(iter_mixed_kernel<0>, smem)) != cudaSuccess) return e;
        iter_mixed_kernel<0><<<grid_for(P.m, block), block, smem, st>>>(P);
    }
    return cudaGetLastError();
}

cudaError_t launch_rescore(const KParams &P, int block, cudaStream_t st)
{
    const size_t smem = swarm_smem_bytes(P.n_obs, 0);
    cudaError_t e;
    if ((e = prepare(rescore_kernel, smem)) != cudaSuccess) return e;
    rescore_kernel<<<grid_for(P.m, block), block, smem, st>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_eval_mixed(const KParams &P, const double *x, int m, double *J, int block,
                              cudaStream_t st)
{
    const size_t smem = mixed_smem_bytes(P.n_obs, P.total_steps);
    cudaError_t e;
    if ((e = prepare(eval_mixed_kernel, smem)) != cudaSuccess) return e;
    eval_mixed_kernel<<<grid_for(m, block), block, smem, st>>>(P, x, m, J, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_propagate_mixed(const KParams &P, const double *x0, int m, double *out,
                                   int block, cudaStream_t st)
{
    const size_t smem = mixed_smem_bytes(P.n_obs, P.total_steps);
    cudaError_t e;
    if ((e = prepare(eval_mixed_kernel, smem)) != cudaSuccess) return e;
    eval_mixed_kernel<<<grid_for(m, block), block, smem, st>>>(P, x0, m, nullptr, out);
    return cudaGetLastError();
}


cudaError_t launch_batch_setup(BatchSlot *slots, const int *ids, int n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    batch_setup_kernel<<<n, 128, 0, st>>>(slots, ids, n);
    return cudaGetLastError();
}

cudaError_t launch_batch_plan(BatchSlot *slots, int n_slots, cudaStream_t st)
{
    if (n_slots <= 0) return cudaSuccess;
    batch_plan_kernel<<<(n_slots + 127) / 128, 128, 0, st>>>(slots, n_slots);
    return cudaGetLastError();
}

cudaError_t launch_batch_round(BatchSlot *slots, const int2 *tiles, int n_tiles, BatchQueue *q,
                               int block, int grid, size_t smem, cudaStream_t st)
{
    if (n_tiles <= 0 || grid <= 0) return cudaSuccess;
    batch_round_kernel<<<grid, block, smem, st>>>(slots, tiles, n_tiles, q);
    return cudaGetLastError();
}

cudaError_t batch_round_prepare(size_t smem) { return prepare(batch_round_kernel, smem); }

int batch_round_occupancy(int block, size_t smem)
{
    int n = 0;
    prepare(batch_round_kernel, smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_round_kernel, block, smem);
    return n;
}


cudaError_t launch_wq_seed(BatchSlot *slots, int n_slots, WorkQueue *q, int2 *ring,
                           unsigned long long *seq, unsigned long long cap, cudaStream_t st)
{
    wq_seed_kernel<<<1, 256, 0, st>>>(slots, n_slots, q, ring, seq, cap);
    return cudaGetLastError();
}

cudaError_t launch_wq_run(BatchSlot *slots, WorkQueue *q, int2 *ring, unsigned long long *seq,
                          unsigned long long cap, unsigned long long budget_ns, int block, int grid,
                          size_t smem, int throughput, cudaStream_t st)
{
    const void *fn = throughput ? (const void *)wq_kernel<3> : (const void *)wq_kernel<2>;
    cudaError_t e = throughput ? prepare(wq_kernel<3>, smem) : prepare(wq_kernel<2>, smem);
    if (e != cudaSuccess) return e;
    void *args[] = {&slots, &q, &ring, &seq, &cap, &budget_ns};
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), args, smem, st);
}

int wq_occupancy(int block, size_t smem, int throughput)
{
    int n = 0;
    if (throughput) {
        prepare(wq_kernel<3>, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, wq_kernel<3>, block, smem);
    } else {
        prepare(wq_kernel<2>, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, wq_kernel<2>, block, smem);
    }
    return n;
}

// The global best of a shard replaced by the whole swarm's (the exchange between shards
// of one swarm): one thread, the values by value.
struct GbestArgs {
    double g[6];
    double gJ;
    int gidx;
};

__global__ void set_gbest_kernel(GBest *gb, GbestArgs a)
{
    if (threadIdx.x != 0) return;
#pragma unroll
    for (int d = 0; d < 6; ++d) gb->g[d] = a.g[d];
    gb->gJ = a.gJ;
    gb->gidx = a.gidx;
}

cudaError_t launch_set_gbest(GBest *gb, const double g[6], double gJ, int gidx, cudaStream_t st)
{
    GbestArgs a;
    for (int d = 0; d < 6; ++d) a.g[d] = g[d];
    a.gJ = gJ;
    a.gidx = gidx;
    set_gbest_kernel<<<1, 32, 0, st>>>(gb, a);
    return cudaGetLastError();
}

cudaError_t launch_lm(const KParams &P, const double *x0, int max_iters, int form, double sig_ra,
                      double sig_dec, double *R, double *out, cudaStream_t st)
{
    const size_t smem = swarm_smem_bytes(P.n_obs, 0);
    cudaError_t e = prepare(lm_kernel, smem);
    if (e != cudaSuccess) return e;
    lm_kernel<<<1, 128, smem, st>>>(P, x0, max_iters, form, sig_ra, sig_dec, R, out);
    return cudaGetLastError();
}

cudaError_t launch_init(const KParams &P, int block, cudaStream_t st)
{
    const size_t smem = swarm_smem_bytes(P.n_obs, P.integrator);
    cudaError_t e;
    if (P.pair && P.integrator == kDOPRI5) {
        if ((e = prepare(init_kernel_pair<kDOPRI5>, smem)) != cudaSuccess) return e;
        init_kernel_pair<kDOPRI5><<<grid_for(2 * P.m, block), block, smem, st>>>(P);
    } else if (P.pair) {
        if ((e = prepare(init_kernel_pair<kRK4>, smem)) != cudaSuccess) return e;
        init_kernel_pair<kRK4><<<grid_for(2 * P.m, block), block, smem, st>>>(P);
    } else if (P.integrator == kRK4 && P.dynamics) {
        if ((e = prepare(init_kernel_er, smem)) != cudaSuccess) return e;
        init_kernel_er<<<grid_for(P.m, block), block, smem, st>>>(P);
    } else if (P.integrator == kRK4) {
        if ((e = prepare(init_kernel<kRK4>, smem)) != cudaSuccess) return e;
        init_kernel<kRK4><<<grid_for(P.m, block), block, smem, st>>>(P);
    } else {
        if ((e = prepare(init_kernel<kDOPRI5>, smem)) != cudaSuccess) return e;
        init_kernel<kDOPRI5><<<grid_for(P.m, block), block, smem, st>>>(P);
    }
    return cudaGetLastError();
}

cudaError_t launch_iter(const KParams &P, int block, int gbest_order, cudaStream_t st)
{
    const size_t smem = swarm_smem_bytes(P.n_obs, P.integrator);
    const int grid = grid_for(P.m, block);
    cudaError_t e;
#define IOD_LAUNCH_ITER(I, L)                                                   \
    do {                                                                        \
        if ((e = prepare(iter_kernel<I, L>, smem)) != cudaSuccess) return e;    \
        iter_kernel<I, L><<<grid, block, smem, st>>>(P);                        \
    } while (0)
    if (P.pair) {
        const int g2 = grid_for(2 * P.m, block);
#define IOD_LAUNCH_PAIR(I, L)                                                        \
    do {                                                                             \
        if ((e = prepare(iter_kernel_pair<I, L>, smem)) != cudaSuccess) return e;    \
        iter_kernel_pair<I, L><<<g2, block, smem, st>>>(P);                          \
    } while (0)
        if (P.integrator == kDOPRI5) {
            if (gbest_order) IOD_LAUNCH_PAIR(kDOPRI5, 1); else IOD_LAUNCH_PAIR(kDOPRI5, 0);
        } else {
            if (gbest_order) IOD_LAUNCH_PAIR(kRK4, 1); else IOD_LAUNCH_PAIR(kRK4, 0);
        }
#undef IOD_LAUNCH_PAIR
    } else if (P.integrator == kRK4 && P.dynamics) {
        if (gbest_order) {
            if ((e = prepare(iter_kernel_er<1>, smem)) != cudaSuccess) return e;
            iter_kernel_er<1><<<grid, block, smem, st>>>(P);
        } else {
            if ((e = prepare(iter_kernel_er<0>, smem)) != cudaSuccess) return e;
            iter_kernel_er<0><<<grid, block, smem, st>>>(P);
        }
    } else if (P.integrator == kRK4) {
        if (gbest_order) IOD_LAUNCH_ITER(kRK4, 1); else IOD_LAUNCH_ITER(kRK4, 0);
    } else {
        if (gbest_order) IOD_LAUNCH_ITER(kDOPRI5, 1); else IOD_LAUNCH_ITER(kDOPRI5, 0);
    }
#undef IOD_LAUNCH_ITER
    return cudaGetLastError();
}

cudaError_t launch_wait_probe(const unsigned int *flag, unsigned int stamp, unsigned long long limit_ns,
                              int *timed_out, unsigned long long *waited_ns, cudaStream_t st)
{
    wait_probe_kernel<<<1, 32, 0, st>>>(flag, stamp, limit_ns, timed_out, waited_ns);
    return cudaGetLastError();
}

cudaError_t launch_fp64_issue_probe(int warps, int lanes, int n, long long *cycles, double *sink, cudaStream_t st)
{
    fp64_issue_probe_kernel<<<1, 32 * warps, 0, st>>>(lanes, n, cycles, sink);
    return cudaGetLastError();
}

cudaError_t launch_split_plan(const KParams &P, int nw, int gsize, cudaStream_t st)
{
    const size_t smem = P.integrator == kDOPRI5 ? sizeof(float) * (size_t)P.n_obs : 0;
    cudaError_t e = prepare(split_plan_kernel, smem);
    if (e != cudaSuccess) return e;
    split_plan_kernel<<<1, 256, smem, st>>>(P, nw, gsize);
    return cudaGetLastError();
}

cudaError_t launch_iter_mixed_balanced(const KParams &P, int gbest_order, int nsm, cudaStream_t st)
{
    size_t smem = mixed_smem_bytes(P.n_obs, P.total_steps);
    if (smem < 120 * 1024) smem = 120 * 1024;     // one block per SM
    const void *fn = gbest_order ? (const void *)iter_mixed_balanced<1> : (const void *)iter_mixed_balanced<0>;
    cudaError_t e = gbest_order ? prepare(iter_mixed_balanced<1>, smem) : prepare(iter_mixed_balanced<0>, smem);
    if (e != cudaSuccess) return e;
    KParams Pc = P;
    void *args[] = {&Pc};
    return cudaLaunchCooperativeKernel(fn, dim3(nsm), dim3(kMixedBalancedThreads), args, smem, st);
}

// Dynamic shared memory of the balanced kernel: the observation table, at least 120 KB so
// that no SM can hold two of its blocks (one block per SM, its warps spread evenly over
// the four sub-partitions).
size_t balanced_smem_bytes(int n_obs)
{
    const size_t need = swarm_smem_bytes(n_obs, kRK4);
    return need > 120 * 1024 ? need : 120 * 1024;
}

cudaError_t launch_iter_balanced(const KParams &P, int mode, int nsm, int wps, cudaStream_t st)
{
    const size_t smem = balanced_smem_bytes(P.n_obs);
    const void *fn;
    cudaError_t e;
#define IOD_BAL(M, E)                                           \
    do {                                                        \
        fn = (const void *)iter_kernel_balanced<M, E>;          \
        e = prepare(iter_kernel_balanced<M, E>, smem);          \
    } while (0)
#define IOD_BAL_DP(M)                                           \
    do {                                                        \
        fn = (const void *)iter_kernel_balanced_dp<M>;          \
        e = prepare(iter_kernel_balanced_dp<M>, smem);          \
    } while (0)
    if (P.integrator == kDOPRI5) {
        if (mode == 2) IOD_BAL_DP(2); else if (mode == 1) IOD_BAL_DP(1); else IOD_BAL_DP(0);
    } else if (P.dynamics) {
        if (mode == 2) IOD_BAL(2, 1); else if (mode == 1) IOD_BAL(1, 1); else IOD_BAL(0, 1);
    } else {
        if (mode == 2) IOD_BAL(2, 0); else if (mode == 1) IOD_BAL(1, 0); else IOD_BAL(0, 0);
    }
#undef IOD_BAL
#undef IOD_BAL_DP
    if (e != cudaSuccess) return e;
    KParams Pc = P;
    void *args[] = {&Pc};
    return cudaLaunchCooperativeKernel(fn, dim3(nsm), dim3(32 * wps), args, smem, st);
}

cudaError_t launch_eval(const KParams &P, const double *x, int m, double *J, int block,
                        cudaStream_t st)
{
    const size_t smem = swarm_smem_bytes(P.n_obs, P.integrator);
    cudaError_t e;
    if (P.integrator == kRK4) {
        if ((e = prepare(eval_kernel<kRK4>, smem)) != cudaSuccess) return e;
        eval_kernel<kRK4><<<grid_for(m, block), block, smem, st>>>(P, x, m, J);
    } else {
        if ((e = prepare(eval_kernel<kDOPRI5>, smem)) != cudaSuccess) return e;
        eval_kernel<kDOPRI5><<<grid_for(m, block), block, smem, st>>>(P, x, m, J);
    }
    return cudaGetLastError();
}

cudaError_t launch_propagate(const KParams &P, const double *x0, int m, double *out, int block,
                             cudaStream_t st)
{
    const size_t smem = swarm_smem_bytes(P.n_obs, P.integrator);
    cudaError_t e;
    if (P.integrator == kRK4) {
        if ((e = prepare(propagate_kernel<kRK4>, smem)) != cudaSuccess) return e;
        propagate_kernel<kRK4><<<grid_for(m, block), block, smem, st>>>(P, x0, m, out);
    } else {
        if ((e = prepare(propagate_kernel<kDOPRI5>, smem)) != cudaSuccess) return e;
        propagate_kernel<kDOPRI5><<<grid_for(m, block), block, smem, st>>>(P, x0, m, out);
    }
    return cudaGetLastError();
}

cudaError_t launch_simulate(double mu, double ecc, double f0, int er, const double *chief,
                            const double *deputy, int n, const double *t, double rtol, double atol,
                            double h0, const double *noise, double *angles, double *ranges,
                            double *chief_pos, int *status, cudaStream_t st)
{
    if (er) {
        simulate_kernel<1><<<1, 32, 0, st>>>(mu, ecc, f0, chief, deputy, n, t, rtol, atol, h0, noise,
                                             angles, ranges, chief_pos, status);
        return cudaGetLastError();
    }
    simulate_kernel<0><<<1, 32, 0, st>>>(mu, 0.0, 0.0, chief, deputy, n, t, rtol, atol, h0, noise,
                                         angles, ranges, chief_pos, status);
    return cudaGetLastError();
}

}  // namespace iod

// =================================================================================
// Allocation-free candidate scoring (iod_score_noalloc).
//
// A variant of the evaluation + global-argmin path for callers that cannot allocate
// device memory.  Its scratch -- the per-block winners and the last-block counter --
// lives in the file-scope array below instead of caller or library allocations.  Every
// GPU that loads this library holds the array (about 128 KB) until the process exits.
// =================================================================================
#include <cuda.h>

#include <cmath>
#include <mutex>

#include "iod.h"

namespace iod {
namespace {

constexpr int kNoAllocBlock = 64;          // threads per block (fixed)
constexpr int kNoAllocMaxBlocks = 2048;    // => at most 131,072 candidates per call
constexpr int kNoAllocMaxDevices = 64;

struct NoAllocScratch {
    unsigned int done_blocks;              // last-block counter; cleared before every call
    unsigned int pad[63];
    BlockBest blk[kNoAllocMaxBlocks];      // one winner per block
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// obs: [6][K] = t, alpha~, beta~, r_c x, y, z.  The RK4 interval table is rebuilt per
// block in shared memory by interval_rule, the set-up kernel's rule.
__global__ void __launch_bounds__(kNoAllocBlock)
score_noalloc_kernel(double mu, int K, const double *__restrict__ obs, double sig_ra,
                     double sig_dec, double dt, const double *__restrict__ X, int m,
                     double *__restrict__ Jout, double *__restrict__ best, NoAllocScratch *scr)
{
    extern __shared__ double sm[];
    double *ra = sm, *dec = sm + K, *rcx = sm + 2 * K, *rcy = sm + 3 * K, *rcz = sm + 4 * K,
           *t = sm + 5 * K, *h = sm + 6 * K;
    int *ns = reinterpret_cast<int *>(sm + 7 * K);
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        t[k] = obs[k];
        ra[k] = obs[K + k];
        dec[k] = obs[2 * K + k];
        rcx[k] = obs[3 * K + k];
        rcy[k] = obs[4 * K + k];
        rcz[k] = obs[5 * K + k];
        interval_rule(k ? obs[k - 1] : 0.0, obs[k], dt, ns[k], h[k]);
    }
    __syncthreads();
    const ObsView O{ra, dec, nullptr, rcx, rcy, rcz, t, h, ns, K};
    const Dyn D{mu, 1.0 - mu};
    CostW W;
    W.w_ra = 1.0 / (sig_ra * sig_ra);
    W.w_dec = 1.0 / (sig_dec * sig_dec);
    W.w_rng = 0.0;
    W.quartic = 0;
    W.use_range = 0;
    KParams P{};
    P.mu = mu;
    P.n_obs = K;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double x[6] = {0, 0, 0, 0, 0, 0};
    double J = CUDART_INF;
    if (i < m) {
#pragma unroll
        for (int d = 0; d < 6; ++d) x[d] = X[(size_t)d * m + i];
        long long steps = 0;
        J = evaluate<kRK4>(P, D, W, O, x, steps);
        Jout[i] = J;
    }
    // block winner
    __shared__ double s_wj[kNoAllocBlock / 32];
    __shared__ int s_wi[kNoAllocBlock / 32];
    __shared__ int s_best;
    __shared__ bool s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double bj = (i < m) ? J : CUDART_INF;
    int bi = (i < m) ? i : INT_MAX;
    warp_argmin(bj, bi);
    if (lane == 0) {
        s_wj[warp] = bj;
        s_wi[warp] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kNoAllocBlock / 32; ++w)
            if (better(s_wj[w], s_wi[w], bj, bi)) {
                bj = s_wj[w];
                bi = s_wi[w];
            }
        s_best = bi;
    }
    __syncthreads();
    if (i == s_best) {
        BlockBest &b = scr->blk[blockIdx.x];
        b.J = J;
        b.idx = i;
#pragma unroll
        for (int d = 0; d < 6; ++d) b.x[d] = x[d];
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(&scr->done_blocks, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // the last block folds every block's winner (lowest index wins ties)
    bj = CUDART_INF;
    bi = INT_MAX;
    int bs = -1;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        const double j = __ldcg(&scr->blk[b].J);
        const int ix = __ldcg(&scr->blk[b].idx);
        if (better(j, ix, bj, bi)) {
            bj = j;
            bi = ix;
            bs = b;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double oj = __shfl_xor_sync(0xffffffffu, bj, off);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
        const int os = __shfl_xor_sync(0xffffffffu, bs, off);
        if (better(oj, oi, bj, bi)) {
            bj = oj;
            bi = oi;
            bs = os;
        }
    }
    __shared__ int s_slot[kNoAllocBlock / 32];
    __syncthreads();
    if (lane == 0) {
        s_wj[warp] = bj;
        s_wi[warp] = bi;
        s_slot[warp] = bs;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kNoAllocBlock / 32; ++w)
            if (better(s_wj[w], s_wi[w], bj, bi)) {
                bj = s_wj[w];
                bi = s_wi[w];
                bs = s_slot[w];
            }
        best[0] = bj;
        best[1] = (double)bi;
#pragma unroll
        for (int d = 0; d < 6; ++d) best[2 + d] = __ldcg(&scr->blk[bs].x[d]);
        scr->done_blocks = 0u;
    }
}

// The scratch array's device address (and the kernel's shared-memory attribute) belong
// to one CUDA context: a cudaDeviceReset, or a new primary context, loads the module
// again, possibly elsewhere.  The cache is therefore keyed on the current context's
// unique id (cuCtxGetId, never reused within a process), reached through the runtime's
// driver entry-point query so that the library links no driver library.
struct NoAllocCache {
    void *ptr = nullptr;
    unsigned long long ctx_id = 0;
};
std::mutex g_noalloc_mu;
NoAllocCache g_noalloc_cache[kNoAllocMaxDevices];

// Unique id of the calling thread's current context; false if there is none or the
// driver does not provide the query (the caller then looks the address up every call).
bool current_context_id(unsigned long long &id)
{
    static CUresult (*get_current)(CUcontext *) = nullptr;
    static CUresult (*get_id)(CUcontext, unsigned long long *) = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void *f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CUresult (*)(CUcontext *)>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CUresult (*)(CUcontext, unsigned long long *)>(f);
    });
    if (!get_current || !get_id) return false;
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return get_id(ctx, &id) == CUDA_SUCCESS;
}

}  // namespace
}  // namespace iod

extern "C" int iod_score_noalloc(double mu, int n_obs, const double *obs, double sigma_ra,
                                 double sigma_dec, double dt, const double *x, int m, double *J,
                                 double *best, void *cuda_stream)
{
    using namespace iod;
    if (!obs || !x || !J || !best) return set_last_error(IOD_EINVAL, "NULL device pointer");
    if (!(mu > 0 && mu < 0.5)) return set_last_error(IOD_EINVAL, "mu must lie in (0, 0.5)");
    if (n_obs < 1) return set_last_error(IOD_EINVAL, "n_obs must be >= 1");
    if (m < 1 || m > kNoAllocBlock * kNoAllocMaxBlocks)
        return set_last_error(IOD_EINVAL, "m must lie in [1, 131072] for iod_score_noalloc");
    if (!(sigma_ra > 0) || !(sigma_dec > 0) || !std::isfinite(sigma_ra) || !std::isfinite(sigma_dec))
        return set_last_error(IOD_EINVAL, "sigma must be finite and > 0");
    if (!(dt > 0) || !std::isfinite(dt)) return set_last_error(IOD_EINVAL, "dt must be finite and > 0");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_last_error(IOD_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return set_last_error(IOD_EINVAL, "device ordinal out of range");
    const size_t smem = (size_t)n_obs * (7 * sizeof(double) + sizeof(int));
    int smax = 0;
    e = cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return set_last_error(IOD_ECUDA, cudaGetErrorString(e));
    if (smem + 1024 > (size_t)smax) return set_last_error(IOD_EINVAL, "n_obs too large for shared memory");
    void *scr = nullptr;
    {
        // once per device and context, with that device current: the scratch array's
        // device address
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        NoAllocCache &C = g_noalloc_cache[dev];
        unsigned long long id = 0;
        const bool known = current_context_id(id);
        if (!known || !C.ptr || C.ctx_id != id) {
            C.ptr = nullptr;
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess) return set_last_error(IOD_ECUDA, cudaGetErrorString(e));
            e = cudaFuncSetAttribute(score_noalloc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     smax - 1024);
            if (e != cudaSuccess) return set_last_error(IOD_ECUDA, cudaGetErrorString(e));
            // the look-up made the device's primary context current if none was
            if (current_context_id(id)) {
                C.ptr = ptr;
                C.ctx_id = id;
            }
            scr = ptr;
        } else {
            scr = C.ptr;
        }
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    NoAllocScratch *s = (NoAllocScratch *)scr;
    e = cudaMemsetAsync(&s->done_blocks, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return set_last_error(IOD_ECUDA, cudaGetErrorString(e));
    const int grid = (m + kNoAllocBlock - 1) / kNoAllocBlock;
    score_noalloc_kernel<<<grid, kNoAllocBlock, smem, st>>>(mu, n_obs, obs, sigma_ra, sigma_dec, dt,
                                                           x, m, J, best, s);
    e = cudaGetLastError();
    return e == cudaSuccess ? IOD_OK : set_last_error(IOD_ECUDA, cudaGetErrorString(e));
}
