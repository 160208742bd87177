"""Shared set-up for the GPU parity tests: one seeded scenario feeds the oracle and the
CUDA library the same inputs (observations come from the oracle's simulation), and
the tolerances the comparisons use.

Tolerances
  * states: 1e-12 relative (infinity norm over the 6-vector) at
    times up to 1 TU.
  * costs: 1e-10 relative, plus the part that FP64 rounding of the angles must leave:
    both sides round alpha and beta to within a few ulps of a number below pi, so a
    residual b carries |db| <= 4 * 2^-53 * pi and its weighted square w b^2 moves by up
    to 2 w |b| db + w db^2; summed over the epochs this is the absolute floor.  When
    the states being compared differ (GPU vs oracle propagation), the angle error of
    each epoch also carries |d rho| / |rho|, where d rho is the measured difference of
    the line of sight rho = r_deputy - r_chief: the deputy's state difference and the
    chief trajectory's (each side propagates its own chief), both a few ulps of |r|
    (~1e-16 LU) but divided by |rho|, which is ~1e-4 LU for deputies tens of km away.
"""
from __future__ import annotations

import math

import numpy as np

import oracle as O
from paper_2207_13175_gb300 import api
from paper_2207_13175_gb300 import inputs as I

STATE_RTOL = 1e-12
COST_RTOL = 1e-10
ANGLE_ULPS = 4.0 * 2.0 ** -53 * math.pi


class Pair:
    """A scenario instantiated on both sides with identical inputs."""

    def __init__(self, sc: I.Scenario, integrator="rk4", cost_form=0, gbest_order=0,
                 use_range=False, sigma_rng=None, block_size=0, obs=None, variant=None,
                 er3bp=None):
        self.sc = sc
        # er3bp = (eccentricity, true anomaly at t = 0): elliptic dynamics on both sides
        self.er3bp = er3bp
        er_kw = {} if er3bp is None else dict(ecc=er3bp[0], f0=er3bp[1])
        # swarm variants of the particle swarm section, the same keys on both sides:
        # tol_tau, tol_window (Algorithm 2), constriction (Eq. 4), init_grid
        self.variant = dict(variant or {})
        if obs is None:
            ra, dec, rng, _ = O.simulate_obs(sc.mu, sc.chief, sc.deputy, sc.t, sc.noise, **er_kw)
        else:
            ra, dec, rng = obs
        self.ra, self.dec, self.rng = ra, dec, rng
        integ = O.RK4 if integrator == "rk4" else O.DOPRI5
        self.sigma_rng = sigma_rng if sigma_rng is not None else 0.01 / I.L_KM
        self.ora = O.Problem(sc.mu, sc.chief, sc.t, ra, dec, *sc.sigma, integrator=integ,
                             dt=sc.dt, rtol=sc.rtol, atol=sc.atol, h0=sc.h0,
                             cost_form=cost_form, rng=rng, sigma_rng=self.sigma_rng,
                             use_range=use_range,
                             **({} if er3bp is None else dict(dynamics=O.ER3BP, **er_kw)))
        self.lo, self.hi = O.bounds_from_chief(sc.chief, sc.r_max_km, sc.v_max_ms, I.L_KM, I.TU_S)
        self.bounds = api.bounds_from_chief(sc.chief, sc.r_max_km, sc.v_max_ms, I.L_KM, I.TU_S)
        opts = api.options(integrator=integ, dt=sc.dt, rtol=sc.rtol, atol=sc.atol, h0=sc.h0,
                           cost_form=cost_form, gbest_order=gbest_order,
                           use_range=int(use_range), sigma_range=self.sigma_rng,
                           block_size=block_size,
                           **({} if er3bp is None else dict(dynamics=api.ER3BP, **er_kw)),
                           **{k: (int(v) if isinstance(v, bool) else v) for k, v in self.variant.items()})
        self.gpu = api.Problem(sc.mu, sc.chief, sc.t, np.stack([ra, dec], 1), sc.sigma,
                               self.bounds, opts, ranges=rng if use_range else None)
        self.gbest_order = gbest_order

    @property
    def d_chief(self) -> np.ndarray:
        """Per epoch, the bound |dr| <= sqrt(3) max_i |dr_i| on the difference between the
        GPU's and the oracle's chief positions r_c(t_k)."""
        if not hasattr(self, "_d_chief"):
            rc = self.gpu.chief_positions()
            self._d_chief = np.max(np.abs(rc - self.ora.rc), axis=1) * math.sqrt(3)
        return self._d_chief

    def pso(self, seed=None, w=None, c1=None, c2=None):
        sc = self.sc
        return O.Pso(self.ora, self.lo, self.hi, w=sc.w if w is None else w,
                     c1=sc.c1 if c1 is None else c1, c2=sc.c2 if c2 is None else c2,
                     seed=sc.seed if seed is None else seed, gbest_order=self.gbest_order,
                     **self.variant)

    def close(self):
        self.gpu.close()


def residuals(pair: Pair, states: np.ndarray):
    """Oracle residuals (b_ra, b_dec) and |rho|, |rho_xy| of one trajectory [K][6]."""
    K = states.shape[0]
    b = np.empty((K, 2))
    rho = np.empty(K)
    rxy = np.empty(K)
    for k in range(K):
        r = states[k, :3] - pair.ora.rc[k]
        a, be, rr = O.angles(r)
        b[k, 0] = math.remainder(pair.ra[k] - a, 2 * math.pi)
        b[k, 1] = pair.dec[k] - be
        rho[k] = rr
        rxy[k] = math.hypot(r[0], r[1])
    return b, rho, rxy


def cost_tolerance(pair: Pair, states: np.ndarray, J_ref: float, dstate=None) -> float:
    """Allowed |J_gpu - J_oracle| for one particle (see the module docstring)."""
    if not math.isfinite(J_ref):
        return 0.0
    sc = pair.sc
    w = np.array([1 / sc.sigma[0] ** 2, 1 / sc.sigma[1] ** 2])
    b, rho, rxy = residuals(pair, states)
    d = np.full((states.shape[0], 2), ANGLE_ULPS)
    if dstate is not None:
        dr = np.max(np.abs(dstate[:, :3]), axis=1) * math.sqrt(3) + pair.d_chief
        d[:, 0] += dr / np.maximum(rxy, 1e-300)
        d[:, 1] += dr / np.maximum(rho, 1e-300)
    per = (2 * np.abs(b) * d + d * d) @ w
    if pair.ora._s.cost_form == O.COST_QUARTIC:
        Jk = (b * b) @ w
        per = 2 * Jk * per + per * per
    return COST_RTOL * abs(J_ref) + float(per.sum())


def rel_state_err(a: np.ndarray, b: np.ndarray) -> float:
    """max over rows of ||a - b||_inf / ||b||_inf (rows are 6-vectors)."""
    a = np.asarray(a).reshape(-1, 6)
    b = np.asarray(b).reshape(-1, 6)
    return float(np.max(np.max(np.abs(a - b), axis=1) / np.max(np.abs(b), axis=1)))


def _min_rel_gap(a, b) -> float:
    """Smallest nonzero |a - b| / |b| over finite pairs (inf if none).  Exactly equal
    costs are left out: they come from identical positions, which both sides evaluate to
    identical costs and so decide identically (no strict improvement; lowest index)."""
    a = np.asarray(a, dtype=float)
    b = np.asarray(b, dtype=float)
    fin = np.isfinite(a) & np.isfinite(b) & (a != b) & (b != 0)
    if not fin.any():
        return np.inf
    return float(np.min(np.abs(a[fin] - b[fin]) / np.abs(b[fin])))


def _best_two_gap(J) -> float:
    """Relative gap between the lowest cost and the next distinct one."""
    u = np.unique(np.asarray(J)[np.isfinite(J)])
    if u.size < 2:
        return np.inf
    return _min_rel_gap(u[1:2], u[0:1])


def oracle_run_recorded(pair, m, iters, seed):
    """Oracle Algorithm 1 with the relative gap of every best-update decision and the
    global best position after every iteration."""
    import oracle
    Sx = pair.pso(seed=seed)
    W = oracle.Swarm(m)
    Sx.init(W)
    gJ, gi, gX, gap = [W.gJ], [W.gidx], [W.g], [_best_two_gap(W.J)]
    for n in range(1, iters + 1):
        pJ_prev, gJ_prev = W.pJ.copy(), W.gJ
        Sx.iterate(W, n)
        g_p = _min_rel_gap(W.J, pJ_prev)                 # personal-best decisions
        g_g = _best_two_gap(W.J)                         # this iteration's argmin
        g_u = _min_rel_gap([np.min(W.J)], [gJ_prev])     # global-best replacement
        gap.append(min(g_p, g_g, g_u))
        gJ.append(W.gJ)
        gi.append(W.gidx)
        gX.append(W.g)
    W.g_trace = np.array(gX)
    return W, np.array(gJ), np.array(gi), np.array(gap)


def trace_cost_tolerances(pair, gX) -> np.ndarray:
    """The per-particle cost tolerance of each traced global best (oracle position), with
    the GPU-vs-oracle state difference of that position's propagation."""
    uniq, inv = np.unique(np.asarray(gX), axis=0, return_inverse=True)
    gpu_states = pair.gpu.propagate(uniq).cpu().numpy()      # [K][6][u]
    tol_u = np.empty(uniq.shape[0])
    for j in range(uniq.shape[0]):
        ref, _, rc = pair.ora.propagate(uniq[j])
        J_ref = pair.ora.cost(uniq[j])
        tol_u[j] = cost_tolerance(pair, ref, J_ref, gpu_states[:, :, j] - ref) if rc == 0 else 0.0
    return tol_u[np.asarray(inv).reshape(-1)]


def assert_trace_parity(S, pair, r, W, gJ, gi, gap, tie=1e-12):
    """gbest index equal at every iteration until the first iteration with a decision
    gap below `tie` (relative; 1e-12 by default); the traced global-best costs
    within the per-particle cost tolerance (1e-10 relative plus the angle-rounding
    floor) while in step; afterwards the final position error is no worse than 1.1x the
    oracle's."""
    n_tie = np.argmax(np.minimum.accumulate(gap) < tie) if np.any(gap < tie) else len(gap)
    gig, gJg = r["gidx_trace"], r["gcost_trace"]
    assert len(gig) == len(gi)
    upto = n_tie if n_tie < len(gi) else len(gi)
    diverged = np.nonzero(gig[:upto] != gi[:upto])[0]
    assert diverged.size == 0, f"gbest index differs at iteration {diverged[0]} (first tie {n_tie})"
    if upto > 0:
        tol = trace_cost_tolerances(pair, W.g_trace[:upto])
        dif = np.abs(gJg[:upto] - gJ[:upto])
        bad = np.nonzero(~(dif <= tol) & ~(gJg[:upto] == gJ[:upto]))[0]
        assert bad.size == 0, (f"traced cost outside tolerance at iteration {bad[0]}: "
                               f"{gJg[bad[0]]!r} vs {gJ[bad[0]]!r}, tolerance {tol[bad[0]]!r}")
    truth = pair.sc.deputy
    err_g = np.linalg.norm(r["state"][:3] - truth[:3])
    err_o = np.linalg.norm(W.g[:3] - truth[:3])
    if upto == len(gi):
        assert np.array_equal(r["state"], W.g)
    assert err_g <= 1.1 * err_o + 1e-12, (err_g, err_o)
    return upto
