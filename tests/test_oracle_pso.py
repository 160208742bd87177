"""Pins of the oracle's swarm (Algorithm 1) and its counter-based generator: published
Philox known answers, convergence to known minima, and invariants the algorithm
implies (monotone bests, bounds, motion along the attractor directions)."""
import math

import numpy as np
import pytest


# Philox4x32-10 known-answer vectors (Salmon et al., SC'11, Random123 distribution)
@pytest.mark.parametrize("ctr,key,expect", [
    ([0, 0, 0, 0], [0, 0], [0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8]),
    ([0xffffffff] * 4, [0xffffffff] * 2, [0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd]),
    ([0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344], [0xa4093822, 0x299f31d0],
     [0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1]),
])
def test_philox_known_answers(O, ctr, key, expect):
    assert O.philox4x32_10(ctr, key).tolist() == expect


def test_u01_construction(O):
    assert O.u01(0, 0) == 0.0
    assert O.u01(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    assert O.u01(1 << 31, 0) == 0.5
    assert O.u01(0, 1 << 6) == 2.0 ** -53
    rng = np.random.default_rng(0)
    u = np.array([O.u01(int(a), int(b)) for a, b in rng.integers(0, 2 ** 32, size=(4000, 2))])
    assert abs(u.mean() - 0.5) < 0.02 and abs(u.var() - 1 / 12) < 0.01


SPHERE_LO = np.array([-1.0, -2.0, -0.5, -3.0, -1.0, -1.0])
SPHERE_HI = np.array([2.0, 1.0, 0.5, 1.0, 1.0, 4.0])
CENTER = np.array([0.3, -0.7, 0.1, -2.2, 0.6, 1.9])


def test_sphere_converges_below_brute_force_grid(O):
    """PSO on sum (x-c)^2 beats the best point of a 4^6 brute-force grid and lands on c."""
    axes = [np.linspace(SPHERE_LO[d], SPHERE_HI[d], 4) for d in range(6)]
    grid = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, 6)
    best_grid = min(O.cost_sphere(CENTER, g) for g in grid)
    W, gJ, gi = O.Pso(CENTER, SPHERE_LO, SPHERE_HI, seed=5).run(32, 300)
    assert gJ[-1] < best_grid
    assert gJ[-1] < 1e-12
    assert np.max(np.abs(W.g - CENTER)) < 1e-6


def test_minimum_on_the_box_face(O):
    c = CENTER.copy()
    c[2] = 5.0                                 # outside: optimum clamps to hi[2]
    W, gJ, _ = O.Pso(c, SPHERE_LO, SPHERE_HI, seed=0).run(32, 300)
    assert W.g[2] == SPHERE_HI[2]
    assert np.max(np.abs(np.delete(W.g - c, 2))) < 1e-6
    assert gJ[-1] == pytest.approx((c[2] - SPHERE_HI[2]) ** 2, rel=1e-12)
    assert np.all(W.x <= SPHERE_HI)


@pytest.mark.parametrize("order", [0, 1])
def test_monotone_bests_and_bounds(O, order):
    S = O.Pso(CENTER, SPHERE_LO, SPHERE_HI, seed=11, gbest_order=order)
    W = O.Swarm(24)
    S.init(W)
    prev_g, prev_p = W.gJ, W.pJ.copy()
    for n in range(1, 60):
        S.iterate(W, n)
        assert W.gJ <= prev_g
        assert np.all(W.pJ <= prev_p)
        assert np.all(W.x >= SPHERE_LO) and np.all(W.x <= SPHERE_HI)
        assert W.gJ == pytest.approx(O.cost_sphere(CENTER, W.g), rel=1e-15)
        assert W.gJ <= W.pJ.min() + 1e-300
        prev_g, prev_p = W.gJ, W.pJ.copy()


def test_initial_positions_uniform_in_box(O):
    S = O.Pso(CENTER, SPHERE_LO, SPHERE_HI, seed=3)
    W = O.Swarm(4096)
    S.init(W)
    width = SPHERE_HI - SPHERE_LO
    u = (W.x - SPHERE_LO) / width
    assert np.all(u >= 0) and np.all(u < 1)
    assert np.all(np.abs(u.mean(0) - 0.5) < 0.02)
    assert np.all(np.abs(u.var(0) - 1 / 12) < 0.01)
    assert np.all(W.v == 0) and np.array_equal(W.p, W.x)
    # the lowest-cost particle is the global best
    J = np.array([O.cost_sphere(CENTER, x) for x in W.x])
    assert W.gidx == int(np.argmin(J)) and np.array_equal(W.g, W.x[W.gidx])


def test_moves_follow_attractors(O):
    """w = 0, c1 = 0, c2 = 1: each move is x + r2 (g - x) with r2 in [0, 1): the new
    position lies on the segment from x to g.  w = c1 = c2 = 0: nothing moves."""
    S = O.Pso(CENTER, SPHERE_LO, SPHERE_HI, seed=7, w=0.0, c1=0.0, c2=1.0)
    W = O.Swarm(64)
    S.init(W)
    x0, g0 = W.x.copy(), W.g.copy()
    S.iterate(W, 1)
    for i in range(64):
        d = g0 - x0[i]
        step = W.x[i] - x0[i]
        if np.linalg.norm(d) == 0:
            assert np.all(step == 0)
            continue
        r = step @ d / (d @ d)
        assert -1e-15 <= r < 1.0
        assert np.allclose(step, r * d, atol=1e-14)
    S0 = O.Pso(CENTER, SPHERE_LO, SPHERE_HI, seed=7, w=0.0, c1=0.0, c2=0.0)
    W0 = O.Swarm(16)
    S0.init(W0)
    xs = W0.x.copy()
    for n in range(1, 5):
        S0.iterate(W0, n)
    assert np.array_equal(W0.x, xs)


def test_pure_inertia_keeps_constant_velocity(O):
    """With c1 = c2 = 0 and w = 1 a particle keeps its velocity until it hits the box."""
    S = O.Pso(CENTER, SPHERE_LO, SPHERE_HI, seed=2, w=1.0, c1=0.0, c2=0.0)
    W = O.Swarm(8)
    S.init(W)
    W.v[:] = 1e-3
    x0 = W.x.copy()
    for n in range(1, 4):
        S.iterate(W, n)
    inside = np.all(x0 + 3e-3 <= SPHERE_HI, axis=1)
    assert np.allclose(W.x[inside], x0[inside] + 3e-3, atol=1e-15)
    assert np.all(W.v[inside] == 1e-3)


def test_determinism_and_seed_dependence(O):
    a = O.Pso(CENTER, SPHERE_LO, SPHERE_HI, seed=9).run(16, 20)
    b = O.Pso(CENTER, SPHERE_LO, SPHERE_HI, seed=9).run(16, 20)
    c = O.Pso(CENTER, SPHERE_LO, SPHERE_HI, seed=10).run(16, 20)
    assert np.array_equal(a[0].x, b[0].x) and np.array_equal(a[1], b[1])
    assert not np.array_equal(a[0].x, c[0].x)


def test_lagged_order_first_iteration_reevaluates(O):
    """Algorithm 1 read literally evaluates the initial positions again in its first
    iteration, so that iteration cannot improve the global best."""
    W, gJ, gi = O.Pso(CENTER, SPHERE_LO, SPHERE_HI, seed=4, gbest_order=1).run(16, 30)
    assert gJ[1] == gJ[0] and gi[1] == gi[0]
    assert gJ[-1] < gJ[0]


def test_iod_tiny_noise_free_converges(O, I):
    """On the tiny workload without noise the swarm's best cost falls by orders of
    magnitude, and more particles/iterations reach a lower cost.  (Position error is not
    asserted: one day of angles-only data leaves the range direction weakly observable,
    so costs near zero still admit errors of order 10 km.)"""
    sc = I.tiny(0, noise=False)
    ra, dec, _, _ = O.simulate_obs(sc.mu, sc.chief, sc.deputy, sc.t, None)
    P = O.Problem(sc.mu, sc.chief, sc.t, ra, dec, *sc.sigma, dt=sc.dt)
    lo, hi = O.bounds_from_chief(sc.chief, sc.r_max_km, sc.v_max_ms, I.L_KM, I.TU_S)
    assert np.all(lo < sc.deputy) and np.all(sc.deputy < hi)
    S = O.Pso(P, lo, hi, seed=0)
    W, gJ, gi = S.run(64, 40)
    assert gJ[-1] < gJ[0] / 100
    W2, gJ2, _ = S.run(256, 100)
    assert gJ2[-1] < gJ[-1] / 1000
    assert W2.steps == 256 * 101 * 247


# ------------------------------------------------------------ variants of the swarm
def test_constriction_factor_closed_form(O):
    """Eq. 4.  Independently of the printed formula: 1/kappa is the larger root of
    z^2 - (phi - 2) z + 1 = 0, so kappa + 1/kappa = phi - 2 and kappa < 1 for phi > 4;
    phi = 4.1 gives Clerc and Kennedy's published 0.7298; kappa -> 1 as phi -> 4."""
    assert O.constriction(2.05, 2.05) == pytest.approx(0.729843788128, abs=1e-12)
    for c1, c2 in [(2.05, 2.05), (1.0, 3.5), (3.0, 3.0), (10.0, 0.5)]:
        k = O.constriction(c1, c2)
        assert 0 < k < 1
        assert k + 1 / k == pytest.approx(c1 + c2 - 2, rel=1e-14)
    assert O.constriction(2.0 + 1e-12, 2.0) == pytest.approx(1.0, abs=1e-5)
    assert O.constriction(50.0, 50.0) == pytest.approx(1 / 98, rel=1e-3)   # ~ 1/(phi-2)


def test_constriction_scales_the_whole_velocity_update(O):
    """From rest (v = 0, p = x after initialisation) one iteration gives
    v = c2 r2 (g - x); with the constriction factor every component, and only that,
    is multiplied by kappa (one rounding)."""
    kw = dict(w=0.9, c1=2.05, c2=2.1, seed=4)
    k = O.constriction(2.05, 2.1)
    Wa, Wb = O.Swarm(40), O.Swarm(40)
    Sa = O.Pso(CENTER, SPHERE_LO, SPHERE_HI, vmax_frac=10.0, **kw)
    Sb = O.Pso(CENTER, SPHERE_LO, SPHERE_HI, vmax_frac=10.0, constriction=True, **kw)
    Sa.init(Wa)
    Sb.init(Wb)
    assert np.array_equal(Wa.x, Wb.x)
    Sa.iterate(Wa, 1)
    Sb.iterate(Wb, 1)
    inside = (Wa.x > SPHERE_LO) & (Wa.x < SPHERE_HI) & (Wb.x > SPHERE_LO) & (Wb.x < SPHERE_HI)
    assert inside.mean() > 0.5
    assert np.array_equal(Wb.v[inside], k * Wa.v[inside])
    assert np.count_nonzero(Wa.v[inside]) > 0.5 * inside.sum()


def test_constriction_makes_an_undamped_swarm_converge(O):
    """w = 1, c1 = c2 = 2.05 does not settle without constriction (the box alone holds
    it); with kappa = 0.7298 the same swarm converges to the minimum."""
    for seed in range(3):
        _, gJ_free, _ = O.Pso(CENTER, SPHERE_LO, SPHERE_HI, w=1.0, c1=2.05, c2=2.05,
                              seed=seed).run(32, 300)
        W, gJ_k, _ = O.Pso(CENTER, SPHERE_LO, SPHERE_HI, w=1.0, c1=2.05, c2=2.05, seed=seed,
                           constriction=True).run(32, 300)
        assert gJ_free[-1] > 1e-4
        assert gJ_k[-1] < 1e-15
        assert np.max(np.abs(W.g - CENTER)) < 1e-7


def test_constriction_rejects_phi_at_most_four(O):
    with pytest.raises(RuntimeError):
        O.Pso(CENTER, SPHERE_LO, SPHERE_HI, c1=2.0, c2=2.0, constriction=True).run(8, 1)


@pytest.mark.parametrize("m", [1, 7, 64, 97, 1000])
def test_grid_initialisation_is_a_latin_hypercube(O, m):
    """Stratified initialisation: along every coordinate each of the m equal strata of
    the box holds exactly one particle, and the draw inside the stratum is the uniform
    initialisation's draw (so m = 1 reproduces it)."""
    Wg, Wu = O.Swarm(m), O.Swarm(m)
    O.Pso(CENTER, SPHERE_LO, SPHERE_HI, seed=3, init_grid=True).init(Wg)
    O.Pso(CENTER, SPHERE_LO, SPHERE_HI, seed=3).init(Wu)
    assert np.all(Wg.x >= SPHERE_LO) and np.all(Wg.x < SPHERE_HI)
    width = SPHERE_HI - SPHERE_LO
    for d in range(6):
        s = np.floor((Wg.x[:, d] - SPHERE_LO[d]) / width[d] * m).astype(int)
        assert sorted(s.tolist()) == list(range(m))
        u_grid = (Wg.x[:, d] - SPHERE_LO[d]) / width[d] * m - s
        u_unif = (Wu.x[:, d] - SPHERE_LO[d]) / width[d]
        assert np.allclose(u_grid, u_unif, atol=1e-9 * m)
    if m == 1:
        assert np.array_equal(Wg.x, Wu.x)
    assert np.all(Wg.v == 0) and np.array_equal(Wg.p, Wg.x)
    assert Wg.gidx == int(np.argmin(Wg.J))


def test_grid_initialisation_strata_differ_between_coordinates(O):
    """The six coordinates use different permutations (no particle sits on the box
    diagonal of strata)."""
    W = O.Swarm(256)
    O.Pso(CENTER, SPHERE_LO, SPHERE_HI, seed=9, init_grid=True).init(W)
    s = np.floor((W.x - SPHERE_LO) / (SPHERE_HI - SPHERE_LO) * 256).astype(int)
    for a in range(6):
        for b in range(a + 1, 6):
            assert np.count_nonzero(s[:, a] == s[:, b]) < 16


FACE_CENTER = np.array([0.3, -0.7, 0.1, -2.2, 5.0, 1.9])   # minimum on the face v = hi


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("tau", [1e-2, 1e-4, 1e-8, 1e-13])
def test_algorithm2_stops_at_the_first_window_hit(O, order, tau):
    """Algorithm 2 against the full run's trace: the stopped run is the same run cut at
    the first iteration n > 10 with |(J_n - J_{n-10})/J_n| < tau (the objective's
    minimum lies on a box face, so the global best plateaus at a positive cost)."""
    S_full = O.Pso(FACE_CENTER, SPHERE_LO, SPHERE_HI, seed=5, gbest_order=order)
    S_tol = O.Pso(FACE_CENTER, SPHERE_LO, SPHERE_HI, seed=5, gbest_order=order, tol_tau=tau)
    _, gJ, gi = S_full.run(32, 300)
    W, gJt, git = S_tol.run(32, 300)
    stop = 300
    for n in range(11, 301):
        if abs((gJ[n] - gJ[n - 10]) / gJ[n]) < tau:
            stop = n
            break
    assert W.iters_done == stop
    assert np.array_equal(gJt, gJ[:stop + 1]) and np.array_equal(git, gi[:stop + 1])
    if tau >= 1e-8:
        assert stop < 300


def test_algorithm2_window_is_a_parameter(O):
    _, gJ, _ = O.Pso(FACE_CENTER, SPHERE_LO, SPHERE_HI, seed=5).run(32, 300)
    W, _, _ = O.Pso(FACE_CENTER, SPHERE_LO, SPHERE_HI, seed=5, tol_tau=1e-4, tol_window=3).run(32, 300)
    n = W.iters_done
    assert n > 3 and abs((gJ[n] - gJ[n - 3]) / gJ[n]) < 1e-4
    assert all(abs((gJ[j] - gJ[j - 3]) / gJ[j]) >= 1e-4 for j in range(4, n))


def cone_problem(O, I, noise=False):
    sc = I.tiny(0, noise=noise)
    ra, dec, _, _ = O.simulate_obs(sc.mu, sc.chief, sc.deputy, sc.t, sc.noise)
    P = O.Problem(sc.mu, sc.chief, sc.t, ra, dec, *sc.sigma, dt=sc.dt)
    lo, hi = O.bounds_from_chief(sc.chief, 1000.0, sc.v_max_ms, I.L_KM, I.TU_S)
    return sc, P, ra, dec, lo, hi


@pytest.mark.parametrize("grid", [False, True])
def test_cone_initialisation_lies_on_the_first_line_of_sight(O, I, grid):
    """Every initial position is seen from the chief at t_0 within k sigma of the first
    observed angles, at a range inside [rho_min, rho_max]; velocities are the uniform
    initialisation's."""
    sc, P, ra, dec, lo, hi = cone_problem(O, I)
    rmin, rmax, k = 20.0 / I.L_KM, 150.0 / I.L_KM, 3.0
    S = O.Pso(P, lo, hi, seed=2, init_cone=True, cone_rho_min=rmin, cone_rho_max=rmax,
              cone_sigmas=k, init_grid=grid)
    Su = O.Pso(P, lo, hi, seed=2, init_grid=grid)
    W, Wu = O.Swarm(300), O.Swarm(300)
    S.init(W)
    Su.init(Wu)
    assert np.array_equal(W.x[:, 3:], Wu.x[:, 3:])
    rel = W.x[:, :3] - sc.chief[:3]
    rng = np.linalg.norm(rel, axis=1)
    assert np.all(rng >= rmin * (1 - 1e-12)) and np.all(rng <= rmax * (1 + 1e-12))
    for r in rel:
        a, b, _ = O.angles(r)
        da = math.remainder(a - ra[0], 2 * math.pi) * math.cos(dec[0])
        assert abs(da) <= k * sc.sigma[0] * (1 + 1e-6)
        assert abs(b - dec[0]) <= k * sc.sigma[1] * (1 + 1e-6)
    # the tilts fill the cone: both signs, out to most of its half-width
    a_off = np.array([math.remainder(O.angles(r)[0] - ra[0], 2 * math.pi) for r in rel])
    assert a_off.min() < -0.8 * k * sc.sigma[0]
    assert a_off.max() > 0.8 * k * sc.sigma[0]
    assert abs(np.mean(rng) - (rmin + rmax) / 2) < 0.1 * (rmax - rmin)


def test_cone_without_width_is_the_line_itself(O, I):
    """As k -> 0 the positions fall on the ray r_c(0) + rho u(alpha_0, beta_0)."""
    sc, P, ra, dec, lo, hi = cone_problem(O, I)
    S = O.Pso(P, lo, hi, seed=3, init_cone=True, cone_rho_min=1e-5, cone_rho_max=3e-4,
              cone_sigmas=1e-9)
    W = O.Swarm(64)
    S.init(W)
    u = np.array([math.cos(dec[0]) * math.cos(ra[0]), math.cos(dec[0]) * math.sin(ra[0]),
                  math.sin(dec[0])])
    rel = W.x[:, :3] - sc.chief[:3]
    perp = rel - np.outer(rel @ u, u)
    # positions are stored about |x| ~ 1, so the offset carries 2^-53 / |rel| of rounding
    assert np.max(np.linalg.norm(perp, axis=1) / np.linalg.norm(rel, axis=1)) < 1e-10
    assert np.all(rel @ u > 0)


def test_cone_contains_the_truth_direction(O, I):
    """Noise-free, the truth's first line of sight is the cone's axis: with the truth's
    range inside [rho_min, rho_max] the initial swarm has particles near the truth's
    position (distance below the range step of the swarm), far closer than uniform
    initialisation in the box puts any."""
    sc, P, ra, dec, lo, hi = cone_problem(O, I)
    rho_t = np.linalg.norm(sc.deputy[:3] - sc.chief[:3])
    Wc, Wu = O.Swarm(512), O.Swarm(512)
    O.Pso(P, lo, hi, seed=4, init_cone=True, cone_rho_min=0.5 * rho_t, cone_rho_max=1.5 * rho_t,
          cone_sigmas=3.0).init(Wc)
    O.Pso(P, lo, hi, seed=4).init(Wu)
    dc = np.min(np.linalg.norm(Wc.x[:, :3] - sc.deputy[:3], axis=1))
    du = np.min(np.linalg.norm(Wu.x[:, :3] - sc.deputy[:3], axis=1))
    assert dc < 0.01 * rho_t and dc < 0.1 * du


def test_cone_needs_the_first_epoch_at_zero(O, I):
    sc = I.tiny(0)
    t = sc.t + 0.01
    ra, dec, _, _ = O.simulate_obs(sc.mu, sc.chief, sc.deputy, t, sc.noise)
    P = O.Problem(sc.mu, sc.chief, t, ra, dec, *sc.sigma, dt=sc.dt)
    lo, hi = O.bounds_from_chief(sc.chief, 100.0, 1.0, I.L_KM, I.TU_S)
    with pytest.raises(RuntimeError):
        O.Pso(P, lo, hi, init_cone=True, cone_rho_min=0.0, cone_rho_max=1e-4).run(8, 0)


def test_uniform_velocity_initialisation(O):
    """velocity_init = 1: every initial velocity component lies within the velocity
    limits vmax_frac (hi - lo), both signs occur, the mean is near zero; positions are
    the zero-velocity initialisation's."""
    W0, W1 = O.Swarm(2000), O.Swarm(2000)
    O.Pso(CENTER, SPHERE_LO, SPHERE_HI, seed=6, vmax_frac=0.3).init(W0)
    O.Pso(CENTER, SPHERE_LO, SPHERE_HI, seed=6, vmax_frac=0.3, velocity_init=1).init(W1)
    assert np.array_equal(W0.x, W1.x) and np.all(W0.v == 0)
    vmax = 0.3 * (SPHERE_HI - SPHERE_LO)
    assert np.all(np.abs(W1.v) <= vmax)
    assert np.all(np.abs(W1.v.mean(axis=0)) < 0.05 * vmax)
    assert np.all(np.abs(W1.v.std(axis=0) - vmax / math.sqrt(3)) < 0.05 * vmax)


def test_per_dimension_random_numbers(O):
    """From rest after initialisation (v = 0, p = x) one iteration gives
    v_d = c2 r2 (g_d - x_d): with one pair per particle the ratio v_d/(g_d - x_d) is the
    same in every dimension, with one pair per dimension it differs, and dimension 0
    keeps the shared pair."""
    kw = dict(w=0.7, c1=1.5, c2=1.5, seed=8, vmax_frac=10.0)
    Wa, Wb = O.Swarm(50), O.Swarm(50)
    Sa = O.Pso(CENTER, SPHERE_LO, SPHERE_HI, **kw)
    Sb = O.Pso(CENTER, SPHERE_LO, SPHERE_HI, per_dim_random=True, **kw)
    Sa.init(Wa)
    Sb.init(Wb)
    g = Wa.g.copy()
    Sa.iterate(Wa, 1)
    Sb.iterate(Wb, 1)
    for i in range(50):
        x0 = Wa.x[i] - Wa.v[i]
        ok = np.abs(g - x0) > 1e-3
        ok &= (Wa.x[i] > SPHERE_LO) & (Wa.x[i] < SPHERE_HI) & (Wb.x[i] > SPHERE_LO) & (Wb.x[i] < SPHERE_HI)
        if ok.sum() < 3 or not ok[0]:
            continue
        ra = Wa.v[i][ok] / (g - x0)[ok]
        rb = Wb.v[i][ok] / (g - x0)[ok]
        assert np.allclose(ra, ra[0], rtol=1e-9) and np.all((ra >= 0) & (ra < 1.5))
        assert np.all((rb >= 0) & (rb < 1.5)) and np.ptp(rb) > 1e-3
        assert rb[0] == pytest.approx(ra[0], rel=1e-12)


def test_bounds_from_chief_hand_values(O):
    """The box about the chief (abstract; "Deputy Chief Scenario"): r_max km becomes
    r_max / L LU on each position axis and v_max m/s becomes (v_max / 1000) TU / L VU on
    each velocity axis.  Expected values are exact rationals rounded once, so a km<->LU
    or m/s<->VU slip (a missing /1000, TU and L swapped, an axis left out) fails."""
    from fractions import Fraction as F
    L, TU = 384400, 375190
    dr = float(F(100, L))                       # 100 km
    dv = float(F(1, 1000) * F(TU, L))           # 1 m/s
    assert abs(dr - 2.6014568158168574e-04) <= 1e-19
    assert abs(dv - 9.760405827263267e-04) <= 1e-18
    lo, hi = O.bounds_from_chief(np.zeros(6), 100.0, 1.0, float(L), float(TU))
    np.testing.assert_allclose(hi, [dr, dr, dr, dv, dv, dv], rtol=2 ** -52, atol=0)
    np.testing.assert_allclose(lo, -hi, rtol=0, atol=0)
    # one LU of radius and one VU of speed: exactly a unit box
    lo, hi = O.bounds_from_chief(np.zeros(6), float(L), 1000.0 * L / TU, float(L), float(TU))
    np.testing.assert_allclose(hi, np.ones(6), rtol=4 * 2 ** -52, atol=0)
    # centred on the chief, axis by axis
    chief = np.array([0.85, -0.01, 0.17, 0.02, 0.26, -0.03])
    lo, hi = O.bounds_from_chief(chief, 250.0, 100.0, float(L), float(TU))
    half = np.array([float(F(250, L))] * 3 + [float(F(100, 1000) * F(TU, L))] * 3)
    np.testing.assert_allclose(hi - chief, half, rtol=1e-12, atol=0)
    np.testing.assert_allclose(chief - lo, half, rtol=1e-12, atol=0)
