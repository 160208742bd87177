"""GPU parity of the swarm variants of the particle swarm section: Algorithm 2's
tolerance stop, the constriction factor of Eq. 4 and the stratified ("grid-like")
initialisation, alone and combined, single problems and batches, against the oracle
on the tiny workload."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ITERS = 60
CONSTRICTED = dict(w=1.0, c1=2.05, c2=2.05)


@pytest.fixture(scope="module")
def S():
    import scenarios
    return scenarios


@pytest.fixture(scope="module")
def I():
    from paper_2207_13175_gb300 import inputs
    return inputs


def tol_margin(gJ, tau, window, upto):
    """Smallest relative distance of Algorithm 2's statistic from tau over the
    iterations the run went through: the GPU's costs carry rounding differences of
    about 1e-13 relative, so the stop decision is only comparable away from tau."""
    worst = math.inf
    for n in range(window + 1, upto + 1):
        K = abs((gJ[n] - gJ[n - window]) / gJ[n])
        worst = min(worst, abs(K - tau) / tau)
    return worst


L_KM = 384400.0
CONE = dict(init_cone=True, cone_rho_min=5.0 / L_KM, cone_rho_max=150.0 / L_KM, cone_sigmas=3.0)

CASES = {
    "constriction": (dict(constriction=True), CONSTRICTED),
    "cone": (CONE, {}),
    "cone-grid": (dict(CONE, init_grid=True), {}),
    "grid": (dict(init_grid=True), {}),
    "tol": (dict(tol_tau=1e-3), {}),
    "tol-window3": (dict(tol_tau=1e-3, tol_window=3), {}),
    "all": (dict(tol_tau=1e-2, constriction=True, init_grid=True), CONSTRICTED),
    "velocity-init": (dict(velocity_init=1), {}),
    "per-dim-r": (dict(per_dim_random=True), {}),
    "vinit-perdim-cone": (dict(CONE, velocity_init=1, per_dim_random=True), {}),
}


@pytest.mark.parametrize("gbest_order", [0, 1])
@pytest.mark.parametrize("case", list(CASES))
def test_variant_trace_parity(S, I, case, gbest_order):
    import oracle as O
    variant, coef = CASES[case]
    sc = I.tiny(0).with_(**coef)
    pair = S.Pair(sc, gbest_order=gbest_order, variant=variant)
    # where Algorithm 2 stops the oracle's run decides how far to record it
    Wt, gJt, _ = pair.pso().run(sc.m, ITERS)
    stop = Wt.iters_done
    if "tol_tau" in variant:
        assert tol_margin(gJt, variant["tol_tau"], variant.get("tol_window", 10), stop) > 1e-6
    W, gJ, gi, gap = S.oracle_run_recorded(pair, sc.m, stop, sc.seed)
    assert np.array_equal(gJ, gJt)
    pair.gpu.run(sc.m, ITERS, sc.w, sc.c1, sc.c2, sc.seed)
    r = pair.gpu.result()
    assert r["iters_done"] == stop
    assert r["rk_steps"] == sc.m * (stop + 1) * 247
    S.assert_trace_parity(S, pair, r, W, gJ, gi, gap)
    if "tol_tau" in variant and stop < ITERS:
        # later launches did nothing: asking for more changes nothing either
        pair.gpu.continue_(5)
        r2 = pair.gpu.result()
        assert r2["iters_done"] == stop and np.array_equal(r2["state"], r["state"])
    pair.close()


def test_grid_initialisation_positions_bit_exact(S, I):
    """iod_run with no iterations leaves the initial swarm: stratified positions (and
    uniform initial velocities) equal the oracle's bit for bit and form a Latin
    hypercube of the box."""
    import oracle as O
    sc = I.tiny(1)
    for m in (1, 97, 1000):
        pair = S.Pair(sc, variant=dict(init_grid=True, velocity_init=1))
        Wo = O.Swarm(m)
        pair.pso(seed=21).init(Wo)
        pair.gpu.run(m, 0, sc.w, sc.c1, sc.c2, 21)
        sw = pair.gpu.swarm_get()
        assert np.array_equal(sw["x"], Wo.x.T) and np.array_equal(sw["v"], Wo.v.T)
        assert np.any(sw["v"] != 0)
        for d in range(6):
            s = np.floor((sw["x"][d] - pair.lo[d]) / (pair.hi[d] - pair.lo[d]) * m).astype(int)
            assert sorted(s.tolist()) == list(range(m))
        pair.close()


@pytest.mark.parametrize("grid", [False, True])
def test_cone_initialisation_positions_bit_exact(S, I, grid):
    """Line-of-sight initial positions equal the oracle's bit for bit (the frame of the
    first observation is formed on the host with the same libm on both sides, the rest
    in round-to-nearest steps in the oracle's order)."""
    import oracle as O
    sc = I.tiny(3)
    for m in (1, 257):
        pair = S.Pair(sc, variant=dict(CONE, init_grid=grid))
        Wo = O.Swarm(m)
        pair.pso(seed=5).init(Wo)
        pair.gpu.run(m, 0, sc.w, sc.c1, sc.c2, 5)
        sw = pair.gpu.swarm_get()
        assert np.array_equal(sw["x"], Wo.x.T)
        assert sw["gidx"] == Wo.gidx
        pair.close()


@pytest.mark.parametrize("variant", [dict(constriction=True), dict(constriction=True, per_dim_random=True)])
def test_constriction_lockstep_bit_exact(S, I, variant):
    """One constricted iteration from the oracle's swarm (optionally with per-dimension
    random numbers): positions and velocities bit for bit."""
    import oracle as O
    sc = I.tiny(2).with_(**CONSTRICTED)
    pair = S.Pair(sc, variant=variant)
    m = 150
    Sx = pair.pso(seed=7)
    W = O.Swarm(m)
    Sx.init(W)
    for n in range(1, 5):
        Sx.iterate(W, n)
    pair.gpu.swarm_set(W.x.T, W.v.T, W.p.T, W.pJ, W.g, W.gJ, W.gidx, 4, sc.w, sc.c1, sc.c2, 7)
    Sx.iterate(W, 5)
    pair.gpu.continue_(1)
    sw = pair.gpu.swarm_get()
    assert np.array_equal(sw["x"], W.x.T) and np.array_equal(sw["v"], W.v.T)
    pair.close()


def test_variant_options_rejected(S, I):
    from paper_2207_13175_gb300 import api
    sc = I.tiny(0)
    pair = S.Pair(sc, variant=dict(constriction=True))
    with pytest.raises(api.IodError):
        pair.gpu.run(64, 2, 0.7, 2.0, 2.0, 0)           # phi = 4: Eq. 4 needs phi > 4
    pair.close()
    for bad in (dict(tol_tau=1e-3, tol_window=0), dict(tol_tau=1e-3, tol_window=32),
                dict(tol_tau=-1.0), dict(constriction=2), dict(init_grid=-1),
                dict(CONE, cone_rho_max=0.0), dict(CONE, cone_sigmas=0.0), dict(velocity_init=2),
                dict(per_dim_random=3)):
        with pytest.raises(api.IodError):
            S.Pair(sc, variant=bad)
    with pytest.raises(api.IodError):           # the cone needs the first epoch at t = 0
        S.Pair(sc.with_(t=sc.t + 0.01), variant=CONE)


def test_tolerance_snapshot_restore(S, I):
    """Algorithm 2's record of past costs travels with a snapshot: a run stopped and
    restored mid-way ends where the uninterrupted run ends."""
    from paper_2207_13175_gb300 import api
    sc = I.tiny(0)
    pair = S.Pair(sc, variant=dict(tol_tau=1e-3))
    G = pair.gpu
    G.run(sc.m, ITERS, seed=sc.seed)
    full = G.result()
    assert full["iters_done"] < ITERS
    G.run(sc.m, 30, seed=sc.seed)
    blob = G.snapshot()
    opts = api.options(dt=sc.dt, tol_tau=1e-3)
    with api.Problem(sc.mu, sc.chief, sc.t, np.stack([pair.ra, pair.dec], 1), sc.sigma,
                     pair.bounds, opts) as G2:
        G2.restore(blob)
        G2.continue_(ITERS - 30)
        r = G2.result()
    assert r["iters_done"] == full["iters_done"]
    assert np.array_equal(r["state"], full["state"]) and r["cost"] == full["cost"]
    pair.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_variants_in_batches_equal_alone(precision):
    """Batches honour the variants: each problem ends where it ends alone, bit for bit
    (with IOD_MIXED a stopped problem still ends with the FP64 re-evaluation)."""
    from paper_2207_13175_gb300 import api
    from test_gpu_batch import alone, make_requests
    kw = dict(dt=1e-3, precision=precision, fp64_last_iters=3, tol_tau=5e-2, tol_window=3,
              constriction=1, init_grid=1, init_cone=1, cone_rho_min=5.0 / L_KM,
              cone_rho_max=250.0 / L_KM, velocity_init=1, per_dim_random=1)
    reqs = make_requests(10, seed=31 + precision)
    for r in reqs:
        r["iters"] = 40
    B = api.Batch(api.options(**kw), budget_bytes=1 << 30, max_resident=32)
    tickets = [B.submit(r["mu"], r["chief"], r["t"], r["angles"], r["sigma"], r["bounds"], r["m"],
                        r["iters"], seed=r["seed"], **CONSTRICTED) for r in reqs]
    B.run(0.0)
    stopped = 0
    for req, t in zip(reqs, tickets):
        got = B.poll(t, trace=True)
        with api.Problem(req["mu"], req["chief"], req["t"], req["angles"], req["sigma"],
                         req["bounds"], api.options(**kw)) as G:
            G.run(req["m"], req["iters"], seed=req["seed"], **CONSTRICTED)
            ref = G.result()
        assert got is not None
        assert got["iters_done"] == ref["iters_done"]
        stopped += ref["iters_done"] < req["iters"]
        assert np.array_equal(got["state"], ref["state"]) and got["cost"] == ref["cost"]
        assert np.array_equal(got["gcost_trace"], ref["gcost_trace"])
    assert stopped > 0
    B.close()


def test_mixed_precision_stop_still_rescored(S, I):
    """IOD_MIXED with Algorithm 2: the FP32 phase stops early, the personal bests are
    still re-evaluated in FP64, so the reported cost is the FP64 cost of the state."""
    from paper_2207_13175_gb300 import api
    sc = I.tiny(0)
    pair = S.Pair(sc)
    ra, dec = pair.ra, pair.dec
    pair.close()
    bounds = api.bounds_from_chief(sc.chief, sc.r_max_km, sc.v_max_ms, I.L_KM, I.TU_S)
    opts = api.options(dt=sc.dt, precision=api.MIXED, fp64_last_iters=10, tol_tau=1e-2)
    with api.Problem(sc.mu, sc.chief, sc.t, np.stack([ra, dec], 1), sc.sigma, bounds, opts) as G:
        G.run(sc.m, 200, sc.w, sc.c1, sc.c2, sc.seed)
        r = G.result()
        assert r["iters_done"] < 190
    with api.Problem(sc.mu, sc.chief, sc.t, np.stack([ra, dec], 1), sc.sigma, bounds,
                     api.options(dt=sc.dt)) as F:
        J = float(F.eval(r["state"][None, :]).cpu()[0])
    assert r["cost"] == pytest.approx(J, rel=1e-12)
