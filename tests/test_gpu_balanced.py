"""The balanced FP64 iteration (one resident warp per FP64 sub-partition, groups of 32
particles cut at epoch boundaries and handed from one warp to the next) reproduces the
grid-scheduled swarm bit for bit: traces, final states, swarm arrays and step counts, for
ragged swarm sizes, both global-best orders, the swarm variants, the mixed form's FP64
iterations and a snapshot taken between launches; and it agrees with the oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

L_KM = 384400.0


def warps():
    import torch
    return 4 * torch.cuda.get_device_properties(0).multi_processor_count


def run_both(sc, bounds, ang, m, iters, seed=9, coef=None, **kw):
    """Runs the same swarm with schedule GRID and BALANCED; returns both (result, swarm)."""
    from paper_2207_13175_gb300 import api
    coef = coef or dict(w=sc.w, c1=sc.c1, c2=sc.c2)
    out = []
    for sched in (api.SCHED_GRID, api.SCHED_BALANCED):
        opts = api.options(dt=sc.dt, schedule=sched, **kw)
        with api.Problem(sc.mu, sc.chief, sc.t, ang, sc.sigma, bounds, opts) as G:
            G.run(m, iters, seed=seed, **coef)
            r = G.result()
            assert r["schedule"] == sched      # the requested form is the one that ran
            out.append((r, G.swarm_get()))
    return out


def assert_same(a, b):
    (r1, w1), (r2, w2) = a, b
    assert r1["iters_done"] == r2["iters_done"]
    assert np.array_equal(r1["state"], r2["state"]) and r1["cost"] == r2["cost"]
    assert r1["gbest_index"] == r2["gbest_index"]
    assert np.array_equal(r1["gcost_trace"], r2["gcost_trace"])
    assert np.array_equal(r1["gidx_trace"], r2["gidx_trace"])
    assert r1["rk_steps"] == r2["rk_steps"] and r1["fp64_steps"] == r2["fp64_steps"]
    for k in ("x", "v", "p", "pJ", "J"):
        assert np.array_equal(w1[k], w2[k]), k


@pytest.mark.parametrize("gbest_order", [0, 1])
@pytest.mark.parametrize("per_warp,extra", [(1, 0), (1, 5), (1, 32 * 37 + 11), (2, 0), (2, 77),
                                            (3, 0), (3, 32 * 150 + 3)])
def test_balanced_equals_grid(gbest_order, per_warp, extra):
    """Swarms of exactly one, two or three groups per sub-partition (every cut at a group
    boundary; one, two or three warps per sub-partition), and ragged sizes with cuts
    inside groups."""
    import scenarios as S
    from paper_2207_13175_gb300 import inputs as I
    sc = I.tiny(1)
    pair = S.Pair(sc)
    ang = np.stack([pair.ra, pair.dec], 1)
    m = 32 * warps() * per_warp + extra
    a, b = run_both(sc, pair.bounds, ang, m, 4, gbest_order=gbest_order)
    assert_same(a, b)
    pair.close()


@pytest.mark.parametrize("variant", [
    dict(tol_tau=0.3, tol_window=2),
    dict(constriction=1, init_grid=1, velocity_init=1, per_dim_random=1),
    dict(init_cone=1, cone_rho_min=5.0 / L_KM, cone_rho_max=150.0 / L_KM, use_range=1,
         sigma_range=0.01 / L_KM),
    dict(cost_form=1),
])
def test_balanced_equals_grid_with_variants(variant):
    """The balanced kernel shares the move, cost and Algorithm 2 code with the grid form."""
    import scenarios as S
    from paper_2207_13175_gb300 import inputs as I
    sc = I.tiny(2)
    use_range = bool(variant.get("use_range", 0))
    pair = S.Pair(sc, use_range=use_range)
    ang = np.stack([pair.ra, pair.dec], 1)
    coef = dict(w=1.0, c1=2.05, c2=2.05) if variant.get("constriction") else None
    kw = dict(variant)
    m = 32 * warps() + 300
    out = []
    from paper_2207_13175_gb300 import api
    for sched in (api.SCHED_GRID, api.SCHED_BALANCED):
        opts = api.options(dt=sc.dt, schedule=sched, **kw)
        with api.Problem(sc.mu, sc.chief, sc.t, ang, sc.sigma, pair.bounds, opts,
                         ranges=pair.rng if use_range else None) as G:
            G.run(m, 40, seed=4, **(coef or dict(w=sc.w, c1=sc.c1, c2=sc.c2)))
            r = G.result()
            assert r["schedule"] == sched
            out.append((r, G.swarm_get()))
    assert_same(*out)
    if "tol_tau" in variant:
        assert out[0][0]["iters_done"] < 40
    pair.close()


@pytest.mark.parametrize("gbest_order", [0, 1])
def test_balanced_er3bp_equals_grid(gbest_order):
    """The elliptic problem's RK4 iterations run balanced too (the stage cosines restart
    at every interval, so a cut at an epoch boundary changes nothing)."""
    import scenarios as S
    from paper_2207_13175_gb300 import api
    from paper_2207_13175_gb300 import inputs as I
    sc = I.tiny(2)
    er = (0.0549, 0.4)
    pair = S.Pair(sc, er3bp=er)
    ang = np.stack([pair.ra, pair.dec], 1)
    a, b = run_both(sc, pair.bounds, ang, 32 * warps() * 3 + 1000, 4, gbest_order=gbest_order,
                    dynamics=api.ER3BP, ecc=er[0], f0=er[1])
    assert_same(a, b)
    pair.close()


def test_balanced_mixed_fp64_iterations_equal_grid():
    """IOD_MIXED's closing FP64 iterations run balanced too, with identical results."""
    import scenarios as S
    from paper_2207_13175_gb300 import api
    from paper_2207_13175_gb300 import inputs as I
    sc = I.tiny(3)
    pair = S.Pair(sc)
    ang = np.stack([pair.ra, pair.dec], 1)
    a, b = run_both(sc, pair.bounds, ang, 32 * warps() + 77, 10, precision=api.MIXED,
                    fp64_last_iters=4)
    assert_same(a, b)
    pair.close()


def sms():
    import torch
    return torch.cuda.get_device_properties(0).multi_processor_count


@pytest.mark.parametrize("gbest_order", [0, 1])
@pytest.mark.parametrize("fp64_last", [0, 3])
def test_balanced_mixed_fp32_iterations_equal_grid(gbest_order, fp64_last):
    """IOD_MIXED's FP32 iterations balanced over 384-particle super-groups (a block's
    warps share the staged chief table): identical to the grid form, ragged size."""
    import scenarios as S
    from paper_2207_13175_gb300 import api
    from paper_2207_13175_gb300 import inputs as I
    sc = I.tiny(4)
    pair = S.Pair(sc)
    ang = np.stack([pair.ra, pair.dec], 1)
    m = 384 * sms() + 32 * 50 + 9
    a, b = run_both(sc, pair.bounds, ang, m, 5, gbest_order=gbest_order, precision=api.MIXED,
                    fp64_last_iters=fp64_last)
    assert_same(a, b)
    pair.close()


def test_balanced_mixed_near_moon_equals_grid():
    """The paper's scenario-1 chief (close lunar passage: FP64 steps near the Moon, cuts
    that start mid-chunk) at the full 65,536 particles: FP32 iterations identical."""
    from paper_2207_13175_gb300 import api
    from paper_2207_13175_gb300 import inputs as I
    sc = I.paper_scale("paper-s1", 0)
    ang, _ = api.simulate_obs(sc.mu, sc.chief, sc.deputy, sc.t, sc.noise)
    bounds = api.bounds_from_chief(sc.chief, sc.r_max_km, sc.v_max_ms, I.L_KM, I.TU_S)
    out = []
    for sched in (api.SCHED_GRID, api.SCHED_AUTO):
        with api.Problem(sc.mu, sc.chief, sc.t, ang, sc.sigma, bounds,
                         api.options(dt=sc.dt, precision=api.MIXED, fp64_last_iters=0,
                                     schedule=sched)) as G:
            G.run(sc.m, 3, sc.w, sc.c1, sc.c2, 0)
            out.append((G.result(), G.swarm_get()))
    assert out[1][0]["schedule"] == api.SCHED_BALANCED       # chosen automatically here
    assert out[0][0]["fp64_steps"] > 0
    assert_same(*out)


def test_balanced_against_oracle():
    """Trace parity with the oracle (the grid form's parity bar) for a balanced run."""
    import scenarios as S
    from paper_2207_13175_gb300 import api
    from paper_2207_13175_gb300 import inputs as I
    sc = I.tiny(0)
    pair = S.Pair(sc)
    m = 32 * warps() + 19
    iters = 3
    W, gJ, gi, gap = S.oracle_run_recorded(pair, m, iters, sc.seed)
    ang = np.stack([pair.ra, pair.dec], 1)
    opts = api.options(dt=sc.dt, schedule=api.SCHED_BALANCED)
    with api.Problem(sc.mu, sc.chief, sc.t, ang, sc.sigma, pair.bounds, opts) as G:
        G.run(m, iters, sc.w, sc.c1, sc.c2, sc.seed)
        r = G.result()
    assert r["rk_steps"] == m * (iters + 1) * 247
    S.assert_trace_parity(S, pair, r, W, gJ, gi, gap)
    pair.close()


def test_balanced_snapshot_between_launches():
    """A run stopped, snapshotted and continued (in the same problem and in a new one)
    ends where the uninterrupted run ends: the hand-off flags never match a stale launch."""
    import scenarios as S
    from paper_2207_13175_gb300 import api
    from paper_2207_13175_gb300 import inputs as I
    sc = I.tiny(1)
    pair = S.Pair(sc)
    ang = np.stack([pair.ra, pair.dec], 1)
    m = 32 * warps() + 200
    opts = api.options(dt=sc.dt, schedule=api.SCHED_BALANCED)
    with api.Problem(sc.mu, sc.chief, sc.t, ang, sc.sigma, pair.bounds, opts) as G:
        G.run(m, 10, sc.w, sc.c1, sc.c2, 3)
        full = G.result()
        G.run(m, 4, sc.w, sc.c1, sc.c2, 3)
        blob = G.snapshot()
        G.continue_(6)
        again = G.result()
        G.restore(blob)
        G.continue_(6)
        same = G.result()
    with api.Problem(sc.mu, sc.chief, sc.t, ang, sc.sigma, pair.bounds, opts) as G2:
        G2.restore(blob)
        G2.continue_(6)
        other = G2.result()
    for r in (again, same, other):
        assert np.array_equal(r["state"], full["state"]) and r["cost"] == full["cost"]
        assert np.array_equal(r["gcost_trace"], full["gcost_trace"])
    pair.close()


def test_balanced_paper_scale_first_iterations():
    """The paper-scale workload (65,536 particles, 200 epochs): the automatic schedule
    (balanced there) and the grid form agree bit for bit over two iterations."""
    from paper_2207_13175_gb300 import api
    from paper_2207_13175_gb300 import inputs as I
    sc = I.paper_scale("halo", 0)
    ang, _ = api.simulate_obs(sc.mu, sc.chief, sc.deputy, sc.t, sc.noise)
    bounds = api.bounds_from_chief(sc.chief, sc.r_max_km, sc.v_max_ms, I.L_KM, I.TU_S)
    out = []
    for sched in (api.SCHED_GRID, api.SCHED_AUTO):
        with api.Problem(sc.mu, sc.chief, sc.t, ang, sc.sigma, bounds,
                         api.options(dt=sc.dt, schedule=sched)) as G:
            G.run(sc.m, 2, sc.w, sc.c1, sc.c2, 0)
            out.append((G.result(), G.swarm_get()))
    assert out[1][0]["schedule"] == api.SCHED_BALANCED     # chosen automatically here
    assert_same(*out)


def test_small_swarms_keep_the_grid_form():
    """Fewer 32-particle groups than FP64 sub-partitions: the grid form runs even when the
    balanced form is asked for (and automatically)."""
    from paper_2207_13175_gb300 import api
    from paper_2207_13175_gb300 import inputs as I
    sc = I.tiny(0)
    b = api.bounds_from_chief(sc.chief, 100.0, 1.0, I.L_KM, I.TU_S)
    for sched in (api.SCHED_AUTO, api.SCHED_BALANCED):
        with api.Problem(sc.mu, sc.chief, sc.t, np.zeros((sc.n_obs, 2)), sc.sigma, b,
                         api.options(dt=sc.dt, schedule=sched)) as G:
            G.run(32 * (warps() - 1), 1)
            assert G.result()["schedule"] == api.SCHED_GRID


def test_schedule_option_validated():
    from paper_2207_13175_gb300 import api
    from paper_2207_13175_gb300 import inputs as I
    sc = I.tiny(0)
    b = api.bounds_from_chief(sc.chief, 100.0, 1.0, I.L_KM, I.TU_S)
    for bad in (dict(schedule=3), dict(schedule=-1)):
        with pytest.raises(api.IodError):
            api.Problem(sc.mu, sc.chief, sc.t, np.zeros((sc.n_obs, 2)), sc.sigma, b, api.options(**bad))


@pytest.mark.parametrize("gbest_order", [0, 1])
@pytest.mark.parametrize("per_warp,extra", [(1, 0), (1, 32 * 37 + 11), (2, 0), (2, 77), (3, 32 * 150 + 3)])
def test_balanced_dopri5_equals_grid(gbest_order, per_warp, extra):
    """DOPRI5 (rtol = atol = 1e-12) under the balanced schedule: every particle resumes the
    uncut sequence of attempts from the handed-over integrator state, so traces, final
    states, swarm arrays and attempt counts equal the grid form's bit for bit (one and two
    warps per sub-partition, ragged sizes, both global-best orders)."""
    import scenarios as S
    from paper_2207_13175_gb300 import api
    from paper_2207_13175_gb300 import inputs as I
    sc = I.tiny(2).with_(integrator="dopri5")
    pair = S.Pair(sc, integrator="dopri5")
    ang = np.stack([pair.ra, pair.dec], 1)
    m = 32 * warps() * per_warp + extra
    a, b = run_both(sc, pair.bounds, ang, m, 3, gbest_order=gbest_order, integrator=api.DOPRI5,
                    rtol=1e-12, atol=1e-12)
    assert_same(a, b)
    pair.close()


def test_balanced_dopri5_paper_scale_choice_and_oracle():
    """At 65,536 particles on the paper-scale arc the automatic choice takes the balanced
    DOPRI5 form on GB300; its initial evaluation's sampled costs match the oracle's."""
    import torch

    import scenarios as S
    from paper_2207_13175_gb300 import api
    from paper_2207_13175_gb300 import inputs as I
    sc = I.paper_scale("halo", 0, integrator="dopri5")
    pair = S.Pair(sc, integrator="dopri5")
    pair.gpu.run(sc.m, 1, sc.w, sc.c1, sc.c2, sc.seed)
    r = pair.gpu.result(trace=False)
    if torch.cuda.get_device_properties(0).multi_processor_count == 152:
        assert r["schedule"] == api.SCHED_BALANCED
    sw = pair.gpu.swarm_get()
    sample = np.arange(0, sc.m, sc.m // 24)
    X = sw["x"][:, sample].T
    states = pair.gpu.propagate(X).cpu().numpy()
    for j, i in enumerate(sample):
        Jo = pair.ora.cost(X[j])
        ref, _, _ = pair.ora.propagate(X[j])
        assert abs(sw["J"][i] - Jo) <= S.cost_tolerance(pair, ref, Jo, states[:, :, j] - ref), i
    pair.close()
