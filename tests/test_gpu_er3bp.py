"""GPU parity of the elliptic restricted three-body dynamics (the paper's future work)
against the oracle, through the C ABI: propagated states, costs, a swarm run and the
Levenberg-Marquardt refinement; and the combinations the library rejects."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ECC, F0 = 0.0549, 0.7


@pytest.fixture(scope="module")
def S():
    import scenarios
    return scenarios


@pytest.fixture(scope="module")
def I():
    from paper_2207_13175_gb300 import inputs
    return inputs


@pytest.mark.parametrize("integrator", ["rk4", "dopri5"])
def test_er3bp_state_parity_after_one_tu(S, I, integrator):
    sc = I.tiny(0)
    t = np.linspace(0.0, 1.0, 41)
    sc = sc.with_(t=t, noise=np.zeros((41, 2)), integrator=integrator)
    pair = S.Pair(sc, integrator=integrator, er3bp=(ECC, F0))
    X = I.particles_in_box(pair.lo, pair.hi, 301, seed=4)
    got = pair.gpu.propagate(X).cpu().numpy()          # [K][6][m]
    worst = 0.0
    for i in range(0, 301, 10):
        ref, _, rc = pair.ora.propagate(X[i])
        assert rc == 0
        g = got[:, :, i]
        worst = max(worst, S.rel_state_err(g[-1], ref[-1]))
    assert worst <= S.STATE_RTOL, worst
    # the elliptic problem is really different from the circular one here
    circ = S.Pair(sc, integrator=integrator)
    ref_c, _, _ = circ.ora.propagate(X[0])
    assert np.max(np.abs(ref_c[-1, :3] - got[-1, :3, 0])) > 1e-5
    pair.close()
    circ.close()


def test_er3bp_cost_and_swarm_parity(S, I):
    sc = I.tiny(0)
    pair = S.Pair(sc, er3bp=(ECC, F0))
    X = I.particles_in_box(pair.lo, pair.hi, 400, seed=5)
    J = pair.gpu.eval(X).cpu().numpy()
    Jo = pair.ora.costs(X)
    assert np.allclose(J, Jo, rtol=1e-9, atol=0)
    iters = 30
    W, gJ, gi, gap = S.oracle_run_recorded(pair, sc.m, iters, sc.seed)
    pair.gpu.run(sc.m, iters, sc.w, sc.c1, sc.c2, sc.seed)
    r = pair.gpu.result()
    assert r["iters_done"] == iters
    S.assert_trace_parity(S, pair, r, W, gJ, gi, gap)
    assert r["cost"] < r["gcost_trace"][0]
    pair.close()


def test_er3bp_refinement_parity(S, I):
    sc = I.paper_scale("halo", 0)
    sc = sc.with_(t=sc.t[::4], noise=sc.noise[::4])
    pair = S.Pair(sc, er3bp=(ECC, F0))
    x0 = sc.deputy + np.array([3.0, -2.0, 1.0, 0, 0, 0]) / I.L_KM
    xg, cg, itg = pair.gpu.refine(x0, 40)
    xo, co, ito, rc = pair.ora.lm_refine(x0, 40)
    assert rc == 0
    assert cg == pytest.approx(co, rel=1e-8)
    assert np.max(np.abs(xg - xo)) < 2e-9
    assert np.linalg.norm(xg[:3] - sc.deputy[:3]) * I.L_KM < 1.0     # metre-level fit
    pair.close()


def test_er3bp_rejected_where_unsupported(I):
    from paper_2207_13175_gb300 import api
    sc = I.tiny(0)
    ang = np.zeros((sc.n_obs, 2))
    b = api.bounds_from_chief(sc.chief, 100.0, 1.0, I.L_KM, I.TU_S)
    for bad in (dict(dynamics=api.ER3BP, ecc=1.0), dict(dynamics=api.ER3BP, ecc=-0.1),
                dict(dynamics=api.ER3BP, ecc=0.05, precision=api.MIXED), dict(dynamics=2)):
        with pytest.raises(api.IodError):
            api.Problem(sc.mu, sc.chief, sc.t, ang, sc.sigma, b, api.options(**bad))
    with pytest.raises(api.IodError):
        api.Batch(api.options(dynamics=api.ER3BP, ecc=0.05), budget_bytes=1 << 26, max_resident=2)


def test_er3bp_observation_synthesis_matches_the_oracle(I):
    """The GPU's elliptic observation synthesis against the oracle's (both DOPRI5 at
    1e-13): angles within 1e-10 rad."""
    import oracle as O
    from paper_2207_13175_gb300 import api
    sc = I.tiny(2)
    ra, dec, rng, _ = O.simulate_obs(sc.mu, sc.chief, sc.deputy, sc.t, sc.noise, ecc=ECC, f0=F0)
    ang, rg = api.simulate_obs(sc.mu, sc.chief, sc.deputy, sc.t, sc.noise, ecc=ECC, f0=F0)
    assert np.max(np.abs(ang[:, 0] - ra)) < 1e-10 and np.max(np.abs(ang[:, 1] - dec)) < 1e-10
    assert np.allclose(rg, rng, rtol=1e-9)
    circ, _ = api.simulate_obs(sc.mu, sc.chief, sc.deputy, sc.t, sc.noise)
    assert np.max(np.abs(circ - ang)) > 1e-6

