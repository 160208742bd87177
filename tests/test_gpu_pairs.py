"""Two threads per particle (a lane pair splitting the two primaries' attractions)
reproduce the one-thread swarm bit for bit: traces, final states, swarm arrays and step
counts, for ragged swarm sizes and both global-best orders."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("gbest_order", [0, 1])
@pytest.mark.parametrize("m", [1, 17, 100, 257])
def test_pairs_equal_single_threads(m, gbest_order):
    import scenarios as S
    from paper_2207_13175_gb300 import api
    from paper_2207_13175_gb300 import inputs as I
    sc = I.tiny(1)
    pair = S.Pair(sc, gbest_order=gbest_order)
    ang = np.stack([pair.ra, pair.dec], 1)
    out = []
    for tpp in (1, 2):
        opts = api.options(dt=sc.dt, gbest_order=gbest_order, threads_per_particle=tpp)
        with api.Problem(sc.mu, sc.chief, sc.t, ang, sc.sigma, pair.bounds, opts) as G:
            G.run(m, 12, sc.w, sc.c1, sc.c2, 9)
            out.append((G.result(), G.swarm_get()))
    (r1, w1), (r2, w2) = out
    assert np.array_equal(r1["state"], r2["state"]) and r1["cost"] == r2["cost"]
    assert np.array_equal(r1["gcost_trace"], r2["gcost_trace"])
    assert np.array_equal(r1["gidx_trace"], r2["gidx_trace"])
    assert r1["rk_steps"] == r2["rk_steps"]
    for k in ("x", "v", "p", "pJ", "J"):
        assert np.array_equal(w1[k], w2[k]), k
    pair.close()


@pytest.mark.parametrize("gbest_order", [0, 1])
@pytest.mark.parametrize("m", [1, 17, 257, 3000])
def test_dopri5_pairs_equal_single_threads(m, gbest_order):
    """DOPRI5 on lane pairs: every pair takes its own adaptive steps (the exchange names the
    pair alone), and the run equals the one-thread run bit for bit, attempts included."""
    import scenarios as S
    from paper_2207_13175_gb300 import api
    from paper_2207_13175_gb300 import inputs as I
    sc = I.tiny(2)
    pair = S.Pair(sc, integrator="dopri5", gbest_order=gbest_order)
    ang = np.stack([pair.ra, pair.dec], 1)
    out = []
    for tpp in (1, 2):
        opts = api.options(integrator=api.DOPRI5, rtol=sc.rtol, atol=sc.atol, h0=sc.h0,
                           gbest_order=gbest_order, threads_per_particle=tpp)
        with api.Problem(sc.mu, sc.chief, sc.t, ang, sc.sigma, pair.bounds, opts) as G:
            G.run(m, 6, sc.w, sc.c1, sc.c2, 5)
            out.append((G.result(), G.swarm_get()))
    (r1, w1), (r2, w2) = out
    assert np.array_equal(r1["state"], r2["state"]) and r1["cost"] == r2["cost"]
    assert np.array_equal(r1["gcost_trace"], r2["gcost_trace"])
    assert np.array_equal(r1["gidx_trace"], r2["gidx_trace"])
    assert r1["rk_steps"] == r2["rk_steps"]
    for k in ("x", "v", "p", "pJ", "J"):
        assert np.array_equal(w1[k], w2[k]), k
    pair.close()


def test_pairs_rejected_outside_fp64_circular(I=None):
    from paper_2207_13175_gb300 import api
    from paper_2207_13175_gb300 import inputs as I
    sc = I.tiny(0)
    b = api.bounds_from_chief(sc.chief, 100.0, 1.0, I.L_KM, I.TU_S)
    for bad in (dict(threads_per_particle=2, precision=api.MIXED),
                dict(threads_per_particle=2, dynamics=api.ER3BP, ecc=0.05),
                dict(threads_per_particle=3)):
        with pytest.raises(api.IodError):
            api.Problem(sc.mu, sc.chief, sc.t, np.zeros((sc.n_obs, 2)), sc.sigma, b, api.options(**bad))


L_KM = 384400.0


@pytest.mark.parametrize("variant", [
    dict(tol_tau=1e-3),
    dict(constriction=1, init_grid=1, velocity_init=1, per_dim_random=1),
    dict(init_cone=1, cone_rho_min=5.0 / L_KM, cone_rho_max=150.0 / L_KM, use_range=0),
])
def test_pairs_equal_single_threads_with_variants(variant):
    """The lane-pair kernels share the initialisation, move and Algorithm 2 code with the
    one-thread kernels: every variant gives the same run either way."""
    import scenarios as S
    from paper_2207_13175_gb300 import api
    from paper_2207_13175_gb300 import inputs as I
    sc = I.tiny(0)
    pair = S.Pair(sc)
    ang = np.stack([pair.ra, pair.dec], 1)
    coef = (1.0, 2.05, 2.05) if variant.get("constriction") else (sc.w, sc.c1, sc.c2)
    out = []
    for tpp in (1, 2):
        opts = api.options(dt=sc.dt, threads_per_particle=tpp, **variant)
        with api.Problem(sc.mu, sc.chief, sc.t, ang, sc.sigma, pair.bounds, opts) as G:
            G.run(sc.m, 60, *coef, sc.seed)
            out.append(G.result())
    assert out[0]["iters_done"] == out[1]["iters_done"]
    assert np.array_equal(out[0]["state"], out[1]["state"])
    assert np.array_equal(out[0]["gcost_trace"], out[1]["gcost_trace"])
    if "tol_tau" in variant:
        assert out[0]["iters_done"] < 60
    pair.close()
