"""Full-size parity against the oracle: the paper-scale DOPRI5 propagation (7-day arc,
200 epochs, tolerance 1e-12), including the paper's scenario-1 chief that passes
0.0118 LU from the Moon, and one post-move FP64 iteration of the 65,536-particle swarm
in the benchmark's launch configuration (the balanced schedule on GB300)."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# Stated bound for 7-day DOPRI5 states (relative, infinity norm per epoch): the two
# sides round differently (FMA contraction, the reciprocal-square-root refinement) and
# the lunar passages amplify those differences over the arc.
DOPRI5_7D_RTOL = 1e-11
STATS = {}


def _record(key, value):
    STATS[key] = value
    out = os.environ.get("IOD_STATS_DIR", "")
    if out and os.path.isdir(out):
        with open(os.path.join(out, "full_size_stats.json"), "w") as f:
            json.dump(STATS, f, indent=1)


@pytest.fixture(scope="module")
def S():
    import scenarios
    return scenarios


@pytest.fixture(scope="module")
def I():
    from paper_2207_13175_gb300 import inputs
    return inputs


@pytest.mark.parametrize("orbit", ["halo", "paper-s1"])
def test_dopri5_paper_scale_against_oracle(S, I, orbit):
    """300 swarm particles (the Philox initial positions, bit-exact on both sides) and 40
    candidates near the truth, propagated by DOPRI5 (rtol = atol = 1e-12) over the 7-day,
    200-epoch arc: states within the stated bound at every epoch, costs within the
    per-particle tolerance, and the attempted-step counts equal (no acceptance flips) or
    the flips counted."""
    import oracle as O
    sc = I.paper_scale(orbit, 0, integrator="dopri5")
    pair = S.Pair(sc, integrator="dopri5")
    m = 300
    pair.gpu.run(m, 0, sc.w, sc.c1, sc.c2, sc.seed)
    r = pair.gpu.result(trace=False)
    Wp = O.Swarm(m)
    O.Pso(pair.ora, pair.lo, pair.hi, seed=sc.seed).init(Wp)
    sw = pair.gpu.swarm_get()
    assert np.array_equal(sw["x"], Wp.x.T)
    # attempted steps of the initial evaluation: per particle on the oracle, summed on the GPU
    steps_o = np.array([pair.ora.propagate(Wp.x[i])[1] for i in range(m)])
    assert steps_o.sum() == Wp.steps
    _record(f"{orbit}_attempts_gpu", int(r["rk_steps"]))
    _record(f"{orbit}_attempts_oracle", int(Wp.steps))
    X = np.vstack([Wp.x, I.near_truth(sc.deputy, 40, 1.0, 0.01, seed=4)])
    out = pair.gpu.propagate(X).cpu().numpy()           # [K][6][n]
    J = pair.gpu.eval(X).cpu().numpy()
    worst, worst_cost = 0.0, 0.0
    for i in range(X.shape[0]):
        ref, _, rc = pair.ora.propagate(X[i])
        assert rc == 0
        worst = max(worst, S.rel_state_err(out[:, :, i], ref))
        Jo = pair.ora.cost(X[i])
        tol = S.cost_tolerance(pair, ref, Jo, out[:, :, i] - ref)
        assert abs(J[i] - Jo) <= tol, (i, J[i], Jo, tol)
        worst_cost = max(worst_cost, abs(J[i] - Jo) / Jo)
    _record(f"{orbit}_state_rel_err_7d", worst)
    _record(f"{orbit}_cost_rel_err_7d", worst_cost)
    _record(f"{orbit}_attempt_flips", int(r["rk_steps"]) - int(Wp.steps))
    assert worst <= DOPRI5_7D_RTOL, worst
    assert r["rk_steps"] == Wp.steps, (r["rk_steps"], Wp.steps)
    pair.close()


def test_post_move_iteration_full_size(S, I):
    """65,536 particles, 200 epochs over 7 days, RK4 dt 5e-4, the benchmark's launch
    configuration: after the GPU's first iteration the oracle is loaded with the GPU's
    swarm and both take the second iteration.  Positions and velocities bit for bit over
    the whole swarm; the costs of sampled particles within the per-particle tolerance
    (all within 1e-9 relative); personal-best decisions equal away from ties; the same
    global best."""
    import oracle as O
    import torch
    from paper_2207_13175_gb300 import api
    sc = I.paper_scale("halo", 0)
    pair = S.Pair(sc)
    G = pair.gpu
    G.run(sc.m, 1, sc.w, sc.c1, sc.c2, sc.seed)
    s1 = G.swarm_get()
    G.continue_(1)
    s2 = G.swarm_get()
    r = G.result(trace=False)
    if torch.cuda.get_device_properties(0).multi_processor_count == 152:
        assert r["schedule"] == api.SCHED_BALANCED
    W = O.Swarm(sc.m)
    W.x[:] = s1["x"].T
    W.v[:] = s1["v"].T
    W.p[:] = s1["p"].T
    W.pJ[:] = s1["pJ"]
    W.J[:] = s1["J"]
    W.g, W.gJ, W.gidx = s1["g"], s1["gJ"], s1["gidx"]
    pJ_prev = W.pJ.copy()
    pair.pso(seed=sc.seed).iterate(W, 2)
    assert np.array_equal(s2["x"], W.x.T)
    assert np.array_equal(s2["v"], W.v.T)
    rel = np.abs(s2["J"] - W.J) / np.abs(W.J)
    assert np.all(rel <= 1e-9), float(np.max(rel))
    sample = np.unique(np.concatenate([np.arange(0, sc.m, sc.m // 64), [sc.m - 1, W.gidx]]))
    states = G.propagate(W.x[sample]).cpu().numpy()
    for j, i in enumerate(sample):
        ref, _, _ = pair.ora.propagate(W.x[i])
        tol = S.cost_tolerance(pair, ref, W.J[i], states[:, :, j] - ref)
        assert abs(s2["J"][i] - W.J[i]) <= tol, (i, s2["J"][i], W.J[i], tol)
    decided = (np.abs(W.J - pJ_prev) > 1e-12 * np.abs(pJ_prev)) | (W.J == pJ_prev)
    assert np.array_equal(s2["p"][:, decided], W.p[decided].T)
    gap = S._best_two_gap(W.J)
    _record("post_move_cost_rel_max", float(np.max(rel)))
    _record("post_move_best_gap", gap)
    if gap > 1e-12:
        assert s2["gidx"] == W.gidx
        assert np.array_equal(s2["g"], W.g)
    pair.close()
