"""The mixed-precision form (FP32 offsets from the chief, FP64 cost sums, FP64
refinement) against the FP64 oracle.  Its error is stated rather than held to the FP64
bar: the bounds asserted here are the stated error figures of the mixed form (STATED
below); the measured errors are written to $IOD_STATS_DIR/mixed_stats.json when that
variable names a directory."""
import json
import math
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# stated errors of the mixed form against the FP64 oracle (positions in LU, angles in
# rad, costs relative); see test bodies for the workloads
STATED = {
    "pos_1tu": 2e-9,           # 0.8 m after 1 TU (tiny geometry)
    "pos_7d": 2e-8,            # 8 m after 7 days (paper-scale halo)
    "cost_rel_far": 2e-5,      # box particles (residuals >> sigma)
}
STATS = {}


def _record(key, value):
    STATS[key] = float(value)
    out = os.environ.get("IOD_STATS_DIR", "")
    if out and os.path.isdir(out):
        with open(os.path.join(out, "mixed_stats.json"), "w") as f:
            json.dump(STATS, f, indent=1)


@pytest.fixture(scope="module")
def S():
    import scenarios
    return scenarios


@pytest.fixture(scope="module")
def I():
    from paper_2207_13175_gb300 import inputs
    return inputs


def mixed_pair(S, I, sc, **kw):
    """A scenario on both sides, the GPU problem in mixed precision."""
    from paper_2207_13175_gb300 import api
    last = kw.pop("last", 50)
    pair = S.Pair(sc, **kw)
    opts = api.options(dt=sc.dt, precision=api.MIXED, fp64_last_iters=last)
    pair.gmix = api.Problem(sc.mu, sc.chief, sc.t, np.stack([pair.ra, pair.dec], 1), sc.sigma,
                            pair.bounds, opts)
    return pair


def test_mixed_states_one_tu(S, I):
    sc = I.tiny(0).with_(t=np.linspace(0, 1.0, 41),
                         noise=np.random.default_rng(1).normal(0, I.ARCSEC, (41, 2)))
    pair = mixed_pair(S, I, sc)
    X = np.vstack([I.particles_in_box(pair.lo, pair.hi, 300, seed=5), sc.deputy[None]])
    out = pair.gmix.propagate(X).cpu().numpy()
    err_p = err_v = 0.0
    for i in range(X.shape[0]):
        ref, _, _ = pair.ora.propagate(X[i])
        err_p = max(err_p, np.max(np.abs(out[:, :3, i] - ref[:, :3])))
        err_v = max(err_v, np.max(np.abs(out[:, 3:, i] - ref[:, 3:])))
    _record("pos_err_1tu_lu", err_p)
    _record("vel_err_1tu_vu", err_v)
    assert err_p <= STATED["pos_1tu"], err_p
    assert err_v <= 10 * STATED["pos_1tu"], err_v
    pair.gmix.close()
    pair.close()


def test_mixed_states_and_costs_paper_scale(S, I):
    sc = I.paper_scale("halo", 0)
    pair = mixed_pair(S, I, sc)
    X = np.vstack([I.particles_in_box(pair.lo, pair.hi, 200, seed=6),
                   I.near_truth(sc.deputy, 56, 2.0, 0.02, seed=7)])
    out = pair.gmix.propagate(X).cpu().numpy()
    J = pair.gmix.eval(X).cpu().numpy()
    err_p, rel_far, ang = 0.0, [], []
    for i in range(X.shape[0]):
        ref, _, _ = pair.ora.propagate(X[i])
        err_p = max(err_p, np.max(np.abs(out[:, :3, i] - ref[:, :3])))
        Jo = pair.ora.cost(X[i])
        if i < 200:
            rel_far.append(abs(J[i] - Jo) / Jo)
        b, rho, _ = S.residuals(pair, ref)
        ang.append(float(np.max(np.abs(out[:, :3, i] - ref[:, :3]).max(axis=1) / rho)))
    _record("pos_err_7d_lu", err_p)
    _record("cost_rel_far_max", max(rel_far))
    _record("cost_rel_far_median", float(np.median(rel_far)))
    _record("angle_err_from_state_7d_rad", max(ang))
    assert err_p <= STATED["pos_7d"], err_p
    assert max(rel_far) <= STATED["cost_rel_far"], max(rel_far)
    pair.gmix.close()
    pair.close()


def O_box(sc, r_km, v_ms):
    import oracle
    from paper_2207_13175_gb300 import inputs as I
    return oracle.bounds_from_chief(sc.chief, r_km, v_ms, I.L_KM, I.TU_S)


def test_mixed_fp64_near_moon(S, I):
    """The paper's scenario-1 chief passes 0.0118 LU from the Moon: candidates within
    50 km / 1 m/s of it pass with it, their steps inside the 0.02 LU radius run in FP64,
    and their states stay close to the FP64 oracle."""
    sc = I.paper_table(1)
    pair = mixed_pair(S, I, sc)
    lo, hi = O_box(sc, 50.0, 1.0)
    X = I.particles_in_box(lo, hi, 64, seed=3)
    out = pair.gmix.propagate(X).cpu().numpy()
    err = max(np.max(np.abs(out[:, :3, i] - pair.ora.propagate(X[i])[0][:, :3]))
              for i in range(X.shape[0]))
    _record("pos_err_moon_7d_lu", err)
    pair.gmix.run(64, 1, seed=1)
    r = pair.gmix.result(trace=False)
    _record("fp64_steps_moon_frac", r["fp64_steps"] / r["rk_steps"])
    assert r["fp64_steps"] > 0
    assert err <= 10 * STATED["pos_7d"], err
    pair.gmix.close()
    pair.close()


def test_mixed_run_against_fp64_oracle(S, I, ):
    """A noise-free paper-shaped solve (halo chief, 200 epochs over 7 days, 512
    particles, 60 iterations, the last 10 in FP64) in mixed precision against the FP64
    oracle's run on the same inputs: the reported cost is FP64, the final position error
    is no worse than 1.1x the oracle's and the final position lies within 1 m of the
    oracle's."""
    from paper_2207_13175_gb300 import api
    sc = I.paper_scale("halo", 2, noise=False)
    pair = mixed_pair(S, I, sc, last=10)
    m, iters = 512, 60
    W, gJ, gi = pair.pso(seed=4).run(m, iters)
    pair.gmix.run(m, iters, sc.w, sc.c1, sc.c2, 4)
    r = pair.gmix.result()
    truth = sc.deputy
    e_mix = np.linalg.norm(r["state"][:3] - truth[:3]) * I.L_KM
    e_ora = np.linalg.norm(W.g[:3] - truth[:3]) * I.L_KM
    _record("run_err_mixed_km", e_mix)
    _record("run_err_oracle_km", e_ora)
    # the reported best cost is an FP64 evaluation of the reported state
    fp = api.Problem(sc.mu, sc.chief, sc.t, np.stack([pair.ra, pair.dec], 1), sc.sigma,
                     pair.bounds, api.options(dt=sc.dt))
    J64 = fp.eval(r["state"][None, :]).cpu().numpy()[0]
    assert abs(J64 - r["cost"]) <= 1e-9 * J64
    assert r["iters_done"] == iters
    assert np.all(np.diff(r["gcost_trace"][iters - 10:]) <= 0)      # FP64 phase monotone
    # the final-error bar (no worse than 1.1x the oracle's), and the final
    # position within 1 m of the oracle's (measured: the same state)
    d_ora = np.linalg.norm(r["state"][:3] - W.g[:3]) * I.L_KM
    _record("run_state_diff_oracle_km", d_ora)
    assert e_mix <= 1.1 * e_ora, (e_mix, e_ora, d_ora)
    assert d_ora <= 1e-3, d_ora
    fp.close()
    pair.gmix.close()
    pair.close()


def test_mixed_deterministic(S, I):
    sc = I.tiny(6)
    pair = mixed_pair(S, I, sc, last=5)
    pair.gmix.run(300, 20, seed=9)
    a = pair.gmix.result()
    pair.gmix.run(300, 20, seed=9)
    b = pair.gmix.result()
    assert np.array_equal(a["state"], b["state"]) and np.array_equal(a["gcost_trace"], b["gcost_trace"])
    assert a["rk_steps"] == 300 * (20 + 1 + 1) * 247      # + one FP64 rescoring pass
    pair.gmix.close()
    pair.close()
