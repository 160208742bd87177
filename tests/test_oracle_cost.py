"""Pins of the oracle's measurement model and cost (Eqs. 5-13) against special cases
with known answers and closed forms."""
import math

import numpy as np
import pytest


@pytest.mark.parametrize("rho,alpha,beta", [
    ((1, 0, 0), 0.0, 0.0),
    ((0, 1, 0), math.pi / 2, 0.0),
    ((-1, 0, 0), math.pi, 0.0),
    ((0, -1, 0), -math.pi / 2, 0.0),
    ((0, 0, 1), 0.0, math.pi / 2),
    ((0, 0, -2), 0.0, -math.pi / 2),
    ((1, 1, 0), math.pi / 4, 0.0),
    ((1, 0, 1), 0.0, math.pi / 4),
    ((-1, -1, math.sqrt(2)), -3 * math.pi / 4, math.pi / 4),
])
def test_angle_special_cases(O, rho, alpha, beta):
    a, b, r = O.angles(np.array(rho, dtype=float) * 3e-4)
    assert a == pytest.approx(alpha, abs=1e-15)
    assert b == pytest.approx(beta, abs=2e-8 if abs(beta) == math.pi / 2 else 1e-15)
    assert r == pytest.approx(3e-4 * np.linalg.norm(rho), rel=1e-15)


def _problem(O, I, sc, obs_from="rk4", noise=True, **kw):
    """Observations generated with the estimator's own integrator (so that J at the
    truth is exactly the weighted noise energy) or with DOPRI5 at 1e-13."""
    nz = sc.noise if noise else np.zeros_like(sc.noise)
    if obs_from == "rk4":
        P0 = O.Problem(sc.mu, sc.chief, sc.t, np.zeros(sc.n_obs), np.zeros(sc.n_obs),
                       *sc.sigma, dt=sc.dt)
        sd, _, _ = P0.propagate(sc.deputy)
        ra, dec, rng = np.empty(sc.n_obs), np.empty(sc.n_obs), np.empty(sc.n_obs)
        for k in range(sc.n_obs):
            ra[k], dec[k], rng[k] = O.angles(sd[k, :3] - P0.rc[k])
        ra, dec = ra + nz[:, 0], dec + nz[:, 1]
    else:
        ra, dec, rng, _ = O.simulate_obs(sc.mu, sc.chief, sc.deputy, sc.t, nz)
    return O.Problem(sc.mu, sc.chief, sc.t, ra, dec, *sc.sigma, dt=sc.dt, rng=rng, **kw)


def test_cost_at_truth_is_weighted_noise_energy(O, I):
    """With observations from the estimator's own propagation plus noise n_k,
    J(truth) = sum_k (n_ra^2/s_ra^2 + n_dec^2/s_dec^2) (CHI2) and
    sum_k (n_ra^2/s_ra^2 + n_dec^2/s_dec^2)^2 (QUARTIC) exactly up to rounding."""
    sc = I.tiny(3)
    sig = (I.ARCSEC, 2.0 * I.ARCSEC)
    sc = sc.with_(sigma=sig)
    per = sc.noise[:, 0] ** 2 / sig[0] ** 2 + sc.noise[:, 1] ** 2 / sig[1] ** 2
    P = _problem(O, I, sc)
    assert P.cost(sc.deputy) == pytest.approx(per.sum(), rel=1e-7)
    Pq = _problem(O, I, sc, cost_form=O.COST_QUARTIC)
    assert Pq.cost(sc.deputy) == pytest.approx((per ** 2).sum(), rel=1e-7)
    # noise-free: zero in both forms, positive away from the truth
    P0 = _problem(O, I, sc, noise=False)
    assert P0.cost(sc.deputy) < 1e-12
    off = sc.deputy + np.array([10 / I.L_KM, 0, 0, 0, 0, 0])
    assert P0.cost(off) > 1e3


def test_range_term(O, I):
    sc = I.tiny(4)
    s_rng = 0.05 / I.L_KM
    P = _problem(O, I, sc, use_range=True, sigma_rng=s_rng)
    base = ((sc.noise / I.ARCSEC) ** 2).sum()
    assert P.cost(sc.deputy) == pytest.approx(base, rel=1e-6)
    # perturb the observed ranges by a known amount: J rises by sum (d/s_rng)^2
    d = 0.01 / I.L_KM
    P2 = O.Problem(sc.mu, sc.chief, sc.t, P.ra, P.dec, *sc.sigma, dt=sc.dt, rng=P.rng + d,
                   sigma_rng=s_rng, use_range=True)
    assert P2.cost(sc.deputy) == pytest.approx(base + sc.n_obs * (d / s_rng) ** 2, rel=1e-6)


def test_truth_with_dopri_observations(O, I):
    sc = I.tiny(0)
    P = _problem(O, I, sc, obs_from="dopri5")
    energy = ((sc.noise / I.ARCSEC) ** 2).sum()
    assert P.cost(sc.deputy) == pytest.approx(energy, rel=1e-5)
    Pn = _problem(O, I, sc, obs_from="dopri5", noise=False)
    assert Pn.cost(sc.deputy) < 1e-8          # integrator-mismatch floor, << 1 sigma


def test_azimuth_residual_wraps(O, I):
    """An observed azimuth one full turn away, or just across +-pi, costs the same as
    the short way round."""
    sc = I.tiny(1)
    P = _problem(O, I, sc)
    J = P.cost(sc.deputy)
    for shift in (2 * math.pi, -2 * math.pi, 4 * math.pi):
        Ps = O.Problem(sc.mu, sc.chief, sc.t, P.ra + shift, P.dec, *sc.sigma, dt=sc.dt)
        assert Ps.cost(sc.deputy) == pytest.approx(J, rel=1e-6)


def test_frame_rotation_invariance(O, I):
    """Rotating every position about z by theta_k at each epoch and adding theta_k to
    the observed azimuths leaves J unchanged (the synodic vs inertial choice of frame
    is immaterial when observations are formed in the same frame)."""
    sc = I.tiny(2)
    P = _problem(O, I, sc)
    sd, _, _ = P.propagate(sc.deputy)
    theta = 0.3 + 2.9 * np.arange(sc.n_obs)
    c, s = np.cos(theta), np.sin(theta)

    def rot(v):
        out = v.copy()
        out[:, 0] = c * v[:, 0] - s * v[:, 1]
        out[:, 1] = s * v[:, 0] + c * v[:, 1]
        return out

    Pr = O.Problem(sc.mu, sc.chief, sc.t, P.ra + theta, P.dec, *sc.sigma, dt=sc.dt)
    Pr.rc[:] = rot(P.rc)
    sdr = sd.copy()
    sdr[:, :3] = rot(sd[:, :3])
    assert Pr.cost_from_states(sdr) == pytest.approx(P.cost_from_states(sd), rel=1e-6)


def test_degenerate_line_of_sight_is_infinite(O, I):
    sc = I.tiny(0)
    P = _problem(O, I, sc)
    sd, _, _ = P.propagate(sc.deputy)
    st = sd.copy()
    st[5, :3] = P.rc[5]
    assert P.cost_from_states(st) == math.inf
    st = sd.copy()
    st[3, 0] = math.nan
    assert P.cost_from_states(st) == math.inf


def test_chi2_statistics_at_truth(O, I):
    """With 1-sigma Gaussian noise J(truth) is chi-square with 2K degrees of freedom."""
    vals = []
    for seed in range(40):
        sc = I.tiny(seed)
        vals.append(_problem(O, I, sc, obs_from="dopri5").cost(sc.deputy))
    K = I.tiny().n_obs
    assert abs(np.mean(vals) - 2 * K) < 4 * math.sqrt(4 * K / len(vals))
