"""Pins of the oracle's Levenberg-Marquardt refinement (Eqs. 14-16): it reaches the
minimum an independent solver (SciPy's MINPACK Levenberg-Marquardt) reaches on the same
residuals, recovers the truth from noise-free data, never increases the cost, and ends
at a stationary point of the least-squares cost."""
import numpy as np
import pytest


def problem(O, I, noise=True, stride=4, seed=0):
    sc = I.paper_scale("halo", seed, noise=noise)
    sc = sc.with_(t=sc.t[::stride], noise=sc.noise[::stride])
    ra, dec, _, _ = O.simulate_obs(sc.mu, sc.chief, sc.deputy, sc.t, sc.noise)
    P = O.Problem(sc.mu, sc.chief, sc.t, ra, dec, *sc.sigma, dt=sc.dt)
    x0 = sc.deputy + np.array([5.0, -3.0, 2.0, 0, 0, 0]) / I.L_KM + np.array([0, 0, 0, 1e-3, -5e-4, 0])
    return sc, P, x0


def test_lm_matches_independent_solver(O, I):
    scipy_opt = pytest.importorskip("scipy.optimize")
    sc, P, x0 = problem(O, I)
    x, c, it, rc = P.lm_refine(x0, 40)
    assert rc == 0 and it < 40
    sol = scipy_opt.least_squares(lambda v: P.lm_residuals(v, O.LM_RESIDUALS), x0, method="lm",
                                  xtol=1e-15, ftol=1e-15, gtol=1e-15,
                                  x_scale=np.array([1, 1, 1, 0.1, 0.1, 0.1]))
    assert c == pytest.approx(2 * sol.cost, rel=1e-7)
    assert np.max(np.abs(x - sol.x)) < 1e-10
    assert c <= P.cost(sc.deputy)            # the least-squares fit beats the truth itself


def test_lm_recovers_truth_without_noise(O, I):
    sc, P, x0 = problem(O, I, noise=False)
    x, c, it, rc = P.lm_refine(x0, 40)
    assert rc == 0
    assert np.max(np.abs(x[:3] - sc.deputy[:3])) < 1e-10      # 4 cm
    assert np.max(np.abs(x[3:] - sc.deputy[3:])) < 1e-9
    assert c < 1e-6
    # the paper's per-epoch chi-square vector has the same noise-free minimiser
    x2, c2, it2, rc2 = P.lm_refine(x0, 200, form=O.LM_EPOCH_CHI2)
    assert rc2 == 0 and np.max(np.abs(x2[:3] - sc.deputy[:3])) < 1e-8


def test_lm_monotone_and_stationary(O, I):
    sc, P, x0 = problem(O, I, seed=3)
    c0 = float(np.sum(P.lm_residuals(x0) ** 2))
    prev = c0
    for n in (1, 2, 4, 8, 30):
        x, c, it, rc = P.lm_refine(x0, n)
        assert c <= prev + 1e-9 * prev
        prev = c
    # at the solution the first-order change of ||r||^2 over a difference step is
    # negligible against the cost itself
    r = P.lm_residuals(x)
    for j in range(6):
        h = 1e-7 * max(abs(x[j]), 0.1)
        e = np.zeros(6)
        e[j] = h
        dJ = 2 * r @ ((P.lm_residuals(x + e) - P.lm_residuals(x - e)) / 2)
        assert abs(dJ) < 1e-6 * prev, (j, dJ, prev)


def test_estimation_error_matches_the_cramer_rao_bound(O, I):
    """With 1 arcsec noise the least-squares estimate's error against the truth is
    distributed as the linearised theory says: (x - x_true)^T F (x - x_true) ~ chi^2_6
    with F = J^T J the Fisher information of the weighted residuals (J by central
    differences at the estimate).  Sixteen seeded problems (paper-scale halo geometry,
    50 epochs over 7 days): every value below 40 (chi^2_6 exceeds 40 with probability
    3e-7), their mean within [3, 9.5] (the mean of sixteen has sd 0.87 about 6)."""
    d2 = []
    for seed in range(16):
        sc, P, _ = problem(O, I, noise=True, seed=seed)
        x, c, it, rc = P.lm_refine(sc.deputy, 40)
        assert rc == 0
        r0 = P.lm_residuals(x)
        Jm = np.empty((r0.size, 6))
        for j in range(6):
            h = 1e-7 * max(abs(x[j]), 0.1)
            e = np.zeros(6)
            e[j] = h
            Jm[:, j] = (P.lm_residuals(x + e) - P.lm_residuals(x - e)) / (2 * h)
        F = Jm.T @ Jm
        dx = x - sc.deputy
        d2.append(float(dx @ F @ dx))
    assert max(d2) < 40.0, d2
    assert 3.0 <= float(np.mean(d2)) <= 9.5, d2
