"""Pins of the oracle's elliptic restricted three-body problem (the paper's future work):
the e = 0 reduction to Eqs. 1-3, equilibria at the Lagrange points for any
eccentricity and true anomaly, the energy-rate identity that ties the right-hand side
to the pulsating potential omega, and Kepler's equation behind the time mapping."""
import math

import numpy as np
import pytest

MU = 0.01215058560962404
ECC = 0.0549


def omega(mu, e, f, s):
    """The pulsating potential, written out independently of the oracle."""
    x, y, z = s[:3]
    r1 = math.sqrt((x + mu) ** 2 + y * y + z * z)
    r2 = math.sqrt((x - 1 + mu) ** 2 + y * y + z * z)
    return (0.5 * (x * x + y * y - e * z * z * math.cos(f)) + (1 - mu) / r1 + mu / r2) / (1 + e * math.cos(f))


def domega_df(mu, e, f, s):
    """Explicit dependence of omega on f at a fixed position."""
    x, y, z = s[:3]
    r1 = math.sqrt((x + mu) ** 2 + y * y + z * z)
    r2 = math.sqrt((x - 1 + mu) ** 2 + y * y + z * z)
    c = 1 + e * math.cos(f)
    om = 0.5 * (x * x + y * y - e * z * z * math.cos(f)) + (1 - mu) / r1 + mu / r2
    return (0.5 * e * z * z * math.sin(f)) / c + om * e * math.sin(f) / c ** 2


def test_zero_eccentricity_is_the_cr3bp(O):
    rng = np.random.default_rng(0)
    for _ in range(50):
        s = np.concatenate([rng.uniform(-1.5, 1.5, 3), rng.uniform(-1, 1, 3)])
        a = O.rhs_er3bp(MU, 0.0, rng.uniform(0, 6.3), s)
        b = np.empty(6)
        O.lib().ora_rhs(MU, O._dp(s), O._dp(b))
        assert np.allclose(a, b, rtol=1e-14, atol=1e-14)


def test_lagrange_points_stay_equilibria(O):
    """omega's gradient vanishes where the CR3BP's does (the z term is zero in the plane),
    so L1-L5 are equilibria of the pulsating frame at every true anomaly."""
    # collinear points from the quintics in gamma (Szebehely)
    g1 = [r for r in np.roots([1, -(3 - MU), 3 - 2 * MU, -MU, 2 * MU, -MU]) if abs(r.imag) < 1e-12 and 0 < r.real < 1][0].real
    g2 = [r for r in np.roots([1, 3 - MU, 3 - 2 * MU, -MU, -2 * MU, -MU]) if abs(r.imag) < 1e-12 and 0 < r.real < 1][0].real
    g3 = [r for r in np.roots([1, 2 + MU, 1 + 2 * MU, -(1 - MU), -2 * (1 - MU), -(1 - MU)]) if abs(r.imag) < 1e-12 and 0 < r.real < 2][0].real
    pts = [(1 - MU - g1, 0, 0), (1 - MU + g2, 0, 0), (-MU - g3, 0, 0),
           (0.5 - MU, math.sqrt(3) / 2, 0), (0.5 - MU, -math.sqrt(3) / 2, 0)]
    for p in pts:
        for f in (0.0, 1.1, 2.5, 4.0):
            ds = O.rhs_er3bp(MU, ECC, f, np.array([*p, 0, 0, 0]))
            assert np.max(np.abs(ds[3:])) < 1e-13, (p, f, ds)


def test_energy_rate_identity(O):
    """Along any solution d/df (|v|^2/2 - omega) = -d(omega)/df at fixed position: the
    Coriolis terms do no work and omega's spatial gradient is the acceleration."""
    integ = pytest.importorskip("scipy.integrate")
    s0 = np.array([1.12, 0.02, -0.15, 0.01, -0.21, 0.005])
    f0, f1 = 0.7, 2.9
    sol = integ.solve_ivp(lambda f, s: O.rhs_er3bp(MU, ECC, f, s), (f0, f1), s0, method="DOP853",
                          rtol=1e-13, atol=1e-13, dense_output=True)
    assert sol.success

    def energy(f):
        s = sol.sol(f)
        return 0.5 * float(s[3:] @ s[3:]) - omega(MU, ECC, f, s)
    work, _ = integ.quad(lambda f: -domega_df(MU, ECC, f, sol.sol(f)), f0, f1, epsabs=1e-13,
                         epsrel=1e-12, limit=400)
    assert energy(f1) - energy(f0) == pytest.approx(work, rel=1e-8, abs=1e-11)
    assert abs(work) > 1e-3            # the identity is not trivially zero here
    # a dropped or sign-flipped term breaks it: the same check on the CR3BP right-hand
    # side (which ignores e) fails
    bad = integ.solve_ivp(lambda f, s: O.rhs_er3bp(MU, 0.0, f, s), (f0, f1), s0, method="DOP853",
                          rtol=1e-13, atol=1e-13, dense_output=True)
    eb = lambda f: 0.5 * float(bad.sol(f)[3:] @ bad.sol(f)[3:]) - omega(MU, ECC, f, bad.sol(f))
    wb, _ = integ.quad(lambda f: -domega_df(MU, ECC, f, bad.sol(f)), f0, f1, limit=400)
    assert abs((eb(f1) - eb(f0)) - wb) > 1e-4


def test_time_to_true_anomaly_follows_keplers_equation(O):
    """f(tau) from the oracle turned back into a mean anomaly by the inverse half-angle
    relation advances by exactly tau; half a period from periapsis lands on apoapsis;
    a full period adds 2 pi; e = 0 is f0 + tau."""
    b = ECC / (1 + math.sqrt(1 - ECC * ECC))

    def mean_anomaly(f):
        E = f - 2 * math.atan(b * math.sin(f) / (1 + b * math.cos(f)))
        return E - ECC * math.sin(E)
    for f0 in (0.0, 0.4, 3.0, -2.0):
        M0 = mean_anomaly(f0)
        prev = f0
        for tau in (0.01, 0.5, 1.0, 2.7, 6.0, 11.3):
            f = O.er3bp_anomaly(ECC, f0, tau)
            assert f > prev
            prev = f
            assert mean_anomaly(f) - M0 == pytest.approx(tau, abs=2e-13)
        assert O.er3bp_anomaly(ECC, f0, 2 * math.pi) - f0 == pytest.approx(2 * math.pi, abs=1e-12)
    assert O.er3bp_anomaly(ECC, 0.0, math.pi) == pytest.approx(math.pi, abs=1e-13)
    assert O.er3bp_anomaly(0.0, 0.3, 1.7) == 0.3 + 1.7


def test_er3bp_problem_reduces_to_the_cr3bp(O, I):
    """A whole ER3BP problem with tiny eccentricity propagates and scores like the CR3BP
    one; with the Moon's eccentricity the deputy's path differs by kilometres."""
    sc = I.tiny(0)
    ra, dec, _, _ = O.simulate_obs(sc.mu, sc.chief, sc.deputy, sc.t, sc.noise)
    Pc = O.Problem(sc.mu, sc.chief, sc.t, ra, dec, *sc.sigma, dt=sc.dt)
    Pe = O.Problem(sc.mu, sc.chief, sc.t, ra, dec, *sc.sigma, dt=sc.dt, dynamics=O.ER3BP,
                   ecc=1e-14, f0=0.3)
    a, _, _ = Pc.propagate(sc.deputy)
    b, _, _ = Pe.propagate(sc.deputy)
    assert np.max(np.abs(a - b)) < 1e-12
    # the chief-deputy distance is ~1e-4 LU, so 1e-12 in the states moves the angles by
    # ~1e-8 rad (~0.002 sigma): the costs agree to ~1e-7 relative
    assert Pe.cost(sc.deputy) == pytest.approx(Pc.cost(sc.deputy), rel=1e-6)
    Pm = O.Problem(sc.mu, sc.chief, sc.t, ra, dec, *sc.sigma, dt=sc.dt, dynamics=O.ER3BP,
                   ecc=ECC, f0=0.3)
    c, _, _ = Pm.propagate(sc.deputy)
    assert np.max(np.abs(a[:, :3] - c[:, :3])) * I.L_KM > 10.0
    # observations simulated in the ER3BP fit the ER3BP problem at the truth
    ra2, dec2, _, _ = O.simulate_obs(sc.mu, sc.chief, sc.deputy, sc.t, None, ecc=ECC, f0=0.3)
    Pm2 = O.Problem(sc.mu, sc.chief, sc.t, ra2, dec2, *sc.sigma, dt=sc.dt, dynamics=O.ER3BP,
                    ecc=ECC, f0=0.3)
    assert Pm2.cost(sc.deputy) < 1e-2
