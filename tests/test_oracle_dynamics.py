"""Pins of the oracle's dynamics and propagators (Eqs. 1-3) against facts the paper
and textbook mechanics fix: equilibria and their linear spectra, the Jacobi integral,
the mirror/time-reversal symmetry, the paper's printed periodic orbits, and the
integrators' orders."""
import math

import numpy as np
import pytest

from oracle import periodic as P


def fd_jacobian(O, mu, s, eps=1e-6):
    s = np.asarray(s, dtype=float)
    A = np.empty((6, 6))
    for j in range(6):
        sp, sm = s.copy(), s.copy()
        sp[j] += eps
        sm[j] -= eps
        A[:, j] = (O.rhs(mu, sp) - O.rhs(mu, sm)) / (2 * eps)
    return A


def test_collinear_points_are_equilibria(O, mu):
    xl1, xl2 = P.collinear_points(mu)
    # L3 from its own quintic: gamma^5 + (2+mu) gamma^4 + (1+2mu) gamma^3 - (1-mu) gamma^2
    #                          - 2(1-mu) gamma - (1-mu) = 0, x_L3 = -mu - gamma
    r = np.roots([1, 2 + mu, 1 + 2 * mu, -(1 - mu), -2 * (1 - mu), -(1 - mu)])
    g3 = [v.real for v in r if abs(v.imag) < 1e-12 and v.real > 0][0]
    xl3 = -mu - g3
    assert xl1 == pytest.approx(0.8369151257723572, abs=1e-13)
    assert xl2 == pytest.approx(1.155682165444884, abs=1e-13)
    assert xl3 == pytest.approx(-1.0050626458102778, abs=1e-13)
    for x in (xl1, xl2, xl3):
        assert np.max(np.abs(O.rhs(mu, [x, 0, 0, 0, 0, 0]))) < 1e-14
    # equilateral points
    for y in (math.sqrt(3) / 2, -math.sqrt(3) / 2):
        assert np.max(np.abs(O.rhs(mu, [0.5 - mu, y, 0, 0, 0, 0]))) < 1e-14
    # and a point that is not an equilibrium
    assert np.max(np.abs(O.rhs(mu, [0.9, 0, 0, 0, 0, 0]))) > 1e-2


def test_linear_spectra_match_closed_forms(O, mu):
    """Eigenvalues of the Jacobian of Eqs. 1-3 at the libration points against their
    closed forms (Szebehely): at L4, lambda^4 + lambda^2 + 27/4 mu(1-mu) = 0; at a collinear
    point with c2 = (1-mu)/r1^3 + mu/r2^3, in-plane lambda^2 = (c2-2 +- sqrt(9c2^2-8c2))/2 and
    out-of-plane lambda^2 = -c2.  These pin the Coriolis and centrifugal terms as well
    as the gravity terms."""
    A = fd_jacobian(O, mu, [0.5 - mu, math.sqrt(3) / 2, 0, 0, 0, 0])
    ev = np.linalg.eigvals(A)
    disc = math.sqrt(1 - 27 * mu * (1 - mu))
    w = sorted([math.sqrt((1 + disc) / 2), math.sqrt((1 - disc) / 2), 1.0])
    got = sorted(set(np.round(np.abs(ev.imag), 7)))
    assert np.max(np.abs(ev.real)) < 1e-7
    assert np.allclose(got, w, atol=1e-7)
    for x in P.collinear_points(mu):
        c2 = (1 - mu) / abs(x + mu) ** 3 + mu / abs(x - 1 + mu) ** 3
        ev = np.linalg.eigvals(fd_jacobian(O, mu, [x, 0, 0, 0, 0, 0]))
        lam_real = math.sqrt((c2 - 2 + math.sqrt(9 * c2 * c2 - 8 * c2)) / 2)
        w_xy = math.sqrt(-(c2 - 2 - math.sqrt(9 * c2 * c2 - 8 * c2)) / 2)
        w_z = math.sqrt(c2)
        assert np.max(np.abs(np.sort(ev.real)[[0, -1]] - [-lam_real, lam_real])) < 1e-6
        imag = sorted(np.abs(ev.imag[np.abs(ev.imag) > 1e-3]))
        assert np.allclose(imag, sorted([w_xy, w_xy, w_z, w_z]), atol=1e-6)


def test_jacobi_constant_rk4_fourth_order(O, mu):
    s0 = [0.85, 0, 0.17, 0, 0.26, 0]
    C0 = O.jacobi(mu, s0)
    drift = []
    for dt in (4e-3, 2e-3, 1e-3):
        s = O.rk4_steps(mu, s0, dt, int(round(1.0 / dt)))
        drift.append(abs(O.jacobi(mu, s) - C0))
    assert drift[2] < 1e-10
    for a, b in zip(drift, drift[1:]):
        assert 12.0 < a / b < 20.0          # 2^4 = 16 per halving


def test_time_reversal_and_mirror_symmetry(O, mu):
    s0 = np.array([0.85, 0.01, 0.17, 0.02, 0.26, -0.01])
    h, n = 1e-3, 500
    s1 = O.rk4_steps(mu, s0, h, n)
    back = O.rk4_steps(mu, s1, -h, n)
    assert np.max(np.abs(back - s0)) < 1e-11
    # (x, -y, z, -vx, vy, -vz) run backwards in time mirrors the forward solution
    M = np.array([1, -1, 1, -1, 1, -1], dtype=float)
    mirrored = O.rk4_steps(mu, M * s0, -h, n)
    assert np.max(np.abs(mirrored - M * s1)) < 1e-13


@pytest.mark.parametrize("name,s0,half_guess,C_printed", [
    # Table 2 deputy (L2 southern halo), Table 2 chief (L2 halo), Table 3 chief (L2 axial)
    ("t2-deputy", [1.140135389, 0, -1.63176653574390E-01, 6.13321115086310E-15, -0.223383154,
                   1.78644826151404E-15], 1.5547, 3.06),
    ("t2-chief", [1.029726968, 0, -1.869397163946E-01, -5.585615805585E-14, -0.119441863,
                  -9.803996218373E-13], 0.8065, 3.04),
    ("t3-chief", [1.21996614837886E+00, 0, -2.49454877925228E-16, 1.10859609358602E-15,
                  -4.27475884185211E-01, 4.09809301627323E-03], 2.1553, 3.01),
])
def test_paper_initial_conditions_are_periodic(O, mu, name, s0, half_guess, C_printed):
    """The paper's printed initial conditions (Tables 2, 3) return to themselves after
    one period under the oracle's dynamics, and have the printed Jacobi constants."""
    s0 = np.asarray(s0, dtype=float)
    assert round(O.jacobi(mu, s0), 2) == pytest.approx(C_printed)
    th = P.first_crossing(mu, s0, t_min=half_guess - 0.2, t_max=half_guess + 0.2, dt=0.005)
    assert th == pytest.approx(half_guess, abs=2e-3)
    out, _, _, rc = O.propagate_dopri5(mu, s0, [2 * th], rtol=1e-13, atol=1e-13)
    assert rc == 0
    # the printed digits (9-15) bound how closely the orbit can close
    assert np.max(np.abs(out[0] - s0)) < 1e-6


def test_self_corrected_orbits_are_periodic(O, mu, I):
    for name, orb in I.chief_orbits().items():
        s0 = np.array(orb["state"])
        out, _, _, rc = O.propagate_dopri5(mu, s0, [orb["period_tu"]], rtol=1e-13, atol=1e-13)
        assert rc == 0
        assert np.max(np.abs(out[0] - s0)) < 1e-10, name
        # and the RK4 propagator at the paper-scale step agrees over a period
        outr, _, rc = O.propagate_rk4(mu, s0, [orb["period_tu"]], 5e-4)
        assert np.max(np.abs(outr[0] - s0)) < 1e-8, name


def test_rk4_grid_lands_on_observation_times(O, I):
    sc = I.tiny()
    ns, h = O.rk4_grid(sc.t, sc.dt)
    assert ns[0] == 0 and h[0] == 0.0
    assert np.all(ns[1:] == 13) and ns.sum() == 247
    sc2 = I.paper_scale("halo")
    ns2, _ = O.rk4_grid(sc2.t, 5e-4)
    assert np.all(ns2[1:] == 17) and ns2.sum() == 3383
    # first time after zero gets its own interval from t = 0
    ns3, h3 = O.rk4_grid([0.0105, 0.011], 1e-3)
    assert ns3.tolist() == [11, 1] and h3[0] == pytest.approx(0.0105 / 11, rel=1e-15)
    with pytest.raises(ValueError):
        O.rk4_grid([0.2, 0.1], 1e-3)


def test_dopri5_step_and_dense_output_orders(O, mu):
    """One DOPRI5 step has local error O(h^5) (ratio ~32 per halving, fifth-order
    solution is O(h^6) locally), and the continuous extension at mid-step is O(h^5);
    the continuous extension reproduces y0, y1 and the end-point derivatives."""
    s0 = np.array([0.85, 0, 0.17, 0, 0.26, 0])

    def exact(t):
        return O.rk4_steps(mu, s0, t / 4000, 4000)

    e_step, e_mid = [], []
    for h in (0.08, 0.04, 0.02):
        s1, k, _ = O.dopri5_attempt(mu, h, s0)
        e_step.append(np.max(np.abs(s1 - exact(h))))
        e_mid.append(np.max(np.abs(O.dopri5_dense(h, s0, k, 0.5) - exact(h / 2))))
    for a, b in zip(e_step, e_step[1:]):
        assert a / b > 40.0            # ~64 for a local O(h^6) error
    for a, b in zip(e_mid, e_mid[1:]):
        assert 20.0 < a / b < 45.0     # ~32 for a local O(h^5) error
    h = 0.05
    s1, k, _ = O.dopri5_attempt(mu, h, s0)
    assert np.max(np.abs(O.dopri5_dense(h, s0, k, 0.0) - s0)) < 1e-16
    assert np.max(np.abs(O.dopri5_dense(h, s0, k, 1.0) - s1)) < 1e-15
    d = 1e-6
    deriv0 = (O.dopri5_dense(h, s0, k, d) - O.dopri5_dense(h, s0, k, -d)) / (2 * d * h)
    deriv1 = (O.dopri5_dense(h, s0, k, 1 + d) - O.dopri5_dense(h, s0, k, 1 - d)) / (2 * d * h)
    assert np.max(np.abs(deriv0 - O.rhs(mu, s0))) < 1e-7
    assert np.max(np.abs(deriv1 - O.rhs(mu, s1))) < 1e-7


def test_dopri5_matches_fine_rk4(O, mu, I):
    s0 = np.array([0.85, 0, 0.17, 0, 0.26, 0])
    t = np.linspace(0, 1.0, 37)
    out, acc, rej, rc = O.propagate_dopri5(mu, s0, t, rtol=1e-12, atol=1e-12)
    assert rc == 0 and acc > 10
    ref, _, _ = O.propagate_rk4(mu, s0, t, 1e-3 / 16)
    assert np.max(np.abs(out - ref)) < 1e-11
    # observation at t = 0 is the initial state itself
    assert np.array_equal(out[0], s0)


def test_rk4_step_size_convergence_to_dopri5(O, mu):
    s0 = np.array([0.85, 0, 0.17, 0, 0.26, 0])
    ref, *_ = O.propagate_dopri5(mu, s0, [1.0], rtol=1e-14, atol=1e-14)
    errs = []
    for dt in (8e-3, 4e-3, 2e-3):
        out, _, _ = O.propagate_rk4(mu, s0, [1.0], dt)
        errs.append(np.max(np.abs(out[0] - ref[0])))
    for a, b in zip(errs, errs[1:]):
        assert 12.0 < a / b < 20.0
