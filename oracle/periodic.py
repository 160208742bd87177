"""Single-shooting differential corrector for symmetric periodic CR3BP orbits.

TEST INFRASTRUCTURE (scenario input generation).  The paper takes its periodic-orbit
initial conditions from JPL's periodic-orbit database, which is not available here;
these orbits stand in for it.  A symmetric orbit leaves the xz-plane perpendicularly
(y = vx = vz = 0) and returns to it perpendicularly after half a period, so the
corrector drives (y, vx[, vz]) at the half-period crossing to zero with Newton's method,
the Jacobian taken by central differences of the oracle's DOPRI5 propagation (tight
tolerances) and the crossing time's column by the equations of motion themselves.
"""
from __future__ import annotations

import numpy as np

from . import propagate_dopri5, rhs

TOL = dict(rtol=1e-13, atol=1e-13, h0=1e-3)


def state_at(mu, s0, t):
    out, _, _, rc = propagate_dopri5(mu, s0, np.array([float(t)]), **TOL)
    if rc != 0:
        raise RuntimeError("propagation failed")
    return out[0]


def collinear_points(mu):
    """x of L1, L2 from their quintics in gamma (Szebehely)."""
    def root(coeffs):
        r = np.roots(coeffs)
        return [v.real for v in r if abs(v.imag) < 1e-12 and 0.0 < v.real < 1.0][0]
    g1 = root([1, -(3 - mu), 3 - 2 * mu, -mu, 2 * mu, -mu])
    g2 = root([1, 3 - mu, 3 - 2 * mu, -mu, -2 * mu, -mu])
    return 1 - mu - g1, 1 - mu + g2


def first_crossing(mu, s0, t_min=0.05, t_max=20.0, dt=0.01):
    """Time of the first y = 0 crossing after t_min (bracket on a grid, then bisect)."""
    grid = np.arange(t_min, t_max, dt)
    out, _, _, rc = propagate_dopri5(mu, s0, grid, **TOL)
    if rc != 0:
        raise RuntimeError("propagation failed")
    y = out[:, 1]
    idx = np.nonzero(np.sign(y[1:]) != np.sign(y[:-1]))[0]
    if idx.size == 0:
        raise RuntimeError("no crossing")
    a, b = grid[idx[0]], grid[idx[0] + 1]
    ya = y[idx[0]]
    for _ in range(60):
        c = 0.5 * (a + b)
        yc = state_at(mu, s0, c)[1]
        if np.sign(yc) == np.sign(ya):
            a, ya = c, yc
        else:
            b = c
    return 0.5 * (a + b)


def correct(mu, s0, thalf, free, tol=1e-13, max_iter=30, eps=1e-7):
    """Newton on the free initial components (indices into the state) plus the half
    period, zeroing y, vx (and vz when three components are free)."""
    s0 = np.array(s0, dtype=float)
    cons = [1, 3] if len(free) == 1 else [1, 3, 5]
    for _ in range(max_iter):
        sf = state_at(mu, s0, thalf)
        F = sf[cons]
        if np.max(np.abs(F)) < tol:
            return s0, thalf
        Jm = np.empty((len(cons), len(free) + 1))
        for j, i in enumerate(free):
            sp, sm = s0.copy(), s0.copy()
            sp[i] += eps
            sm[i] -= eps
            Jm[:, j] = (state_at(mu, sp, thalf)[cons] - state_at(mu, sm, thalf)[cons]) / (2 * eps)
        Jm[:, -1] = rhs(mu, sf)[cons]
        d = np.linalg.solve(Jm, -F)
        for j, i in enumerate(free):
            s0[i] += d[j]
        thalf += d[-1]
    sf = state_at(mu, s0, thalf)
    if np.max(np.abs(sf[cons])) > 1e-11:
        raise RuntimeError("corrector did not converge")
    return s0, thalf


def lyapunov_l1(mu, ax=0.02):
    """Planar Lyapunov orbit about L1 starting ax inside the libration point, with the
    linearised in-plane mode as the first guess."""
    xl1, _ = collinear_points(mu)
    r1, r2 = abs(xl1 + mu), abs(xl1 - 1 + mu)
    c2 = (1 - mu) / r1 ** 3 + mu / r2 ** 3
    w = np.sqrt((2 - c2 + np.sqrt(9 * c2 * c2 - 8 * c2)) / 2)
    vy0 = (w * w + 1 + 2 * c2) * ax / 2
    s0 = np.array([xl1 - ax, 0, 0, 0, vy0, 0])
    return correct(mu, s0, np.pi / w, free=[4])


def halo_l2_north(mu, z0=0.05, start=None, step=0.01):
    """Northern L2 halo with z0 at the x-axis crossing, by natural-parameter
    continuation in z0 from a known member (default: the z-mirror of the paper's
    Table 2 deputy, x0 = 1.140135389, z0 = -0.163176653574390, vy0 = -0.223383154)."""
    if start is None:
        start = np.array([1.140135389, 0, 0.163176653574390, 0, -0.223383154, 0])
    s0 = np.array(start, dtype=float)
    thalf = first_crossing(mu, s0)
    s0, thalf = correct(mu, s0, thalf, free=[0, 4])
    z = s0[2]
    while abs(z - z0) > 1e-15:
        z = max(z0, z - step) if z > z0 else min(z0, z + step)
        s0 = s0.copy()
        s0[2] = z
        s0, thalf = correct(mu, s0, thalf, free=[0, 4])
    return s0, thalf


def dro(mu, ax=0.2):
    """Distant retrograde orbit crossing the x-axis ax beyond the Moon, moving with
    vy < 0 there: scan vy for a sign change of vx at the first crossing, then Newton."""
    x0 = 1 - mu + ax
    vys = np.linspace(-0.9, -0.05, 35)
    prev = None
    for vy in vys:
        s0 = np.array([x0, 0, 0, 0, vy, 0])
        try:
            th = first_crossing(mu, s0)
        except RuntimeError:
            prev = None
            continue
        vx = state_at(mu, s0, th)[3]
        if prev is not None and np.sign(vx) != np.sign(prev[1]):
            s0 = np.array([x0, 0, 0, 0, 0.5 * (vy + prev[0]), 0])
            return correct(mu, s0, first_crossing(mu, s0), free=[4])
        prev = (vy, vx)
    raise RuntimeError("no DRO found")
