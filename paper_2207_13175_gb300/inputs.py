"""Seeded synthetic inputs for PSO initial orbit determination workloads.

This module holds none of the method's arithmetic: no propagation, no measurement
model, no cost and no swarm.  It draws the scenario's free quantities (the truth
deputy's offset from the chief, the observation noise, the observation times) with
numpy's seeded generator and names the workload shapes.  Both the CUDA library's
tests and the oracle's tests take their inputs from here; each side then builds its
own bounds, chief trajectory and observations.

Shapes follow the paper's workloads (Results section and Tables 2-3: 7-day arcs,
10-35 equally spaced angle measurements, halo/axial L2 chiefs, position/velocity
boxes about a known state) and the two standard sizes used here:

* ``tiny``: chief (0.85, 0, 0.17, 0, 0.26, 0); deputy offset uniform by volume in a
  10-100 km shell with a 0-1 m/s velocity offset in a random direction; 20 angle pairs
  over 1 day with 1 arcsec noise; RK4 dt 1e-3 TU; 256 particles, 100 iterations;
  box chief +-100 km / +-1 m/s per axis.
* ``paper_scale``: one of three self-corrected periodic chiefs (L1 planar Lyapunov
  Ax = 0.02, L2 northern halo z0 = 0.05, DRO x-amplitude 0.2); offsets 1-500 km and
  0-5 m/s; 200 angle pairs over 7 days with 1 arcsec noise; RK4 dt 5e-4 TU or DOPRI5
  rtol 1e-12; 65,536 particles, 500 iterations; box chief +-500 km / +-5 m/s.
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field, replace

import numpy as np

MU = 0.01215058560962404          # Earth-Moon mass parameter
L_KM = 384400.0                   # length unit: Earth-Moon distance
TU_S = 375190.0                   # time unit
DAY_TU = 86400.0 / TU_S
ARCSEC = math.pi / 648000.0

_ORBITS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "chief_orbits.json")


def chief_orbits() -> dict:
    """Initial states (nondimensional, at a perpendicular x-axis crossing) and periods
    of the three periodic chief orbits, as written by the differential corrector."""
    with open(_ORBITS) as f:
        return json.load(f)["orbits"]


@dataclass
class Scenario:
    name: str
    chief: np.ndarray                 # (6,) chief state at t = 0 (known)
    deputy: np.ndarray                # (6,) truth deputy state at t = 0
    t: np.ndarray                     # (K,) observation times, TU
    noise: np.ndarray                 # (K, 2) angle noise to add, radians
    sigma: tuple = (ARCSEC, ARCSEC)   # (sigma_ra, sigma_dec), radians
    r_max_km: float = 100.0           # box half-width per position axis
    v_max_ms: float = 1.0             # box half-width per velocity axis
    integrator: str = "rk4"           # "rk4" | "dopri5"
    dt: float = 1e-3
    rtol: float = 1e-12
    atol: float = 1e-12
    h0: float = 1e-3
    m: int = 256
    iters: int = 100
    w: float = 0.7
    c1: float = 1.5
    c2: float = 1.5
    seed: int = 0
    mu: float = MU
    meta: dict = field(default_factory=dict)

    @property
    def n_obs(self) -> int:
        return int(self.t.size)

    def with_(self, **kw) -> "Scenario":
        return replace(self, **kw)


def _unit_vector(rng: np.random.Generator) -> np.ndarray:
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def truth_offset(rng: np.random.Generator, r_min_km, r_max_km, v_min_ms, v_max_ms):
    """Offset of the deputy from the chief: a direction uniform on the sphere with the
    radius uniform by volume in the shell, and an independent velocity offset with a
    uniform direction and a uniform magnitude.  Returned nondimensional."""
    u = rng.uniform()
    r_km = (r_min_km ** 3 + u * (r_max_km ** 3 - r_min_km ** 3)) ** (1.0 / 3.0)
    dr = _unit_vector(rng) * r_km / L_KM
    dv_ms = rng.uniform(v_min_ms, v_max_ms)
    dv = _unit_vector(rng) * (dv_ms / 1000.0) / (L_KM / TU_S)
    return np.concatenate([dr, dv]), r_km, dv_ms


def tiny(seed: int = 0, noise: bool = True) -> Scenario:
    rng = np.random.default_rng(seed)
    chief = np.array([0.85, 0.0, 0.17, 0.0, 0.26, 0.0])
    off, r_km, dv_ms = truth_offset(rng, 10.0, 100.0, 0.0, 1.0)
    K = 20
    t = np.linspace(0.0, DAY_TU, K)
    nz = rng.normal(0.0, ARCSEC, size=(K, 2)) if noise else np.zeros((K, 2))
    return Scenario(name=f"tiny{'' if noise else '-noisefree'}-s{seed}", chief=chief,
                    deputy=chief + off, t=t, noise=nz, r_max_km=100.0, v_max_ms=1.0,
                    integrator="rk4", dt=1e-3, m=256, iters=100, seed=seed,
                    meta={"offset_km": r_km, "offset_ms": dv_ms})


# The paper's printed chief states (Tables 2 and 3, nondimensional): the 7.15-day L2
# halo of scenario 1, which passes 0.0118 LU from the Moon, and the 19.1-day L2 axial
# orbit of scenario 2; and its L2 southern halo deputy.
PAPER_CHIEFS = {
    1: np.array([1.029726968, 0.0, -1.869397163946e-01, -5.585615805585e-14,
                 -0.119441863, -9.803996218373e-13]),
    2: np.array([1.21996614837886e00, 0.0, -2.49454877925228e-16,
                 1.10859609358602e-15, -4.27475884185211e-01, 4.09809301627323e-03]),
}
PAPER_DEPUTY = np.array([1.140135389, 0.0, -1.63176653574390e-01, 6.13321115086310e-15,
                         -0.223383154, 1.78644826151404e-15])


def paper_scale(orbit: str = "halo", seed: int = 0, integrator: str = "rk4",
                noise: bool = True) -> Scenario:
    """The paper-scale workload: 65,536 particles, 500 iterations, 200 angle pairs over
    7 days, a deputy 1-500 km / 0-5 m/s from the chief.  orbit: one of the corrected
    chief orbits ("lyapunov", "halo", "dro") or "paper-s1", the paper's scenario-1
    chief (its close lunar passage exercises the mixed form's near-Moon FP64 steps)."""
    if orbit == "paper-s1":
        chief = PAPER_CHIEFS[1].copy()
    else:
        chief = np.array(chief_orbits()[orbit]["state"], dtype=float)
    rng = np.random.default_rng(1000 + seed)
    off, r_km, dv_ms = truth_offset(rng, 1.0, 500.0, 0.0, 5.0)
    K = 200
    t = np.linspace(0.0, 7.0 * DAY_TU, K)
    nz = rng.normal(0.0, ARCSEC, size=(K, 2)) if noise else np.zeros((K, 2))
    return Scenario(name=f"paper-scale-{orbit}-{integrator}{'' if noise else '-noisefree'}-s{seed}",
                    chief=chief, deputy=chief + off, t=t, noise=nz, r_max_km=500.0,
                    v_max_ms=5.0, integrator=integrator, dt=5e-4, rtol=1e-12, atol=1e-12,
                    m=65536, iters=500, seed=seed,
                    meta={"orbit": orbit, "offset_km": r_km, "offset_ms": dv_ms})


def paper_table(scenario: int = 1, noise: bool = False, seed: int = 0) -> Scenario:
    """The paper's printed geometries (Tables 2 and 3): L2 southern halo deputy, chief on
    the 7.15-day L2 halo (scenario 1, 35 measurements) or the 19.1-day L2 axial orbit
    (scenario 2, 10 measurements), 7-day arc, box +-250 km / +-0.1 km/s about the truth
    deputy (the paper seeds about the truth, not the chief)."""
    deputy = PAPER_DEPUTY.copy()
    chief = PAPER_CHIEFS[scenario].copy()
    K = 35 if scenario == 1 else 10
    rng = np.random.default_rng(2000 + seed)
    t = np.linspace(0.0, 7.0 * DAY_TU, K)
    nz = rng.normal(0.0, ARCSEC, size=(K, 2)) if noise else np.zeros((K, 2))
    return Scenario(name=f"paper-table-{scenario}", chief=chief, deputy=deputy, t=t, noise=nz,
                    r_max_km=250.0, v_max_ms=100.0, integrator="rk4", dt=5e-4, m=4096,
                    iters=200, seed=seed, meta={"box_about": "deputy"})


def particles_in_box(lo, hi, m: int, seed: int = 0) -> np.ndarray:
    """m candidate states uniform in the box [lo, hi] (numpy's generator; used to feed
    both sides the same particle set in evaluation tests).  Shape (m, 6)."""
    rng = np.random.default_rng(seed)
    lo = np.asarray(lo, dtype=float)
    hi = np.asarray(hi, dtype=float)
    return lo + rng.uniform(size=(m, 6)) * (hi - lo)


def near_truth(deputy, m: int, scale_km: float, scale_ms: float, seed: int = 0) -> np.ndarray:
    """m states scattered about the truth by Gaussian offsets of the given scales."""
    rng = np.random.default_rng(seed)
    off = np.empty((m, 6))
    off[:, :3] = rng.normal(size=(m, 3)) * scale_km / L_KM
    off[:, 3:] = rng.normal(size=(m, 3)) * (scale_ms / 1000.0) / (L_KM / TU_S)
    return np.asarray(deputy, dtype=float)[None, :] + off


def batched_instance(rng: np.random.Generator, index: int = 0, iters_range=(100, 500),
                     swarm_sizes=(1024, 4096, 16384), noise: bool = True) -> Scenario:
    """One instance of the batched workload: a chief from the three corrected families at
    a random phase of its period (the phase is returned in meta; the caller propagates
    the chief's initial condition by it), 10-400 angle pairs over 1-7 days, a swarm of
    1,024 / 4,096 / 16,384 particles and 100-500 iterations.  With noise=False the
    angles carry no noise; every other draw is the same (the generator advances alike)."""
    names = ("halo", "dro", "lyapunov")
    name = names[int(rng.integers(0, 3))]
    orb = chief_orbits()[name]
    phase = float(rng.uniform(0.0, orb["period_tu"]))
    K = int(rng.integers(10, 401))
    T = float(rng.uniform(1.0, 7.0)) * DAY_TU
    off, r_km, dv_ms = truth_offset(rng, 1.0, 500.0, 0.0, 5.0)
    nz = rng.normal(0.0, ARCSEC, (K, 2))
    return Scenario(name=f"batched-{index}-{name}{'' if noise else '-noisefree'}",
                    chief=np.array(orb["state"], dtype=float),
                    deputy=off, t=np.linspace(0.0, T, K), noise=nz if noise else np.zeros((K, 2)),
                    r_max_km=500.0, v_max_ms=5.0, integrator="rk4", dt=5e-4,
                    m=int(rng.choice(swarm_sizes)), iters=int(rng.integers(iters_range[0], iters_range[1] + 1)),
                    seed=int(rng.integers(0, 2 ** 31)),
                    meta={"orbit": name, "phase_tu": phase, "offset_km": r_km, "offset_ms": dv_ms,
                          "deputy_is_offset": True})


def poisson_arrivals(rate_per_s: float, n: int, seed: int = 0) -> np.ndarray:
    """n arrival times (s) of a Poisson process with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))
