"""Plain FP64 CPU oracle for PSO initial orbit determination in the CR3BP.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's CPU
baseline leg are the only callers.  The product library never imports this package,
and this package imports nothing from the product.

The arithmetic lives in ``iod_oracle.c`` (compiled with ``-O2 -ffp-contract=off``,
single-threaded); this module only marshals numpy arrays through ctypes.
Parity status: every function is pinned by the ``-m "not gpu"`` tests; the Philox
generator is pinned by published known-answer vectors.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "iod_oracle.c")
_HDR = os.path.join(_HERE, "iod_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

RK4, DOPRI5 = 0, 1
LM_RESIDUALS, LM_EPOCH_CHI2 = 0, 1
COST_CHI2, COST_QUARTIC = 0, 1
GBEST_SYNC, GBEST_LAGGED = 0, 1
OBJ_IOD, OBJ_SPHERE = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library beside its source."""
    stale = (not os.path.exists(_LIB) or
             os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                        "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


class DopriOpts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("atol", C.c_double), ("h0", C.c_double),
                ("max_steps", C.c_longlong)]


class Problem_(C.Structure):
    _fields_ = [("mu", C.c_double), ("n_obs", C.c_int),
                ("t", C.POINTER(C.c_double)), ("ra", C.POINTER(C.c_double)),
                ("dec", C.POINTER(C.c_double)), ("rng", C.POINTER(C.c_double)),
                ("sigma_ra", C.c_double), ("sigma_dec", C.c_double), ("sigma_rng", C.c_double),
                ("rc", C.POINTER(C.c_double)), ("integrator", C.c_int), ("dt", C.c_double),
                ("dp", DopriOpts), ("cost_form", C.c_int), ("use_range", C.c_int),
                ("dynamics", C.c_int), ("ecc", C.c_double), ("f0", C.c_double)]


class Pso_(C.Structure):
    _fields_ = [("objective", C.c_int), ("ctx", C.c_void_p),
                ("lo", C.c_double * 6), ("hi", C.c_double * 6),
                ("w", C.c_double), ("c1", C.c_double), ("c2", C.c_double),
                ("vmax_frac", C.c_double), ("gbest_order", C.c_int), ("seed", C.c_uint64),
                ("tol_tau", C.c_double), ("tol_window", C.c_int), ("constriction", C.c_int),
                ("init_grid", C.c_int), ("init_cone", C.c_int), ("cone_rho_min", C.c_double),
                ("cone_rho_max", C.c_double), ("cone_sigmas", C.c_double),
                ("velocity_init", C.c_int), ("per_dim_random", C.c_int)]


class Swarm_(C.Structure):
    _fields_ = [("m", C.c_int), ("x", C.POINTER(C.c_double)), ("v", C.POINTER(C.c_double)),
                ("p", C.POINTER(C.c_double)), ("pJ", C.POINTER(C.c_double)),
                ("J", C.POINTER(C.c_double)), ("g", C.c_double * 6), ("gJ", C.c_double),
                ("gidx", C.c_int), ("steps", C.c_longlong), ("iters_done", C.c_int)]


_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)
_LL = C.POINTER(C.c_longlong)
_U32 = C.POINTER(C.c_uint32)


def lib() -> C.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            sig = {
                "ora_rhs": (None, [C.c_double, _D, _D]),
                "ora_jacobi": (C.c_double, [C.c_double, _D]),
                "ora_rk4_grid": (C.c_int, [C.c_int, _D, C.c_double, _I, _D]),
                "ora_rk4_step": (None, [C.c_double, C.c_double, _D]),
                "ora_propagate_rk4": (C.c_int, [C.c_double, _D, C.c_int, _D, C.c_double, _D, _LL]),
                "ora_dopri5_attempt": (C.c_double, [C.c_double, C.c_double, _D, _D, _D, _D,
                                                    C.c_double, C.c_double]),
                "ora_dopri5_dense": (None, [C.c_double, _D, _D, C.c_double, _D]),
                "ora_propagate_dopri5": (C.c_int, [C.c_double, _D, C.c_int, _D,
                                                   C.POINTER(DopriOpts), _D, _LL, _LL]),
                "ora_angles": (None, [_D, _D, _D, _D]),
                "ora_propagate": (C.c_int, [C.POINTER(Problem_), _D, _D, _LL]),
                "ora_cost_from_states": (C.c_double, [C.POINTER(Problem_), _D]),
                "ora_cost": (C.c_double, [C.POINTER(Problem_), _D, _LL]),
                "ora_cost_sphere": (C.c_double, [_D, _D]),
                "ora_philox4x32_10": (None, [_U32, _U32, _U32]),
                "ora_u01": (C.c_double, [C.c_uint32, C.c_uint32]),
                "ora_pso_init": (C.c_int, [C.POINTER(Pso_), C.POINTER(Swarm_)]),
                "ora_pso_iterate": (C.c_int, [C.POINTER(Pso_), C.POINTER(Swarm_), C.c_int]),
                "ora_pso_run": (C.c_int, [C.POINTER(Pso_), C.POINTER(Swarm_), C.c_int, _D, _I]),
                "ora_bounds_from_chief": (None, [_D, C.c_double, C.c_double, C.c_double,
                                                 C.c_double, _D, _D]),
                "ora_simulate_obs": (C.c_int, [C.c_double, _D, _D, C.c_int, _D,
                                               C.POINTER(DopriOpts), _D, _D, _D, _D, _D]),
                "ora_lm_residuals": (C.c_int, [C.POINTER(Problem_), _D, C.c_int, _D]),
                "ora_constriction": (C.c_double, [C.c_double, C.c_double]),
                "ora_rhs_er3bp": (None, [C.c_double, C.c_double, C.c_double, _D, _D]),
                "ora_er3bp_anomaly": (C.c_double, [C.c_double, C.c_double, C.c_double]),
                "ora_simulate_obs_er3bp": (C.c_int, [C.c_double, C.c_double, C.c_double, _D, _D,
                                                     C.c_int, _D, C.POINTER(DopriOpts), _D, _D,
                                                     _D, _D, _D]),
                "ora_lm_refine": (C.c_int, [C.POINTER(Problem_), _D, C.c_int, C.c_int, _D, _D, _I]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _dp(a) -> "C.POINTER(C.c_double)":
    return a.ctypes.data_as(_D)


def _f64(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


# ---------------------------------------------------------------- dynamics
def rhs(mu: float, s) -> np.ndarray:
    s = _f64(s, (6,))
    out = np.empty(6)
    lib().ora_rhs(mu, _dp(s), _dp(out))
    return out


def jacobi(mu: float, s) -> float:
    return lib().ora_jacobi(mu, _dp(_f64(s, (6,))))


def rk4_grid(t, dt: float):
    t = _f64(t)
    ns = np.empty(t.size, dtype=np.int32)
    h = np.empty(t.size)
    rc = lib().ora_rk4_grid(t.size, _dp(t), dt, ns.ctypes.data_as(_I), _dp(h))
    if rc != 0:
        raise ValueError("invalid time grid")
    return ns, h


def rk4_steps(mu: float, s0, h: float, n: int) -> np.ndarray:
    s = _f64(s0, (6,)).copy()
    L = lib()
    for _ in range(int(n)):
        L.ora_rk4_step(mu, h, _dp(s))
    return s


def propagate_rk4(mu: float, s0, t, dt: float):
    t = _f64(t)
    out = np.empty((t.size, 6))
    steps = C.c_longlong(0)
    rc = lib().ora_propagate_rk4(mu, _dp(_f64(s0, (6,))), t.size, _dp(t), dt, _dp(out),
                                 C.byref(steps))
    return out, int(steps.value), rc


def dopri_opts(rtol=1e-12, atol=1e-12, h0=1e-3, max_steps=10_000_000) -> DopriOpts:
    return DopriOpts(rtol, atol, h0, max_steps)


def propagate_dopri5(mu: float, s0, t, rtol=1e-12, atol=1e-12, h0=1e-3, max_steps=10_000_000):
    t = _f64(t)
    out = np.empty((t.size, 6))
    acc, rej = C.c_longlong(0), C.c_longlong(0)
    o = dopri_opts(rtol, atol, h0, max_steps)
    rc = lib().ora_propagate_dopri5(mu, _dp(_f64(s0, (6,))), t.size, _dp(t), C.byref(o),
                                    _dp(out), C.byref(acc), C.byref(rej))
    return out, int(acc.value), int(rej.value), rc


def dopri5_attempt(mu: float, h: float, s, rtol=1e-12, atol=1e-12):
    """One DOPRI5 attempt from s; returns (s1, k[7][6], err)."""
    s = _f64(s, (6,))
    k1 = rhs(mu, s)
    s1 = np.empty(6)
    k = np.empty((7, 6))
    err = lib().ora_dopri5_attempt(mu, h, _dp(s), _dp(k1), _dp(s1), _dp(k), rtol, atol)
    return s1, k, err


def dopri5_dense(h: float, s, k, theta: float) -> np.ndarray:
    s = _f64(s, (6,))
    k = _f64(k, (7, 6))
    out = np.empty(6)
    lib().ora_dopri5_dense(h, _dp(s), _dp(k), theta, _dp(out))
    return out


# ---------------------------------------------------------------- measurement / cost
def angles(rho):
    rho = _f64(rho, (3,))
    a, b, r = C.c_double(), C.c_double(), C.c_double()
    lib().ora_angles(_dp(rho), C.byref(a), C.byref(b), C.byref(r))
    return a.value, b.value, r.value


class Problem:
    """An IOD problem as the oracle sees it.  The chief trajectory r_c(t_k) is computed
    here by the oracle's own integrator on the problem's grid."""

    def __init__(self, mu, chief, t, ra, dec, sigma_ra, sigma_dec, integrator=RK4, dt=1e-3,
                 rtol=1e-12, atol=1e-12, h0=1e-3, cost_form=COST_CHI2, rng=None,
                 sigma_rng=1.0, use_range=False, max_steps=10_000_000, dynamics=0, ecc=0.0,
                 f0=0.0):
        self.mu = float(mu)
        self.chief = _f64(chief, (6,)).copy()
        self.t = _f64(t).copy()
        self.ra = _f64(ra).copy()
        self.dec = _f64(dec).copy()
        self.rng = _f64(rng).copy() if rng is not None else np.zeros_like(self.t)
        self.integrator = integrator
        self.opts = dopri_opts(rtol, atol, h0, max_steps)
        self.rc = np.zeros((self.t.size, 3))
        self._s = Problem_(self.mu, self.t.size, _dp(self.t), _dp(self.ra), _dp(self.dec),
                           _dp(self.rng), float(sigma_ra), float(sigma_dec), float(sigma_rng),
                           _dp(self.rc), integrator, float(dt), self.opts, cost_form,
                           int(bool(use_range)), int(dynamics), float(ecc), float(f0))
        states, _, rc = self.propagate(self.chief)
        if rc != 0:
            raise ValueError("chief propagation failed")
        self.rc[:] = states[:, :3]

    @property
    def n_obs(self) -> int:
        return self.t.size

    def propagate(self, s0):
        out = np.empty((self.t.size, 6))
        steps = C.c_longlong(0)
        rc = lib().ora_propagate(C.byref(self._s), _dp(_f64(s0, (6,))), _dp(out), C.byref(steps))
        return out, int(steps.value), rc

    def cost(self, x) -> float:
        steps = C.c_longlong(0)
        return lib().ora_cost(C.byref(self._s), _dp(_f64(x, (6,))), C.byref(steps))

    def costs(self, X) -> np.ndarray:
        X = _f64(X).reshape(-1, 6)
        return np.array([self.cost(X[i]) for i in range(X.shape[0])])

    def cost_from_states(self, states) -> float:
        return lib().ora_cost_from_states(C.byref(self._s), _dp(_f64(states, (self.t.size, 6))))

    def lm_residuals(self, x, form=0) -> np.ndarray:
        r = np.empty(2 * self.t.size if form == 0 else self.t.size)
        lib().ora_lm_residuals(C.byref(self._s), _dp(_f64(x, (6,))), form, _dp(r))
        return r

    def lm_refine(self, x0, max_iters=30, form=0):
        """Levenberg-Marquardt from x0: (state, cost, iterations, status)."""
        out = np.empty(6)
        cost = C.c_double()
        it = C.c_int()
        rc = lib().ora_lm_refine(C.byref(self._s), _dp(_f64(x0, (6,))), max_iters, form, _dp(out),
                                 C.byref(cost), C.byref(it))
        return out, cost.value, it.value, rc

    def steps_per_eval(self, x) -> int:
        steps = C.c_longlong(0)
        lib().ora_cost(C.byref(self._s), _dp(_f64(x, (6,))), C.byref(steps))
        return int(steps.value)


def cost_sphere(center, x) -> float:
    return lib().ora_cost_sphere(_dp(_f64(center, (6,))), _dp(_f64(x, (6,))))


# ---------------------------------------------------------------- Philox
def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(4)
    k = np.ascontiguousarray(key, dtype=np.uint32).reshape(2)
    out = np.empty(4, dtype=np.uint32)
    lib().ora_philox4x32_10(c.ctypes.data_as(_U32), k.ctypes.data_as(_U32),
                            out.ctypes.data_as(_U32))
    return out


ER3BP = 1


def rhs_er3bp(mu, e, f, s):
    ds = np.empty(6)
    lib().ora_rhs_er3bp(mu, e, f, _dp(_f64(s, (6,))), _dp(ds))
    return ds


def er3bp_anomaly(e, f0, tau) -> float:
    return lib().ora_er3bp_anomaly(float(e), float(f0), float(tau))


def constriction(c1: float, c2: float) -> float:
    return lib().ora_constriction(c1, c2)


def u01(a: int, b: int) -> float:
    return lib().ora_u01(a & 0xFFFFFFFF, b & 0xFFFFFFFF)


# ---------------------------------------------------------------- swarm
class Swarm:
    """Swarm state as numpy AoS arrays ([m][6] rows) shared with the C oracle."""

    def __init__(self, m: int):
        self.m = int(m)
        self.x = np.zeros((m, 6))
        self.v = np.zeros((m, 6))
        self.p = np.zeros((m, 6))
        self.pJ = np.zeros(m)
        self.J = np.zeros(m)
        self._s = Swarm_(self.m, _dp(self.x), _dp(self.v), _dp(self.p), _dp(self.pJ),
                         _dp(self.J), (C.c_double * 6)(), 0.0, 0, 0, 0)

    @property
    def g(self) -> np.ndarray:
        return np.array(self._s.g[:])

    @g.setter
    def g(self, val):
        for d in range(6):
            self._s.g[d] = float(val[d])

    gJ = property(lambda s: s._s.gJ, lambda s, v: setattr(s._s, "gJ", float(v)))
    gidx = property(lambda s: s._s.gidx, lambda s, v: setattr(s._s, "gidx", int(v)))
    steps = property(lambda s: s._s.steps, lambda s, v: setattr(s._s, "steps", int(v)))
    iters_done = property(lambda s: s._s.iters_done)

    def copy(self) -> "Swarm":
        o = Swarm(self.m)
        for a in ("x", "v", "p", "pJ", "J"):
            getattr(o, a)[:] = getattr(self, a)
        o.g, o.gJ, o.gidx, o.steps = self.g, self.gJ, self.gidx, self.steps
        return o


class Pso:
    """Algorithm 1 settings.  ``objective`` is a :class:`Problem` (IOD cost) or a
    6-vector (the sphere test objective centred there)."""

    def __init__(self, objective, lo, hi, w=0.7, c1=1.5, c2=1.5, seed=0,
                 gbest_order=GBEST_SYNC, vmax_frac=1.0, tol_tau=0.0, tol_window=10,
                 constriction=False, init_grid=False, init_cone=False, cone_rho_min=0.0,
                 cone_rho_max=0.0, cone_sigmas=3.0, velocity_init=0, per_dim_random=False):
        if isinstance(objective, Problem):
            self._keep = objective
            kind, ctx = OBJ_IOD, C.cast(C.pointer(objective._s), C.c_void_p)
        else:
            self._keep = _f64(objective, (6,)).copy()
            kind, ctx = OBJ_SPHERE, C.c_void_p(self._keep.ctypes.data)
        lo = _f64(lo, (6,))
        hi = _f64(hi, (6,))
        self._s = Pso_(kind, ctx, (C.c_double * 6)(*lo), (C.c_double * 6)(*hi), w, c1, c2,
                       vmax_frac, gbest_order, seed & 0xFFFFFFFFFFFFFFFF, tol_tau, tol_window,
                       int(bool(constriction)), int(bool(init_grid)), int(bool(init_cone)),
                       cone_rho_min, cone_rho_max, cone_sigmas, int(velocity_init),
                       int(bool(per_dim_random)))

    def init(self, W: Swarm):
        rc = lib().ora_pso_init(C.byref(self._s), C.byref(W._s))
        if rc != 0:
            raise RuntimeError(f"ora_pso_init failed: {rc}")

    def iterate(self, W: Swarm, n: int):
        rc = lib().ora_pso_iterate(C.byref(self._s), C.byref(W._s), n)
        if rc != 0:
            raise RuntimeError(f"ora_pso_iterate failed: {rc}")

    def run(self, m: int, iters: int):
        W = Swarm(m)
        gJ = np.empty(iters + 1)
        gi = np.empty(iters + 1, dtype=np.int32)
        rc = lib().ora_pso_run(C.byref(self._s), C.byref(W._s), iters, _dp(gJ),
                               gi.ctypes.data_as(_I))
        if rc != 0:
            raise RuntimeError(f"ora_pso_run failed: {rc}")
        n = W.iters_done + 1
        return W, gJ[:n], gi[:n]


# ---------------------------------------------------------------- scenario helpers
def bounds_from_chief(chief, r_max_km, v_max_ms, L_km, TU_s):
    lo = np.empty(6)
    hi = np.empty(6)
    lib().ora_bounds_from_chief(_dp(_f64(chief, (6,))), r_max_km, v_max_ms, L_km, TU_s,
                                _dp(lo), _dp(hi))
    return lo, hi


def simulate_obs(mu, chief0, deputy0, t, noise=None, rtol=1e-13, atol=1e-13, h0=1e-3,
                 ecc=None, f0=0.0):
    """Observed (ra, dec, range) of the deputy from the chief, both propagated with
    DOPRI5 at the given tolerance, plus ``noise`` ([n][2] radians) if given.  With
    ``ecc`` set, the dynamics are the ER3BP (eccentricity ecc, true anomaly f0 at t = 0)."""
    t = _f64(t)
    n = t.size
    ra, dec, rng = np.empty(n), np.empty(n), np.empty(n)
    rc = np.empty((n, 3))
    o = dopri_opts(rtol, atol, h0)
    nz = _f64(noise, (n, 2)) if noise is not None else None
    if ecc is None:
        r = lib().ora_simulate_obs(mu, _dp(_f64(chief0, (6,))), _dp(_f64(deputy0, (6,))), n,
                                   _dp(t), C.byref(o), _dp(nz) if nz is not None else None,
                                   _dp(ra), _dp(dec), _dp(rng), _dp(rc))
    else:
        r = lib().ora_simulate_obs_er3bp(mu, float(ecc), float(f0), _dp(_f64(chief0, (6,))),
                                         _dp(_f64(deputy0, (6,))), n, _dp(t), C.byref(o),
                                         _dp(nz) if nz is not None else None,
                                         _dp(ra), _dp(dec), _dp(rng), _dp(rc))
    if r != 0:
        raise RuntimeError("observation simulation failed")
    return ra, dec, rng, rc
