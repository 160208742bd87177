"""Python binding of the IOD library: argument marshalling over the C ABI.

PyTorch provides device memory (its caching allocator is installed as the library's
allocator hook) and streams (each problem runs on the caller's current stream).  All
arithmetic runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional

import numpy as np

from ._native import (ALLOC_FN, RELEASE_FN, BatchStats, IodError, Options, Request, Result,
                      check, lib)

RK4, DOPRI5 = 0, 1
CR3BP, ER3BP = 0, 1
FP64, MIXED = 0, 1
COST_CHI2, COST_QUARTIC = 0, 1
GBEST_SYNC, GBEST_LAGGED = 0, 1
SCHED_AUTO, SCHED_GRID, SCHED_BALANCED = 0, 1, 2

_D = C.POINTER(C.c_double)
_allocator_refs = None


def _f64(a, n=None) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_D)


def use_torch_allocator() -> None:
    """Route the library's device allocations through PyTorch's caching allocator."""
    global _allocator_refs
    if _allocator_refs is not None:
        return
    import torch

    def _alloc(nbytes, ctx):
        try:
            dev = torch.cuda.current_device()
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev,
                                                      torch.cuda.current_stream(dev))
        except Exception:
            return None

    def _release(ptr, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    refs = (ALLOC_FN(_alloc), RELEASE_FN(_release))
    check(lib().iod_set_allocator(refs[0], refs[1], None), "iod_set_allocator")
    _allocator_refs = refs


def options(**kw) -> Options:
    o = Options()
    check(lib().iod_options_default(C.byref(o)), "iod_options_default")
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def selftest_wait(limit_s: float, set_flag: bool = False):
    """The library's bounded device wait (iod_selftest_wait) on a flag that nothing sets
    (or that is set already): returns (gave_up, seconds waited)."""
    timed_out = C.c_int(-1)
    waited = C.c_double(0.0)
    check(lib().iod_selftest_wait(float(limit_s), int(bool(set_flag)), C.byref(timed_out),
                                  C.byref(waited)), "iod_selftest_wait")
    return bool(timed_out.value), waited.value


def selftest_fp64_issue(warps: int, lanes: int, n: int = 20000) -> float:
    """SM cycles per dependent FP64 FMA with `warps` warps in one block, `lanes` lanes of
    each active (iod_selftest_fp64_issue)."""
    out = C.c_double(0.0)
    check(lib().iod_selftest_fp64_issue(int(warps), int(lanes), int(n), C.byref(out)),
          "iod_selftest_fp64_issue")
    return out.value


def bounds_from_chief(chief, r_max_km, v_max_ms, L_km, TU_s) -> np.ndarray:
    out = np.empty(12)
    check(lib().iod_bounds_from_chief(_ptr(_f64(chief, 6)), r_max_km, v_max_ms, L_km, TU_s,
                                      _ptr(out)), "iod_bounds_from_chief")
    return out


def simulate_obs(mu, chief, deputy, t, noise=None, rtol=1e-13, atol=1e-13, h0=1e-3, ecc=None,
                 f0=0.0):
    """Observed (angles [K][2], ranges [K]) synthesised on the GPU; with ``ecc`` set, in
    the elliptic restricted problem (true anomaly f0 at t = 0)."""
    t = _f64(t)
    K = t.size
    ang = np.empty((K, 2))
    rng = np.empty(K)
    nz = _f64(noise, 2 * K) if noise is not None else None
    if ecc is None:
        check(lib().iod_simulate_obs(mu, _ptr(_f64(chief, 6)), _ptr(_f64(deputy, 6)), K, _ptr(t),
                                     rtol, atol, h0, _ptr(nz) if nz is not None else None,
                                     _ptr(ang), _ptr(rng)), "iod_simulate_obs")
    else:
        check(lib().iod_simulate_obs_er3bp(mu, float(ecc), float(f0), _ptr(_f64(chief, 6)),
                                           _ptr(_f64(deputy, 6)), K, _ptr(t), rtol, atol, h0,
                                           _ptr(nz) if nz is not None else None, _ptr(ang),
                                           _ptr(rng)), "iod_simulate_obs_er3bp")
    return ang, rng


class Problem:
    """One IOD problem on the current CUDA device and stream."""

    def __init__(self, mu, chief, t, angles, sigma, bounds, opts: Optional[Options] = None,
                 ranges=None, stream=None, torch_allocator: bool = True):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the IOD library needs a CUDA GPU")
        if torch_allocator:
            use_torch_allocator()
        self._h = C.c_void_p()
        t = _f64(t)
        K = t.size
        self.n_obs = K
        o = opts if opts is not None else options()
        self.opts = o
        args = [float(mu), _ptr(_f64(chief, 6)), K, _ptr(t), _ptr(_f64(angles, 2 * K))]
        if ranges is not None:
            args.append(_ptr(_f64(ranges, K)))
            fn, name = lib().iod_create_ranged, "iod_create_ranged"
        else:
            fn, name = lib().iod_create, "iod_create"
        args += [_ptr(_f64(sigma, 2)), _ptr(_f64(bounds, 12)), C.byref(o), C.byref(self._h)]
        check(fn(*args), name)
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        check(lib().iod_set_stream(self._h, C.c_void_p(s.cuda_stream)), "iod_set_stream")
        self.m = 0

    # ---------------------------------------------------------------- lifecycle
    def close(self) -> None:
        if self._h:
            lib().iod_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---------------------------------------------------------------- swarm
    def run(self, m: int, iters: int, w=0.7, c1=1.5, c2=1.5, seed=0) -> None:
        check(lib().iod_run(self._h, int(m), int(iters), float(w), float(c1), float(c2),
                            int(seed) & 0xFFFFFFFFFFFFFFFF), "iod_run")
        self.m = int(m)

    def continue_(self, iters: int) -> None:
        check(lib().iod_continue(self._h, int(iters)), "iod_continue")

    def result(self, trace: bool = True) -> dict:
        r = Result()
        cap = 0
        if trace:
            cap = 1 << 16
            tj = np.zeros(cap)
            ti = np.zeros(cap, dtype=np.int32)
            r.gcost_trace = tj.ctypes.data_as(_D)
            r.gidx_trace = ti.ctypes.data_as(C.POINTER(C.c_int))
            r.trace_capacity = cap
        check(lib().iod_result(self._h, C.byref(r)), "iod_result")
        out = {"state": np.array(r.state[:]), "cost": r.cost, "gbest_index": r.gbest_index,
               "iters_done": r.iters_done, "rk_steps": r.rk_steps, "fp64_steps": r.fp64_steps,
               "schedule": r.schedule}
        if trace:
            n = min(r.iters_done + 1, cap)
            out["gcost_trace"] = tj[:n].copy()
            out["gidx_trace"] = ti[:n].copy()
        return out

    def swarm_get(self) -> dict:
        m = self.m
        x, v, p = np.empty((6, m)), np.empty((6, m)), np.empty((6, m))
        pJ, J, g = np.empty(m), np.empty(m), np.empty(6)
        gJ = C.c_double()
        gi, it = C.c_int(), C.c_int()
        check(lib().iod_swarm_get(self._h, _ptr(x), _ptr(v), _ptr(p), _ptr(pJ), _ptr(J), _ptr(g),
                                  C.byref(gJ), C.byref(gi), C.byref(it)), "iod_swarm_get")
        return {"x": x, "v": v, "p": p, "pJ": pJ, "J": J, "g": g, "gJ": gJ.value,
                "gidx": gi.value, "iter": it.value}

    def swarm_set(self, x, v, p, pJ, g, gJ, gidx, iter_, w=0.7, c1=1.5, c2=1.5, seed=0) -> None:
        x = _f64(x).reshape(6, -1)
        m = x.shape[1]
        check(lib().iod_swarm_set(self._h, m, _ptr(x), _ptr(_f64(v, 6 * m)), _ptr(_f64(p, 6 * m)),
                                  _ptr(_f64(pJ, m)), _ptr(_f64(g, 6)), float(gJ), int(gidx),
                                  int(iter_), float(w), float(c1), float(c2),
                                  int(seed) & 0xFFFFFFFFFFFFFFFF), "iod_swarm_set")
        self.m = m

    def gbest_get(self):
        """(state, cost, whole-swarm index, last completed iteration) of the global best."""
        g = np.empty(6)
        gJ = C.c_double()
        gi, it = C.c_int(), C.c_int()
        check(lib().iod_gbest_get(self._h, _ptr(g), C.byref(gJ), C.byref(gi), C.byref(it)),
              "iod_gbest_get")
        return g, gJ.value, gi.value, it.value

    def gbest_set(self, g, gJ, gidx) -> None:
        """Replace the global best (the exchange between the shards of one swarm)."""
        check(lib().iod_gbest_set(self._h, _ptr(_f64(g, 6)), float(gJ), int(gidx)),
              "iod_gbest_set")

    def snapshot(self) -> bytes:
        n = C.c_size_t(0)
        check(lib().iod_snapshot(self._h, None, C.byref(n)), "iod_snapshot")
        buf = C.create_string_buffer(n.value)
        check(lib().iod_snapshot(self._h, buf, C.byref(n)), "iod_snapshot")
        return buf.raw[: n.value]

    def restore(self, blob: bytes) -> None:
        buf = C.create_string_buffer(blob, len(blob))
        check(lib().iod_restore(self._h, buf, len(blob)), "iod_restore")
        self.m = int(np.frombuffer(blob[12:16], dtype=np.int32)[0])

    # ---------------------------------------------------------------- debug entries
    def eval(self, x):
        """Costs of candidate states x: a CUDA float64 tensor [6][m] (or numpy [m][6])."""
        import torch
        X = self._dev_soa(x)
        m = X.shape[1]
        J = torch.empty(m, dtype=torch.float64, device=X.device)
        check(lib().iod_eval(self._h, C.c_void_p(X.data_ptr()), m, C.c_void_p(J.data_ptr())),
              "iod_eval")
        return J

    def propagate(self, x0):
        """States at every t_k: tensor [K][6][m]."""
        import torch
        X = self._dev_soa(x0)
        m = X.shape[1]
        out = torch.empty((self.n_obs, 6, m), dtype=torch.float64, device=X.device)
        check(lib().iod_propagate(self._h, C.c_void_p(X.data_ptr()), m,
                                  C.c_void_p(out.data_ptr())), "iod_propagate")
        return out

    def refine(self, x0, max_iters: int = 30, form: int = 0):
        """Levenberg-Marquardt from x0: (state, cost, iterations)."""
        out = np.empty(6)
        cost = C.c_double()
        it = C.c_int()
        check(lib().iod_refine(self._h, _ptr(_f64(x0, 6)), int(max_iters), int(form), _ptr(out),
                               C.byref(cost), C.byref(it)), "iod_refine")
        return out, cost.value, it.value

    def chief_positions(self) -> np.ndarray:
        rc = np.empty((self.n_obs, 3))
        check(lib().iod_chief_positions(self._h, _ptr(rc)), "iod_chief_positions")
        return rc

    @staticmethod
    def _dev_soa(x):
        import torch
        if isinstance(x, torch.Tensor):
            X = x.to(device="cuda", dtype=torch.float64)
            if X.dim() != 2 or X.shape[0] != 6:
                raise ValueError("expected a [6][m] tensor")
            return X.contiguous()
        a = np.asarray(x, dtype=np.float64).reshape(-1, 6)
        return torch.from_numpy(np.ascontiguousarray(a.T)).to("cuda")


class Batch:
    """Many resident problems advanced round by round (the batch/serving interface)."""

    EBUSY, ECANCELLED = -5, -6

    def __init__(self, opts: Optional[Options] = None, budget_bytes: int = 8 << 30,
                 max_resident: int = 1024, torch_allocator: bool = True):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the IOD library needs a CUDA GPU")
        if torch_allocator:
            use_torch_allocator()
        self._h = C.c_void_p()
        self.opts = opts if opts is not None else options()
        check(lib().iod_batch_create(C.byref(self.opts), int(budget_bytes), int(max_resident),
                                     C.byref(self._h)), "iod_batch_create")
        self._keep = {}

    def close(self):
        if self._h:
            lib().iod_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_block_sizes(self, max_swarm, block):
        n = len(block)
        ms = (C.c_int * n)(*[min(int(v), 2 ** 31 - 1) for v in max_swarm])
        bl = (C.c_int * n)(*[int(v) for v in block])
        check(lib().iod_batch_set_block_sizes(self._h, n, ms, bl), "iod_batch_set_block_sizes")

    def autotune(self, max_swarm, samples, candidates=(64, 128, 256), uniform=True):
        """Time candidate block sizes on one sample request per size class (tuples
        (mu, chief, t, angles, sigma, bounds, m, iters[, seed])) and set the fastest."""
        n = len(samples)
        keep = []
        reqs = (Request * n)()
        for k, smp in enumerate(samples):
            mu, chief, t, ang, sig, bnd, m, iters = smp[:8]
            seed = smp[8] if len(smp) > 8 else 0
            t = _f64(t)
            arrs = [_f64(chief, 6), t, _f64(ang, 2 * t.size), _f64(sig, 2), _f64(bnd, 12)]
            keep.append(arrs)
            reqs[k] = Request(float(mu), _ptr(arrs[0]), t.size, _ptr(arrs[1]), _ptr(arrs[2]),
                              _ptr(arrs[3]), _ptr(arrs[4]), int(m), int(iters), 0.7, 1.5, 1.5, int(seed))
        ms = (C.c_int * n)(*[min(int(v), 2 ** 31 - 1) for v in max_swarm])
        cand = (C.c_int * len(candidates))(*[int(v) for v in candidates])
        out = (C.c_int * n)()
        times = np.zeros(n * len(candidates))
        check(lib().iod_batch_autotune(self._h, n, ms, reqs, len(candidates), cand, int(uniform), out,
                                       _ptr(times)), "iod_batch_autotune")
        return list(out), times.reshape(n, len(candidates))

    @staticmethod
    def _requests(samples):
        n = len(samples)
        keep = []
        reqs = (Request * n)()
        for k, smp in enumerate(samples):
            mu, chief, t, ang, sig, bnd, m, iters = smp[:8]
            seed = smp[8] if len(smp) > 8 else 0
            t = _f64(t)
            arrs = [_f64(chief, 6), t, _f64(ang, 2 * t.size), _f64(sig, 2), _f64(bnd, 12)]
            keep.append(arrs)
            reqs[k] = Request(float(mu), _ptr(arrs[0]), t.size, _ptr(arrs[1]), _ptr(arrs[2]),
                              _ptr(arrs[3]), _ptr(arrs[4]), int(m), int(iters), 0.7, 1.5, 1.5, int(seed))
        return reqs, keep

    def set_step_sizes(self, max_swarm, dt):
        n = len(dt)
        ms = (C.c_int * n)(*[min(int(v), 2 ** 31 - 1) for v in max_swarm])
        d = _f64(dt)
        check(lib().iod_batch_set_step_sizes(self._h, n, ms, _ptr(d)), "iod_batch_set_step_sizes")

    def autotune_dt(self, max_swarm, samples, candidates, angle_budget, n_probe=64):
        """Largest RK4 step bound per size class whose lines of sight stay within
        angle_budget (rad) of a DOPRI5 reference on the sample's initial particles; sets
        it on the batch.  Returns (dt per class, errors [class][candidate])."""
        n = len(samples)
        reqs, keep = self._requests(samples)
        ms = (C.c_int * n)(*[min(int(v), 2 ** 31 - 1) for v in max_swarm])
        cand = _f64(candidates)
        out = np.zeros(n)
        err = np.zeros(n * cand.size)
        check(lib().iod_batch_autotune_dt(self._h, n, ms, reqs, cand.size, _ptr(cand), float(angle_budget),
                                          int(n_probe), _ptr(out), _ptr(err)), "iod_batch_autotune_dt")
        return out.tolist(), err.reshape(n, cand.size)

    def submit(self, mu, chief, t, angles, sigma, bounds, m, iters, w=0.7, c1=1.5, c2=1.5,
               seed=0) -> int:
        t = _f64(t)
        K = t.size
        arrs = [_f64(chief, 6), t, _f64(angles, 2 * K), _f64(sigma, 2), _f64(bounds, 12)]
        q = Request(float(mu), _ptr(arrs[0]), K, _ptr(arrs[1]), _ptr(arrs[2]), _ptr(arrs[3]),
                    _ptr(arrs[4]), int(m), int(iters), float(w), float(c1), float(c2),
                    int(seed) & 0xFFFFFFFFFFFFFFFF)
        tk = C.c_longlong()
        check(lib().iod_batch_submit(self._h, C.byref(q), C.byref(tk)), "iod_batch_submit")
        return tk.value

    def step(self, rounds: int) -> None:
        check(lib().iod_batch_step(self._h, int(rounds)), "iod_batch_step")

    def run(self, seconds: float = 0.0) -> None:
        """Persistent scheduling for up to `seconds` of device time (0: to completion)."""
        check(lib().iod_batch_run(self._h, float(seconds)), "iod_batch_run")

    def poll(self, ticket: int, trace: bool = False):
        """The result dict once finished, None while queued or running."""
        r = Result()
        if trace:
            cap = 1 << 16
            tj = np.zeros(cap)
            ti = np.zeros(cap, dtype=np.int32)
            r.gcost_trace = tj.ctypes.data_as(_D)
            r.gidx_trace = ti.ctypes.data_as(C.POINTER(C.c_int))
            r.trace_capacity = cap
        code = lib().iod_batch_poll(self._h, int(ticket), C.byref(r))
        if code == self.EBUSY:
            return None
        check(code, "iod_batch_poll")
        out = {"state": np.array(r.state[:]), "cost": r.cost, "gbest_index": r.gbest_index,
               "iters_done": r.iters_done, "rk_steps": r.rk_steps, "fp64_steps": r.fp64_steps,
               "pso_state": np.array(r.pso_state[:]), "pso_cost": r.pso_cost,
               "refine_iters": r.refine_iters, "fallback": r.fallback}
        if trace:
            n = min(r.iters_done + 1, cap)
            out["gcost_trace"] = tj[:n].copy()
            out["gidx_trace"] = ti[:n].copy()
        return out

    def times(self, ticket: int):
        a, b, c = C.c_double(), C.c_double(), C.c_double()
        check(lib().iod_batch_times(self._h, int(ticket), C.byref(a), C.byref(b), C.byref(c)),
              "iod_batch_times")
        return a.value, b.value, c.value

    def cancel(self, ticket: int) -> None:
        check(lib().iod_batch_cancel(self._h, int(ticket)), "iod_batch_cancel")

    def stats(self) -> dict:
        st = BatchStats()
        check(lib().iod_batch_get_stats(self._h, C.byref(st)), "iod_batch_get_stats")
        return {k: getattr(st, k) for k, _ in BatchStats._fields_}


__all__ = ["Problem", "Batch", "options", "bounds_from_chief", "simulate_obs", "use_torch_allocator",
           "IodError", "RK4", "DOPRI5", "CR3BP", "ER3BP", "FP64", "MIXED", "COST_CHI2", "COST_QUARTIC", "GBEST_SYNC",
           "GBEST_LAGGED"]
