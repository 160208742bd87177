"""Benchmark: PSO initial orbit determination, paper-scale workload, one GB300.

Workload (the paper-scale configuration): L2 northern halo chief, deputy 1-500 km /
0-5 m/s away, 200 angle pairs over 7 days with 1 arcsec noise, RK4 dt 5e-4 TU (3,383
steps per evaluation), 65,536 particles, w = 0.7, c1 = c2 = 1.5.  One step is one full
swarm iteration: move, propagate every particle to every epoch, angles, cost, personal
and global bests (one fused kernel launch).  Inputs are synthetic (seeded), observations
are synthesised on the GPU by the library itself.

Output: one JSON line.  `value` is particle RK4 steps per second over the timed
iterations (CUDA events on the launching stream, L2 flushed between steps); `e2e`
runs the same metric through the public C ABI from pinned host buffers (create, run
one iteration after initialisation, read the result, destroy) every step.
`--impl reference` times the CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

ORBIT = "halo"
M = 65536
# algorithmic FP64 operations (add, sub, mul, div, sqrt = 1 each; an FMA counts as its
# multiply and add): per RK4 step 4 x 27 (equations of
# motion with shared subexpressions) + 78 (stage combinations); per epoch 22
# (relative position, line of sight, two angles, residuals, weighted squares); per
# particle move 50
FLOP_PER_STEP = 4 * 27 + 78
FLOP_PER_EPOCH = 22
FLOP_PER_MOVE = 50
# FP64 peak derived from unit counts and clocks: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop
# x 2070 MHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
# mixed form: its roofline counts the method's work, the same algorithmic operations as
# the FP64 form (FLOP_PER_STEP, FLOP_PER_EPOCH, FLOP_PER_MOVE), executed in FP32 against
# the FP32 peak (152 SMs x 128 FP32 FMA/clk x 2 flop x 2070 MHz).  Beside it, the FP32
# operations the Encke form itself issues per relative RK4 step (per primary 44: Encke
# terms 11, q 1, |R+D|^2 1, rsqrt 1, gm/r^3 3, F(q) series 15, D - F R 6, accumulate 6;
# linear terms 4 per stage; stage combinations 78; compensated update 24)
FLOP32_ISSUED_PER_STEP = 4 * (2 * 44 + 4) + 78 + 24
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# DOPRI5 5(4), algorithmic FP64 operations per attempted step: six new right-hand sides
# (6 x 27; the seventh stage is the next step's first), the stage states and the
# fifth-order solution (20 tableau terms x 6 components x 2, h folded into the
# coefficients), the error estimate and its norm (6 x 17 + 2) and the step-size
# controller (5, the power counted as one); per epoch the continuous extension (52 for
# the six weight polynomials, 6 x 13 for the components) and the measurement and cost
# (22); per particle move 50
FLOP_PER_DP_ATTEMPT = 6 * 27 + 20 * 6 * 2 + (6 * 17 + 2) + 5
FLOP_PER_DP_EPOCH = 52 + 6 * 13 + FLOP_PER_EPOCH
# DRAM bytes (read + write) per launch from ncu captures of the current kernels: the grid
# FP64 iteration captured at 16,384 particles (2.59 MB; the swarm state is the only DRAM
# data, so it scales with the particles) times 4; the mixed iteration captured at the
# full 65,536 particles (10.64 MB)
TRAFFIC_FP64_65K = 2590464 * 4
# the balanced FP64 iteration (the automatic choice for 65,536 particles on 152 SMs),
# mean of three full-size launches of the current kernel (10.75 MB read, 1 KB written)
TRAFFIC_FP64_BAL_65K = 10753365
TRAFFIC_MIXED_65K = 10640000
# the balanced mixed iteration (the automatic choice at 65,536 particles on 152 SMs),
# mean of three full-size launches of the current kernel (10.77 MB read, 0.2 KB written)
TRAFFIC_MIXED_BAL_65K = 10771200
# the balanced DOPRI5 iteration (queued epoch costs), mean of four full-size launches of
# the current kernel (10.43 MB read, 0.27 MB written: the lanes' epoch queues in local memory)
TRAFFIC_DP_BAL_65K = 10434880 + 270528
METRIC = "IOD solves/s and particle RK steps/s at <=1 km error; p50/p99 solve latency"
_T0 = time.perf_counter()


def log(msg: str) -> None:
    """Progress on stderr (the JSON line alone goes to stdout)."""
    print(f"[bench {time.perf_counter() - _T0:7.1f} s] {msg}", file=sys.stderr, flush=True)
UNIT = "particle RK4 steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--particles", type=int, default=M,
                    help="swarm size (the workload is 65,536; smaller only for profiling)")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision leg")
    ap.add_argument("--no-mixed-solve", action="store_true", help="skip the full mixed solve")
    ap.add_argument("--no-dopri5", action="store_true", help="skip the DOPRI5 iteration leg")
    ap.add_argument("--er3bp", action="store_true",
                    help="also time FP64 iterations with the elliptic restricted dynamics")
    ap.add_argument("--per-orbit", type=int, default=2, metavar="SEEDS",
                    help="solve every chief orbit (and the paper's scenario-1 chief) with SEEDS "
                         "seeds, mixed and FP64 DOPRI5 (and FP64 RK4 for seed 0), with the errors "
                         "against the truth (0: skip)")
    ap.add_argument("--schedule", choices=["auto", "grid", "balanced"], default="auto",
                    help="work distribution of the FP64 and mixed iteration legs "
                         "(iod_options.schedule; auto by default)")
    ap.add_argument("--dopri5-threads", type=int, choices=[0, 1, 2], default=0,
                    help="threads per particle of the DOPRI5 leg (0: the library's choice)")
    ap.add_argument("--sweep-warps", action="store_true",
                    help="also time FP64 and mixed iterations at swarm sizes that put exactly "
                         "1-4 warps on every sub-partition, grid and balanced (slow; off by default)")
    ap.add_argument("--per-orbit-rk4-all", action="store_true",
                    help="with --per-orbit, solve every seed with FP64 RK4 too (default: seed 0 only)")
    ap.add_argument("--no-serving", action="store_true", help="skip the batched and serving legs")
    ap.add_argument("--variant-instances", type=int, default=128,
                    help="instances (the first of the set) for the batch variants: fixed step, "
                         "50 FP64 swarm iterations, and the headline form on the same subset")
    ap.add_argument("--batch-instances", type=int, default=1024,
                    help="noise-free instances of the batched workload in the head-to-head")
    ap.add_argument("--no-paper-table", action="store_true",
                    help="skip the paper's two printed scenarios (accuracy beside its Table 1)")
    ap.add_argument("--serve-loads", default="0.5,0.9,1.5",
                    help="comma-separated arrival rates as fractions of the measured capacity")
    ap.add_argument("--serve-rates", default="50,200,1000",
                    help="comma-separated absolute arrival rates (requests/s)")
    ap.add_argument("--serve-max-requests", type=int, default=64,
                    help="most requests per serving load")
    ap.add_argument("--fp64-sample", type=int, default=8,
                    help="instances solved by the plain FP64 form one at a time (seeded sample)")
    ap.add_argument("--alone-sample", type=int, default=8,
                    help="served requests also run alone, per load (the latency floor)")
    ap.add_argument("--profile-case", choices=["dopri5", "dopri5-divergence", "batch", "alone", "fp64-issue"],
                    default=None,
                    help="run one small case of a kernel for an ncu capture and exit")
    ap.add_argument("--no-tune-dt", dest="tune_dt", action="store_false",
                    help="batched form at the fixed RK4 step 5e-4 instead of autotuned steps")
    ap.add_argument("--dt-candidates", default="2e-3,1e-3,5e-4",
                    help="RK4 step bounds the batched form's autotuner may choose from")
    ap.add_argument("--refine-iters", type=int, default=400,
                    help="most Levenberg-Marquardt iterations closing each solve (0: swarm only); "
                         "400 is the iteration cap of the least-squares solver the paper used")
    ap.add_argument("--refine-gate", type=float, default=10.0,
                    help="batched and served solves whose refined cost exceeds this many units per "
                         "epoch are solved again in FP64 (0: off)")
    ap.add_argument("--mixed-fp64-last", type=int, default=0,
                    help="FP64 swarm iterations at the end of a mixed solve that Levenberg-"
                         "Marquardt closes (per-orbit, batched and served solves; the personal "
                         "bests are re-evaluated in FP64 in every case)")
    ap.add_argument("--oracle-subset", type=int, default=4,
                    help="cheapest batched instances also solved by the oracle (CPU-baseline leg)")
    return ap.parse_args()


def workload(seed: int = 0):
    from paper_2207_13175_gb300 import inputs as I
    return I.paper_scale(ORBIT, seed)


def workload_config(sc, steps_per_eval):
    return {"workload": f"paper-scale PSO-IOD: {ORBIT} chief, {sc.m} particles, "
                        f"{sc.n_obs} angle pairs over 7 d, RK4 dt {sc.dt}",
            "orbit": ORBIT, "particles": sc.m, "n_obs": sc.n_obs, "arc_days": 7.0,
            "integrator": "rk4", "dt_tu": sc.dt, "rk4_steps_per_eval": steps_per_eval,
            "iterations_per_solve": sc.iters, "step": "one swarm iteration",
            "l2": "flushed (256 MiB write) between timed steps"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
                pw.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_median": statistics.median(pw) if pw else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_setup(n_gpus):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return rank, world, local


def aggregate(local_seconds: float, local_units: float, world: int):
    """Max of the per-rank timed seconds and sum of the units over ranks."""
    if world == 1:
        return local_seconds, local_units
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([local_seconds], dtype=torch.float64, device=dev)
    u = torch.tensor([local_units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


_ORA_PROBLEM = None


def _oracle_pool_init(args):
    """Worker set-up: each process builds its own oracle problem."""
    global _ORA_PROBLEM
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import oracle as O
    mu, chief, t, ra, dec, sra, sdec, dt = args
    _ORA_PROBLEM = O.Problem(mu, chief, t, ra, dec, sra, sdec, dt=dt)


def _oracle_pool_eval(X):
    """Costs of a block of candidate states; returns how many were evaluated."""
    _ORA_PROBLEM.costs(X)
    return len(X)


def _oracle_solve_instance(job):
    """One batched instance solved by the oracle from its own inputs: the chief phased by
    its own DOPRI5 (tolerance 1e-13), noise-free observations from its own simulation,
    its own box, then its Algorithm 1 run.  Returns (final state, seconds)."""
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import oracle as O
    from paper_2207_13175_gb300 import inputs as I
    mu, chief0, phase, offset, t, sigma, r_km, v_ms, dt, m, iters, seed, refine = job
    t0 = time.perf_counter()
    st, _, _, rc = O.propagate_dopri5(mu, chief0, [phase], rtol=1e-13, atol=1e-13)
    chief = st[0]
    deputy = chief + offset
    ra, dec, _, _ = O.simulate_obs(mu, chief, deputy, t)
    P = O.Problem(mu, chief, t, ra, dec, *sigma, dt=dt)
    lo, hi = O.bounds_from_chief(chief, r_km, v_ms, I.L_KM, I.TU_S)
    W, _, _ = O.Pso(P, lo, hi, seed=seed).run(m, iters)
    x = W.g
    if refine > 0:
        x, _, _, _ = P.lm_refine(W.g, refine)
    return x.tolist(), deputy.tolist(), time.perf_counter() - t0


def oracle_batched_subset(subset):
    """The oracle on the cheapest noise-free batched instances (one spawned process per
    instance): its solve time and truth error, and how far the GPU's FP64 (one at a time)
    and mixed (batched) final positions lie from its own."""
    import multiprocessing as mp

    import numpy as np
    jobs = []
    for e in subset:
        sc = e["sc"]
        jobs.append((sc.mu, sc.chief, sc.meta["phase_tu"], sc.deputy, sc.t, sc.sigma, sc.r_max_km,
                     sc.v_max_ms, sc.dt, sc.m, sc.iters, sc.seed, e["refine_iters"]))
    ctx = mp.get_context("spawn")
    with ctx.Pool(max(1, len(jobs))) as pool:
        got = pool.map(_oracle_solve_instance, jobs)
    out = []
    for e, (g, dep_o, sec) in zip(subset, got):
        g = np.array(g)
        km = lambda a, b: float(np.linalg.norm(np.asarray(a)[:3] - np.asarray(b)[:3]) * 384400.0)
        out.append({"index": e["index"], "m": e["sc"].m, "iters": e["sc"].iters,
                    "n_obs": int(e["sc"].t.size), "work": e["work"], "oracle_s": sec,
                    "oracle_pos_err_km": km(g, dep_o),
                    "fp64_gpu_vs_oracle_km": km(e["fp64_state"], g),
                    "mixed_batch_vs_oracle_km": km(e["mixed_state"], g),
                    "truth_gpu_vs_oracle_km": km(e["deputy"], dep_o)})
    return out


def cpu_baseline(sc, sample_m=2048, sample_iters=9):
    """The oracle, as it stands, on bounded samples of the workload (the full problem:
    200 epochs, RK4 dt 5e-4).  Single-threaded: a 2,048-particle swarm for 9 iterations.
    All host cores: one evaluation of a 65,536-candidate set (the swarm size of the
    workload) split over a pool of processes (spawned), each running the oracle on its
    share; pool start-up is outside the timed region."""
    import multiprocessing as mp

    import numpy as np

    import oracle as O
    from paper_2207_13175_gb300 import inputs as I
    ra, dec, _, _ = O.simulate_obs(sc.mu, sc.chief, sc.deputy, sc.t, sc.noise)
    P = O.Problem(sc.mu, sc.chief, sc.t, ra, dec, *sc.sigma, dt=sc.dt)
    lo, hi = O.bounds_from_chief(sc.chief, sc.r_max_km, sc.v_max_ms, I.L_KM, I.TU_S)
    t0 = time.perf_counter()
    W, _, _ = O.Pso(P, lo, hi, w=sc.w, c1=sc.c1, c2=sc.c2, seed=sc.seed).run(sample_m, sample_iters)
    dt = time.perf_counter() - t0
    single = {"value": W.steps / dt, "unit": UNIT, "cores": 1,
              "sample": f"{sample_m} particles x {sample_iters + 1} evaluations of the same "
                        f"problem ({W.steps} RK4 steps, {dt:.1f} s, single-threaded)"}
    spe = int(P.steps_per_eval(sc.deputy))
    cores = os.cpu_count() or 1
    X = I.particles_in_box(lo, hi, M, seed=3)
    chunks = np.array_split(X, cores * 4)
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores, initializer=_oracle_pool_init,
                  initargs=((sc.mu, sc.chief, sc.t, ra, dec, sc.sigma[0], sc.sigma[1], sc.dt),)) as pool:
        pool.map(_oracle_pool_eval, [c[:1] for c in chunks[:cores]])     # start every worker
        t0 = time.perf_counter()
        n = sum(pool.map(_oracle_pool_eval, chunks))
        dt_all = time.perf_counter() - t0
    steps = n * spe
    return {"value": steps / dt_all, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} candidate states x 1 evaluation ({steps} RK4 steps) over {cores} "
                      f"processes, {dt_all:.1f} s",
            "single_thread": single}


def reference_arm(args):
    """--impl reference: the CPU oracle, as it stands, on all host cores (a pool of
    spawned processes each running the oracle on its share); each step evaluates one
    fresh set of 16,384 candidate states of the same problem in the box."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import multiprocessing as mp

    import numpy as np

    import oracle as O
    from paper_2207_13175_gb300 import inputs as I
    O.build()
    sc = workload(0)
    ra, dec, _, _ = O.simulate_obs(sc.mu, sc.chief, sc.deputy, sc.t, sc.noise)
    P = O.Problem(sc.mu, sc.chief, sc.t, ra, dec, *sc.sigma, dt=sc.dt)
    lo, hi = O.bounds_from_chief(sc.chief, sc.r_max_km, sc.v_max_ms, I.L_KM, I.TU_S)
    spe = int(P.steps_per_eval(sc.deputy))
    cores = os.cpu_count() or 1
    sample = 16384
    sets = [np.array_split(I.particles_in_box(lo, hi, sample, seed=100 + k), cores * 4)
            for k in range(args.warmup + args.steps)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores, initializer=_oracle_pool_init,
                  initargs=((sc.mu, sc.chief, sc.t, ra, dec, sc.sigma[0], sc.sigma[1], sc.dt),)) as pool:
        for k in range(args.warmup):
            pool.map(_oracle_pool_eval, sets[k])
        t0 = time.perf_counter()
        n = 0
        for k in range(args.warmup, args.warmup + args.steps):
            n += sum(pool.map(_oracle_pool_eval, sets[k]))
        dt = time.perf_counter() - t0
    steps = n * spe
    value = steps / dt
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": workload_config(sc, spe),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"each step: costs of {sample} candidate states of the same "
                                      f"problem ({spe} RK4 steps each) over {cores} processes"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def profile_case(args):
    """--profile-case: run one small case of a kernel for an ncu capture, then exit.
    dopri5: the paper-scale halo workload with DOPRI5 (65,536 particles or --particles),
    initialised, then --steps iterations (iter_kernel<DOPRI5>).  batch: 24 noise-free
    instances of the batched workload (8 per swarm size) cut to 100 iterations, with the
    head-to-head's options (mixed, no FP64 swarm tail, Levenberg-Marquardt, step 2e-3),
    solved by one persistent launch (wq_kernel) after a warm-up launch.  alone: one 1,024-particle request with the serving options, solved by
    one persistent launch after a warm-up launch (the latency floor of a request).
    fp64-issue: the library's FP64 chain diagnostic by warps and active lanes."""
    import torch

    from paper_2207_13175_gb300 import api
    from paper_2207_13175_gb300 import inputs as I
    out = {"profile_case": args.profile_case}
    if args.profile_case == "dopri5":
        sc = I.paper_scale(ORBIT, 0, integrator="dopri5").with_(m=args.particles)
        ang, _ = api.simulate_obs(sc.mu, sc.chief, sc.deputy, sc.t, sc.noise)
        bounds = api.bounds_from_chief(sc.chief, sc.r_max_km, sc.v_max_ms, I.L_KM, I.TU_S)
        opts = api.options(integrator=api.DOPRI5, rtol=sc.rtol, atol=sc.atol, h0=sc.h0)
        with api.Problem(sc.mu, sc.chief, sc.t, ang, sc.sigma, bounds, opts) as G:
            G.run(sc.m, 0, sc.w, sc.c1, sc.c2, sc.seed)
            s0 = G.result(trace=False)["rk_steps"]
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            G.continue_(args.steps)
            e1.record()
            r = G.result(trace=False)
        out.update(ms_per_iteration=e0.elapsed_time(e1) / args.steps, particles=sc.m,
                   attempts_per_particle_iteration=(r["rk_steps"] - s0) / (sc.m * args.steps))
    elif args.profile_case == "dopri5-divergence":
        # the DOPRI5 iteration's divergence cost: the swarm after three iterations (lagged
        # order, so that the iteration evaluates the positions it is given) against the
        # same swarm with every 32-particle group holding 32 copies of its first particle
        import numpy as np
        sc = I.paper_scale(ORBIT, 0, integrator="dopri5").with_(m=args.particles)
        ang, _ = api.simulate_obs(sc.mu, sc.chief, sc.deputy, sc.t, sc.noise)
        bounds = api.bounds_from_chief(sc.chief, sc.r_max_km, sc.v_max_ms, I.L_KM, I.TU_S)
        opts = api.options(integrator=api.DOPRI5, rtol=sc.rtol, atol=sc.atol, h0=sc.h0, gbest_order=1)
        with api.Problem(sc.mu, sc.chief, sc.t, ang, sc.sigma, bounds, opts) as G:
            G.run(sc.m, 3, sc.w, sc.c1, sc.c2, sc.seed)
            sw = G.swarm_get()

            def timed(x, v, p, pJ):
                best, att = None, 0
                for _ in range(3):
                    G.swarm_set(x, v, p, pJ, sw["g"], sw["gJ"], sw["gidx"], sw["iter"], sc.w, sc.c1, sc.c2,
                                sc.seed)
                    s0 = G.result(trace=False)["rk_steps"]
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    G.continue_(1)
                    e1.record()
                    torch.cuda.synchronize()
                    ms = e0.elapsed_time(e1)
                    best = ms if best is None else min(best, ms)
                    att = G.result(trace=False)["rk_steps"] - s0
                return best, att

            t_real, a_real = timed(sw["x"], sw["v"], sw["p"], sw["pJ"])
            rep = (np.arange(sc.m) // 32) * 32
            t_rep, a_rep = timed(sw["x"][:, rep], sw["v"][:, rep], sw["p"][:, rep], sw["pJ"][rep])
        out.update(swarm_ms=t_real, swarm_attempts=int(a_real), replicated_ms=t_rep,
                   replicated_attempts=int(a_rep), divergence_cost=t_real / t_rep * a_rep / a_real - 1.0)
    elif args.profile_case == "fp64-issue":
        # SM cycles per dependent FP64 FMA by warps in one block and active lanes per warp
        out["cycles_per_fma"] = {f"{w} warps": {f"{ln} lanes": api.selftest_fp64_issue(w, ln)
                                                for ln in (1, 8, 16, 32)} for w in (1, 2, 4, 8)}
    elif args.profile_case == "alone":
        # one noise-free 1,024-particle request of the serving mix, alone on the GPU, with
        # the serving options (mixed, no FP64 swarm tail, refinement, step 2e-3)
        inst = [x for x in batched_instances(40, seed=100, noise=False) if x[0].m == 1024][:1]
        opts = api.options(dt=5e-4, precision=api.MIXED, fp64_last_iters=0, refine_iters=60)
        run_batch([inst[0][0]], opts, block=128, dts=([1 << 30], [2e-3]))   # warm-up
        res, wall, _ = run_batch([inst[0][0]], opts, block=128, dts=([1 << 30], [2e-3]))
        q = inst[0][0]
        out.update(launch_wall_s=wall, particles=q.m, iterations=q.iters, epochs=int(q.t.size),
                   rk_steps=res[0]["rk_steps"], refine_iters=res[0]["refine_iters"],
                   pos_err_km=pos_err_km(res[0]["state"], inst[0][1]))
    else:
        # 24 noise-free instances of the batched workload (8 of each swarm size) cut to 100
        # iterations, with the head-to-head's options: mixed precision without an FP64
        # swarm tail, refinement, step 2e-3, 128-thread blocks
        pool = batched_instances(80, seed=7, noise=False)
        inst = []
        for m in (1024, 4096, 16384):
            inst += [x for x in pool if x[0].m == m][:8]
        reqs = [x[0] for x in inst]
        for q in reqs:
            q.iters = 100
        opts = api.options(dt=5e-4, precision=api.MIXED, fp64_last_iters=0, refine_iters=60)
        dts = ([1 << 30], [2e-3])
        run_batch(reqs[:3], opts, block=128, dts=dts)    # warm-up launch
        res, wall, _ = run_batch(reqs, opts, block=128, dts=dts)
        steps = sum(r["rk_steps"] for r in res)
        out.update(launch_wall_s=wall, instances=len(reqs), rk_steps=steps,
                   rk_steps_per_s=steps / wall,
                   pos_err_km_max=max(pos_err_km(r["state"], d) for r, (_, d, _, _) in zip(res, inst)))
    print(json.dumps(out))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.profile_case:
        return profile_case(args)
    import numpy as np
    import torch

    from paper_2207_13175_gb300 import api
    from paper_2207_13175_gb300 import inputs as I

    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sc = workload(rank).with_(m=args.particles)   # independent problems per rank (weak scaling)
    ang, _ = api.simulate_obs(sc.mu, sc.chief, sc.deputy, sc.t, sc.noise)
    bounds = api.bounds_from_chief(sc.chief, sc.r_max_km, sc.v_max_ms, I.L_KM, I.TU_S)
    stream = torch.cuda.current_stream(dev)
    opts = api.options(dt=sc.dt, schedule=sched_option(args))
    G = api.Problem(sc.mu, sc.chief, sc.t, ang, sc.sigma, bounds, opts, stream=stream)
    G.run(sc.m, 0, sc.w, sc.c1, sc.c2, sc.seed)
    r0 = G.result(trace=False)
    spe = r0["rk_steps"] // sc.m          # RK4 steps per evaluation (3,383)
    for _ in range(args.warmup):
        G.continue_(1)
    torch.cuda.synchronize(dev)

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize(dev)
    t_wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        G.continue_(1)
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    per_ms = [a.elapsed_time(b) for a, b in ev]
    local_s = sum(per_ms) / 1e3
    max_s, units = aggregate(local_s, float(sc.m) * spe * args.steps, world)
    value = units / max_s
    ms_per_step = max_s / args.steps * 1e3
    r = G.result(trace=False)
    assert r["iters_done"] == args.warmup + args.steps
    balanced = r["schedule"] == api.SCHED_BALANCED
    if balanced:
        kernel = "iter_kernel_balanced<SYNC>"
        traffic = TRAFFIC_FP64_BAL_65K if sc.m == M else None
        traffic_src = "ncu dram__bytes_read.sum + dram__bytes_write.sum, capture of a 65,536-particle launch"
    else:
        kernel = "iter_kernel<RK4,SYNC>"
        traffic = TRAFFIC_FP64_65K * sc.m // M if sc.m % 16384 == 0 else None
        traffic_src = "ncu dram__bytes_read.sum + dram__bytes_write.sum, 16,384-particle capture scaled by particles"
    flop_launch = sc.m * (spe * FLOP_PER_STEP + sc.n_obs * FLOP_PER_EPOCH + FLOP_PER_MOVE)
    achieved = flop_launch / (statistics.mean(per_ms) / 1e3) / 1e12
    G.close()

    log(f"FP64 leg: {ms_per_step:.2f} ms per iteration")
    mixed = None if args.no_mixed else mixed_leg(args, sc, ang, bounds, stream, dev, world, spe)
    log("mixed leg done")
    dopri = None if args.no_dopri5 else dopri5_leg(args, sc, ang, bounds, stream, dev, world)
    log("DOPRI5 leg done")
    orbits = per_orbit_leg(args, stream, dev) if args.per_orbit > 0 and world == 1 else None
    sweep = sweep_warps_leg(stream, dev) if args.sweep_warps and world == 1 else None
    er3bp = er3bp_leg(args, sc, bounds, stream, dev, world) if args.er3bp else None
    batched = None if args.no_serving or world > 1 else batched_and_serving_leg(args)
    log("batched and serving legs done")
    e2e = None if args.no_e2e else end_to_end(args, sc, ang, bounds, opts, stream, dev, world)
    log("end-to-end leg done")
    table = None if args.no_paper_table or world > 1 else paper_table_leg(stream, dev)
    log("paper-scenario leg done")
    if mixed is not None and "solve_s" in mixed:
        mixed["fp64_solve_s_extrapolated"] = ms_per_step * (sc.iters + 1) / 1e3
        mixed["speedup_vs_fp64_solve"] = mixed["fp64_solve_s_extrapolated"] / mixed["solve_s"]
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(sc, spe),
        "particle_iterations_per_s": units / spe / max_s,
        "solves_per_s_extrapolated": value / (float(sc.m) * spe * (sc.iters + 1)),
        "solves_per_s_extrapolated_note": "one iteration's rate extrapolated to 501 evaluations; "
                                          "measured complete solves are the per_orbit_* fields",
        "solve_latency_s_extrapolated": ms_per_step * (sc.iters + 1) / 1e3,
        "wall_s_timed_region": t_wall,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                     "traffic": traffic, "traffic_source": traffic_src, "kernel": kernel,
                     "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2070 MHz",
                     "flop_per_launch": flop_launch},
        "e2e": e2e,
        "mixed": mixed,
        "dopri5": dopri,
        "er3bp": er3bp,
        "per_orbit": orbits,
        "sweep_warps": sweep,
        "batched_serving": batched,
        "paper_table": table,
        "clocks": clk,
        "gpu_launches": args.steps,
    }
    subset = batched.pop("_oracle_subset", None) if batched else None
    if orbits:
        for form in ("mixed", "dopri5", "fp64"):
            rows = [r[form] for r in orbits if form in r]
            if rows:
                out[f"per_orbit_{form}_solves_per_s"] = len(rows) / sum(x["s"] for x in rows)
                out[f"per_orbit_{form}_pos_err_km_max"] = max(x["pos_err_km"] for x in rows)
                out[f"per_orbit_{form}_swarm_only_pos_err_km_max"] = max(x["swarm_pos_err_km"] for x in rows)
                out[f"per_orbit_{form}_solves"] = len(rows)
    if batched:
        out.update(head_to_head_fields(batched))
        if len(batched.get("instance_records", [])) > 128:
            batched.pop("instance_records")
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        out["cpu_baseline"] = cpu_baseline(sc)
        out["cpu_baseline"]["tiny"] = tiny_leg(stream, dev)
        if subset:
            rows = oracle_batched_subset(subset)
            out["cpu_baseline"]["batched_subset"] = rows
            out["fp64_vs_oracle_pos_km_max"] = max(r["fp64_gpu_vs_oracle_km"] for r in rows)
            out["mixed_vs_oracle_pos_km_max"] = max(r["mixed_batch_vs_oracle_km"] for r in rows)
            out["oracle_subset_pos_err_km_max"] = max(r["oracle_pos_err_km"] for r in rows)
        log("CPU baseline done")
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def mixed_leg(args, sc, ang, bounds, stream, dev, world, spe):
    """The mixed-precision form of the same workload: the FP32 iteration kernel timed
    like the FP64 one, then one complete solve (500 iterations: 450 FP32, FP64
    rescoring of every personal best, 50 FP64) timed end to end on the device."""
    import torch

    from paper_2207_13175_gb300 import api
    opts = api.options(dt=sc.dt, precision=api.MIXED, fp64_last_iters=50, schedule=sched_option(args))
    G = api.Problem(sc.mu, sc.chief, sc.t, ang, sc.sigma, bounds, opts, stream=stream)
    G.run(sc.m, 0, sc.w, sc.c1, sc.c2, sc.seed)
    for _ in range(args.warmup):
        G.continue_(1)
    torch.cuda.synchronize(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize(dev)
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        G.continue_(1)
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    per_ms = [a.elapsed_time(b) for a, b in ev]
    max_s, units = aggregate(sum(per_ms) / 1e3, float(sc.m) * spe * args.steps, world)
    flop = sc.m * (spe * FLOP_PER_STEP + sc.n_obs * FLOP_PER_EPOCH + FLOP_PER_MOVE)
    flop_issued = sc.m * spe * FLOP32_ISSUED_PER_STEP
    sec = statistics.mean(per_ms) / 1e3
    achieved = flop / sec / 1e12
    balanced = G.result(trace=False)["schedule"] == api.SCHED_BALANCED
    out = {"kernel": "iter_mixed_balanced<SYNC>" if balanced else "iter_mixed_kernel<SYNC>",
           "ms_per_step": max_s / args.steps * 1e3,
           "value": units / max_s, "unit": UNIT,
           "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                        "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                        "traffic": (TRAFFIC_MIXED_BAL_65K if balanced else TRAFFIC_MIXED_65K)
                        if sc.m == M else None,
                        "peak_source": "derived: 152 SMs x 128 FP32 FMA/clk x 2 flop x 2070 MHz",
                        "flop_per_launch": flop,
                        "flop_basis": "the method's algorithmic operations (186 per RK4 step, 22 per "
                                      "epoch, 50 per move), as for the FP64 form",
                        "issued_flop_per_launch": flop_issued,
                        "issued_achieved": flop_issued / sec / 1e12,
                        "issued_frac": flop_issued / sec / 1e12 / FP32_PEAK_TFLOPS}}
    if not args.no_mixed_solve:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(world)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        G.run(sc.m, sc.iters, sc.w, sc.c1, sc.c2, sc.seed)
        e1.record(stream)
        r = G.result(trace=False)
        solve_s, n_solves = aggregate(e0.elapsed_time(e1) / 1e3, 1.0, world)
        from paper_2207_13175_gb300 import inputs as I
        out.update({
            "solve_s": solve_s, "solves_per_s": n_solves / solve_s,
            "solve": f"{sc.iters} iterations ({sc.iters - 50} FP32, FP64 rescoring, 50 FP64), "
                     f"{sc.m} particles, device time",
            "solve_rk_steps": r["rk_steps"], "solve_fp64_moon_steps": r["fp64_steps"],
            "solve_pos_err_km": float(((r["state"][:3] - sc.deputy[:3]) ** 2).sum() ** 0.5 * I.L_KM),
            "solve_vel_err_ms": float(((r["state"][3:] - sc.deputy[3:]) ** 2).sum() ** 0.5
                                      * I.L_KM / I.TU_S * 1e3),
            "fp64_solve_s_extrapolated": None})
    G.close()
    return out


def dopri5_leg(args, sc, ang, bounds, stream, dev, world, iters=3):
    """The same workload with the DOPRI5 5(4) integrator at rtol = atol = 1e-12 (dense
    output at the epochs): a few FP64 iterations timed like the RK4 ones; the unit is
    attempted DOPRI5 steps (six new stage evaluations each)."""
    import torch

    from paper_2207_13175_gb300 import api
    opts = api.options(integrator=api.DOPRI5, rtol=sc.rtol, atol=sc.atol, h0=sc.h0,
                       threads_per_particle=args.dopri5_threads)
    G = api.Problem(sc.mu, sc.chief, sc.t, ang, sc.sigma, bounds, opts, stream=stream)
    G.run(sc.m, 1, sc.w, sc.c1, sc.c2, sc.seed)
    s0 = G.result(trace=False)["rk_steps"]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(iters)]
    barrier(world)
    torch.cuda.synchronize(dev)
    for k in range(iters):
        ev[k][0].record(stream)
        G.continue_(1)
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    r_end = G.result(trace=False)
    steps = r_end["rk_steps"] - s0
    balanced = r_end["schedule"] == api.SCHED_BALANCED
    G.close()
    per_ms = [a.elapsed_time(b) for a, b in ev]
    max_s, units = aggregate(sum(per_ms) / 1e3, float(steps), world)
    attempts = steps / iters
    flop = attempts * FLOP_PER_DP_ATTEMPT + sc.m * (sc.n_obs * FLOP_PER_DP_EPOCH + FLOP_PER_MOVE)
    achieved = flop / (statistics.mean(per_ms) / 1e3) / 1e12
    return {"kernel": "iter_kernel_balanced_dp<SYNC>" if balanced else "iter_kernel<DOPRI5,SYNC>",
            "ms_per_step": max_s / iters * 1e3,
            "value": units / max_s, "unit": "particle DOPRI5 attempted steps/s",
            "attempts_per_particle_iteration": steps / (iters * sc.m),
            "tolerances": f"rtol = atol = {sc.rtol}",
            "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                         "traffic": TRAFFIC_DP_BAL_65K if balanced and sc.m == M else None,
                         "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2070 MHz",
                         "flop_per_launch": flop,
                         "flop_basis": f"{FLOP_PER_DP_ATTEMPT} per attempted step, {FLOP_PER_DP_EPOCH} per "
                                       f"epoch (continuous extension + cost), {FLOP_PER_MOVE} per move"}}


def tiny_leg(stream, dev):
    """Part of the CPU-baseline leg.  The small configuration (256 particles, 100
    iterations, 20 epochs over a day, RK4 dt 1e-3): the oracle's solve, single-threaded
    on the host, from its own synthesised observations, and one complete FP64 solve of
    the same inputs on the GPU (device time), with both errors against the truth."""
    import numpy as np
    import torch

    import oracle as O
    from paper_2207_13175_gb300 import api
    from paper_2207_13175_gb300 import inputs as I
    O.build()
    sc = I.tiny(0)
    ra, dec, _, _ = O.simulate_obs(sc.mu, sc.chief, sc.deputy, sc.t, sc.noise)
    ang = np.stack([ra, dec], 1)
    box = api.bounds_from_chief(sc.chief, sc.r_max_km, sc.v_max_ms, I.L_KM, I.TU_S)
    with api.Problem(sc.mu, sc.chief, sc.t, ang, sc.sigma, box, api.options(dt=sc.dt), stream=stream) as G:
        G.run(sc.m, sc.iters, sc.w, sc.c1, sc.c2, sc.seed)        # warm-up
        G.result(trace=False)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        G.run(sc.m, sc.iters, sc.w, sc.c1, sc.c2, sc.seed)
        e1.record(stream)
        r = G.result(trace=False)
        gpu_s = e0.elapsed_time(e1) / 1e3
    P = O.Problem(sc.mu, sc.chief, sc.t, ra, dec, *sc.sigma, dt=sc.dt)
    lo, hi = O.bounds_from_chief(sc.chief, sc.r_max_km, sc.v_max_ms, I.L_KM, I.TU_S)
    t0 = time.perf_counter()
    W, _, _ = O.Pso(P, lo, hi, w=sc.w, c1=sc.c1, c2=sc.c2, seed=sc.seed).run(sc.m, sc.iters)
    ora_s = time.perf_counter() - t0
    err = lambda x: float(np.linalg.norm(np.asarray(x)[:3] - sc.deputy[:3]) * I.L_KM)
    return {"workload": "256 particles x 100 iterations, 20 angle pairs over 1 d, RK4 dt 1e-3",
            "gpu_solve_s": gpu_s, "oracle_solve_s_single_thread": ora_s,
            "rk_steps": r["rk_steps"], "gpu_pos_err_km": err(r["state"]), "oracle_pos_err_km": err(W.g),
            "same_final_state": bool(np.array_equal(r["state"], W.g))}


def er3bp_leg(args, sc, bounds, stream, dev, world, iters=3, ecc=0.0549, f0=0.0):
    """The same workload in the elliptic restricted problem (the Moon's eccentricity,
    pulsating frame, true anomaly from 0), observations synthesised in that problem: a
    few FP64 RK4 iterations timed like the circular ones."""
    import numpy as np
    import torch

    from paper_2207_13175_gb300 import api
    ang, _ = api.simulate_obs(sc.mu, sc.chief, sc.deputy, sc.t, sc.noise, ecc=ecc, f0=f0)
    opts = api.options(dt=sc.dt, dynamics=api.ER3BP, ecc=ecc, f0=f0)
    G = api.Problem(sc.mu, sc.chief, sc.t, ang, sc.sigma, bounds, opts, stream=stream)
    G.run(sc.m, 1, sc.w, sc.c1, sc.c2, sc.seed)
    s0 = G.result(trace=False)["rk_steps"]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(iters)]
    barrier(world)
    torch.cuda.synchronize(dev)
    for k in range(iters):
        ev[k][0].record(stream)
        G.continue_(1)
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    r_end = G.result(trace=False)
    steps = r_end["rk_steps"] - s0
    G.close()
    per_ms = [a.elapsed_time(b) for a, b in ev]
    max_s, units = aggregate(sum(per_ms) / 1e3, float(steps), world)
    kern = "iter_kernel_balanced<SYNC, elliptic>" if r_end["schedule"] == api.SCHED_BALANCED else "iter_kernel_er<SYNC>"
    return {"kernel": kern, "ms_per_step": max_s / iters * 1e3,
            "value": units / max_s, "unit": UNIT, "eccentricity": ecc,
            "steps_per_particle_iteration": steps / (iters * sc.m)}


def sched_option(args):
    from paper_2207_13175_gb300 import api
    return {"auto": api.SCHED_AUTO, "grid": api.SCHED_GRID, "balanced": api.SCHED_BALANCED}[args.schedule]


def sweep_warps_leg(stream, dev):
    """Iteration times of the halo workload at m = 4 SMs x 32 x k particles (k = 1..4
    warps on every FP64 sub-partition when one thread per particle): FP64 in the grid
    form (32- and 128-thread blocks) and balanced, and the mixed form's FP32 iterations in
    the grid form (128-thread blocks) and balanced (from one 384-particle super-group per
    SM).  3 iterations timed by CUDA events after one untimed."""
    import torch

    from paper_2207_13175_gb300 import api
    from paper_2207_13175_gb300 import inputs as I
    sc = I.paper_scale(ORBIT, 0)
    ang, _ = api.simulate_obs(sc.mu, sc.chief, sc.deputy, sc.t, sc.noise)
    bounds = api.bounds_from_chief(sc.chief, sc.r_max_km, sc.v_max_ms, I.L_KM, I.TU_S)
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    forms = [("fp64 grid 32", api.FP64, api.SCHED_GRID, 32), ("fp64 grid 128", api.FP64, api.SCHED_GRID, 128),
             ("fp64 balanced", api.FP64, api.SCHED_BALANCED, 0),
             ("mixed grid 128", api.MIXED, api.SCHED_GRID, 128), ("mixed balanced", api.MIXED, api.SCHED_BALANCED, 0)]
    rows = []
    for k in (1, 2, 3, 4):
        m = 4 * nsm * 32 * k
        row = {"warps_per_subpartition": k, "particles": m}
        for name, prec, sched, bs in forms:
            opts = api.options(dt=sc.dt, precision=prec, fp64_last_iters=0, schedule=sched, block_size=bs)
            with api.Problem(sc.mu, sc.chief, sc.t, ang, sc.sigma, bounds, opts, stream=stream) as G:
                G.run(m, 0, sc.w, sc.c1, sc.c2, 0)
                G.continue_(1)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize(dev)
                e0.record(stream)
                G.continue_(3)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                ran = G.result(trace=False)["schedule"]
                row[name] = {"ms": e0.elapsed_time(e1) / 3,
                             "ran": "balanced" if ran == api.SCHED_BALANCED else "grid"}
        log("sweep k=%d: " % k + ", ".join("%s %.2f ms (%s)" % (n, row[n]["ms"], row[n]["ran"]) for n, *_ in forms))
        rows.append(row)
    return rows


def per_orbit_leg(args, stream, dev):
    """Each corrected chief orbit (L1 Lyapunov, L2 halo, DRO) and the paper's scenario-1
    chief (its lunar passage at 0.0118 LU puts the mixed form's FP64 near-Moon steps to
    work) with its seeded deputies: complete solves (500 iterations, 65,536 particles) in
    mixed precision (RK4 dt 5e-4) and in FP64 with DOPRI5 (rtol = atol = 1e-12) for every
    seed, and in FP64 with RK4 dt 5e-4 for seed 0 (all seeds with --per-orbit-rk4-all),
    each closed by Levenberg-Marquardt from the swarm's best (the paper's pipeline);
    errors against the truth (swarm alone and refined) and times."""
    import numpy as np
    import torch

    from paper_2207_13175_gb300 import api
    from paper_2207_13175_gb300 import inputs as I
    out = []
    for orbit in ("lyapunov", "halo", "dro", "paper-s1"):
        for seed in range(args.per_orbit):
            sc = I.paper_scale(orbit, seed)
            ang, _ = api.simulate_obs(sc.mu, sc.chief, sc.deputy, sc.t, sc.noise)
            bounds = api.bounds_from_chief(sc.chief, sc.r_max_km, sc.v_max_ms, I.L_KM, I.TU_S)
            row = {"orbit": orbit, "seed": seed, "offset_km": sc.meta["offset_km"],
                   "offset_ms": sc.meta["offset_ms"]}
            last = args.mixed_fp64_last if args.refine_iters > 0 else 50
            forms = [("mixed", api.options(dt=sc.dt, precision=api.MIXED, fp64_last_iters=last)),
                     ("dopri5", api.options(integrator=api.DOPRI5, rtol=sc.rtol, atol=sc.atol, h0=sc.h0))]
            if seed == 0 or args.per_orbit_rk4_all:
                forms.append(("fp64", api.options(dt=sc.dt)))
            for name, opts in forms:
                with api.Problem(sc.mu, sc.chief, sc.t, ang, sc.sigma, bounds, opts, stream=stream) as G:
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    torch.cuda.synchronize(dev)
                    e0.record(stream)
                    G.run(sc.m, sc.iters, sc.w, sc.c1, sc.c2, sc.seed)
                    e1.record(stream)
                    r = G.result(trace=False)
                    swarm_s = e0.elapsed_time(e1) / 1e3
                    x, c = r["state"], r["cost"]
                    t0 = time.perf_counter()
                    if args.refine_iters > 0:
                        # the paper's pipeline: Levenberg-Marquardt from the swarm's best
                        # (FP64 RK4 on the problem's grid, like every refinement here)
                        with api.Problem(sc.mu, sc.chief, sc.t, ang, sc.sigma, bounds,
                                         api.options(dt=sc.dt), stream=stream) as R:
                            x, c, _ = R.refine(r["state"], args.refine_iters)
                    lm_s = time.perf_counter() - t0
                    err = lambda y: float(np.linalg.norm(np.asarray(y)[:3] - sc.deputy[:3]) * I.L_KM)
                    row[name] = {"s": swarm_s + lm_s, "swarm_s": swarm_s, "refine_s": lm_s,
                                 "cost": c, "swarm_cost": r["cost"],
                                 "pos_err_km": err(x), "swarm_pos_err_km": err(r["state"]),
                                 "vel_err_ms": float(np.linalg.norm(np.asarray(x)[3:] - sc.deputy[3:])
                                                     * I.L_KM / I.TU_S * 1e3),
                                 "rk_steps": r["rk_steps"], "fp64_steps": r["fp64_steps"],
                                 "state": np.asarray(x).tolist(), "swarm_state": r["state"].tolist()}
            ref = row["fp64"] if "fp64" in row else row["dopri5"]
            row["mixed_vs_fp64_pos_km"] = float(np.linalg.norm(
                np.array(row["mixed"]["state"][:3]) - np.array(ref["state"][:3])) * I.L_KM)
            log(f"{orbit} seed {seed}: " + ", ".join(
                f"{name} {row[name]['swarm_pos_err_km']:.3f} -> {row[name]['pos_err_km']:.3f} km in "
                f"{row[name]['s']:.1f} s" for name, _ in forms))
            out.append(row)
    return out


def batched_instances(n, seed=7, noise=False):
    """n instances of the batched workload (chiefs phased along their orbits on the GPU,
    observations synthesised on the GPU; noise-free unless noise is set).  Returns
    (serve.Request, truth deputy state, RK4 work of one solve in particle steps, the
    generator's scenario: unphased chief, phase, truth offset)."""
    import numpy as np

    from paper_2207_13175_gb300 import api
    from paper_2207_13175_gb300 import inputs as I
    from paper_2207_13175_gb300.serve import Request
    rng = np.random.default_rng(seed)
    out = []
    for j in range(n):
        sc = I.batched_instance(rng, j, noise=noise)
        ph = sc.meta["phase_tu"]
        # the chief's state at its random phase: DOPRI5 propagation of the corrected IC
        with api.Problem(sc.mu, sc.chief, np.array([ph]), np.zeros((1, 2)), sc.sigma,
                         api.bounds_from_chief(sc.chief, 1.0, 1.0, I.L_KM, I.TU_S),
                         api.options(integrator=api.DOPRI5, rtol=1e-13, atol=1e-13)) as P:
            chief = P.propagate(sc.chief[None, :]).cpu().numpy()[0, :, 0]
        deputy = chief + sc.deputy
        ang, _ = api.simulate_obs(sc.mu, chief, deputy, sc.t, sc.noise)
        b = api.bounds_from_chief(chief, sc.r_max_km, sc.v_max_ms, I.L_KM, I.TU_S)
        work = sc.m * (sc.iters + 1) * rk4_steps_per_eval(sc.t, sc.dt)
        out.append((Request(sc.mu, chief, sc.t, ang, sc.sigma, b, sc.m, sc.iters, sc.seed), deputy, work, sc))
    return out


def rk4_steps_per_eval(t, dt):
    """RK4 steps of one propagation under the interval rule (n_k = max(1, ceil(span/dt -
    1e-9)) per interval; none for an empty span).  Used only to weight samples."""
    import math
    n, prev = 0, 0.0
    for tk in t:
        span = float(tk) - prev
        if span != 0.0:
            n += max(1, math.ceil(span / dt - 1e-9))
        prev = float(tk)
    return n


def pos_err_km(state, deputy):
    import numpy as np

    from paper_2207_13175_gb300 import inputs as I
    return float(np.linalg.norm(np.asarray(state)[:3] - np.asarray(deputy)[:3]) * I.L_KM)


def run_batch(reqs, opts, block=None, budget=32 << 30, dts=None):
    """Solve requests as one batch under the persistent scheduler; returns (results,
    wall seconds, stats).  dts: (size classes, RK4 step bound per class)."""
    import torch

    from paper_2207_13175_gb300 import api
    B = api.Batch(opts, budget_bytes=budget, max_resident=1024)
    if block is not None:
        B.set_block_sizes([1 << 30], [block])
    if dts is not None:
        B.set_step_sizes(*dts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tk = [B.submit(q.mu, q.chief, q.t, q.angles, q.sigma, q.bounds, q.m, q.iters, q.w, q.c1, q.c2,
                   q.seed) for q in reqs]
    for _ in range(100):
        B.run(0.0)                   # persistent scheduling to completion
        if all(B.poll(t) is not None for t in tk):
            break
    else:
        raise RuntimeError("batch did not finish")
    wall = time.perf_counter() - t0
    res = [B.poll(t) for t in tk]
    st = B.stats()
    B.close()
    return res, wall, st


def head_to_head_fields(h):
    """Top-level fields of the head-to-head: solves/s (all, and counting only solves at
    <= 1 km from the truth) of the batched mixed form, the plain FP64 form one at a time
    and the served form at each load, with latencies and the alone floor."""
    import numpy as np
    out = {"h2h_instances": h["instances"], "h2h_noise": h["noise"],
           "batched_mixed_solves_per_s": h["batch_solves_per_s"],
           "batched_mixed_solves_per_s_le_1km": h["batch_solves_per_s_le_1km"],
           "batched_mixed_frac_le_1km": h["frac_within_1km"],
           "batched_mixed_swarm_only_frac_le_1km": h["swarm_only_frac_within_1km"],
           "h2h_refine_iters": h["refine_iters"],
           "batched_mixed_fp64_fallbacks": h["fp64_fallbacks"],
           "batched_mixed_dt_by_class": h["autotuned_dt_by_class"],
           "fp64_alone_solves_per_s": h["fp64_one_at_a_time_solves_per_s"],
           "fp64_alone_solves_per_s_le_1km": h["fp64_one_at_a_time_solves_per_s_le_1km"],
           "fp64_alone_frac_le_1km": h["fp64_one_at_a_time_frac_within_1km"],
           "fp64_alone_sample_work_ratio": h["fp64_sample_work_ratio"],
           "speedup_batched_vs_fp64": h["speedup_batched_mixed_vs_fp64_one_at_a_time"],
           "speedup_batched_vs_fp64_le_1km": h["speedup_le_1km"],
           "batched_mixed_subset_solves_per_s_le_1km": h["headline_form_on_variant_subset"]["batch_solves_per_s_le_1km"],
           "batched_mixed_fixed_dt_solves_per_s_le_1km": (h["fixed_dt_5e-4"] or {}).get("batch_solves_per_s_le_1km"),
           "batched_mixed_fp64_last_iters": h["fp64_last_iters"],
           "batched_mixed_fp32_peak_frac": h["roofline"]["frac"],
           "batched_mixed_fp64_tail_50_solves_per_s_le_1km": (h["fp64_tail_50"] or {}).get("batch_solves_per_s_le_1km"),
           "fp64_alone_tuned_dt_solves_per_s": h["fp64_one_at_a_time_tuned_dt_solves_per_s"],
           "speedup_batched_vs_fp64_tuned_dt": h["speedup_batched_mixed_vs_fp64_tuned_dt"],
           "mixed_vs_fp64_pos_km_median": float(np.median(h["mixed_batch_vs_fp64_pos_km"])),
           "mixed_vs_fp64_pos_km_max": float(np.max(h["mixed_batch_vs_fp64_pos_km"]))}
    for r in h.get("serving", []):
        tag = r["label"]
        out[tag + "_solves_per_s"] = r["solves_per_s"]
        out[tag + "_solves_per_s_le_1km"] = r["solves_per_s_le_1km"]
        out[tag + "_frac_le_1km"] = r["frac_within_1km"]
        out[tag + "_p50_s"] = r["latency_p50_s"]
        out[tag + "_p99_s"] = r["latency_p99_s"]
        out[tag + "_alone_p50_s"] = r["alone_latency_p50_s"]
        out[tag + "_alone_p99_s"] = r["alone_latency_p99_s"]
        out[tag + "_arrival_per_s"] = r["arrival_rate_per_s"]
        out[tag + "_queued_max"] = r["queued_max"]
    return out


def batched_and_serving_leg(args):
    """The head-to-head on noise-free instances of the batched workload (10-400 epochs
    over 1-7 days, 1,024 / 4,096 / 16,384 particles, 100-500 iterations): the mixed
    FP32/FP64 form solved as one batch, against the plain FP64 form one problem at a
    time on a seeded uniform sample of the same instances; solves/s counted at <= 1 km
    from the truth.  Then the serving loop on fresh seeded instances with Poisson
    arrivals at fractions of the measured batch capacity, beside the latency of a sample
    of the same requests run alone."""
    import numpy as np
    import torch

    from paper_2207_13175_gb300 import api
    from paper_2207_13175_gb300 import inputs as I
    from paper_2207_13175_gb300.serve import serve
    inst = batched_instances(args.batch_instances, seed=7, noise=False)
    reqs = [r for r, _, _, _ in inst]
    work = np.array([w for _, _, w, _ in inst], dtype=float)
    # a solve is the paper's pipeline: the swarm, then Levenberg-Marquardt from its best
    last = args.mixed_fp64_last if args.refine_iters > 0 else 50
    gate = args.refine_gate if args.refine_iters > 0 else 0.0
    opts = api.options(dt=5e-4, precision=api.MIXED, fp64_last_iters=last, refine_iters=args.refine_iters,
                       refine_gate=gate)
    B = api.Batch(opts, budget_bytes=32 << 30, max_resident=1024)
    # autotuner: one sample per size class, one block size for the persistent scheduler
    classes = [1024, 4096, 16384]
    samples = []
    for m in classes:
        q = next((q for q in reqs if q.m == m), reqs[0])
        samples.append((q.mu, q.chief, q.t, q.angles, q.sigma, q.bounds, q.m, q.iters, q.seed))
    log(f"batched leg: {len(reqs)} noise-free instances prepared")
    # step size per class first (checked against a DOPRI5 reference of each class's
    # sample: lines of sight within a tenth of the 1 arcsec noise), then the block size
    dt_cands = [float(v) for v in args.dt_candidates.split(",")]
    if args.tune_dt:
        dt_tuned, dt_err = B.autotune_dt(classes, samples, dt_cands, 0.1 * I.ARCSEC, n_probe=64)
    else:
        dt_tuned, dt_err = [5e-4] * len(classes), np.zeros((len(classes), 0))
        B.set_step_sizes(classes, dt_tuned)
    tuned, tune_ms = B.autotune(classes, samples, candidates=(64, 128, 256), uniform=True)
    B.close()
    log(f"autotuned step sizes {dt_tuned}, block size {tuned[0]}")
    dts = (classes, dt_tuned)
    res, wall, st = run_batch(reqs, opts, block=tuned[0], dts=dts)
    log(f"batch solved in {wall:.1f} s")
    # the variants on the first nv instances, beside the headline form on the same subset
    nv = min(args.variant_instances, len(reqs))
    sub_reqs, sub_inst = reqs[:nv], inst[:nv]

    def variant(o, d):
        r_v, w_v, _ = run_batch(sub_reqs, o, block=tuned[0], dts=d)
        e_v = np.array([pos_err_km(r["state"], dep) for r, (_, dep, _, _) in zip(r_v, sub_inst)])
        return r_v, {"instances": nv, "batch_wall_s": w_v, "batch_solves_per_s": nv / w_v,
                     "batch_solves_per_s_le_1km": float((e_v <= 1.0).sum()) / w_v,
                     "frac_within_1km": float((e_v <= 1.0).mean())}

    res_s, same_subset = variant(opts, dts)
    log(f"headline form on the first {nv} instances in {same_subset['batch_wall_s']:.1f} s")
    fixed = None
    if args.tune_dt:
        # at the plain form's fixed step (5e-4)
        _, fixed = variant(opts, (classes, [5e-4] * len(classes)))
        log(f"the same at the fixed step in {fixed['batch_wall_s']:.1f} s")
    tail50 = None
    if last != 50:
        # with 50 FP64 swarm iterations before the refinement
        o50 = api.options(dt=5e-4, precision=api.MIXED, fp64_last_iters=50, refine_iters=args.refine_iters,
                          refine_gate=gate)
        res_t, tail50 = variant(o50, dts)
        dif_t = np.array([np.linalg.norm(a["state"][:3] - b["state"][:3]) * I.L_KM for a, b in zip(res_s, res_t)])
        tail50.update(final_pos_diff_km_max=float(dif_t.max()), final_pos_diff_km_median=float(np.median(dif_t)))
        log(f"the same with 50 FP64 iterations in {tail50['batch_wall_s']:.1f} s")
    steps = sum(r["rk_steps"] for r in res)
    # the batch's algorithmic work: RK4 steps, per-evaluation epochs (the initial swarm,
    # every iteration and the FP64 rescoring of the personal bests) and moves; the
    # refinement's few propagations are left out
    flop = float(sum(r["rk_steps"] * FLOP_PER_STEP + q.m * (q.iters + 2) * q.t.size * FLOP_PER_EPOCH
                     + q.m * q.iters * FLOP_PER_MOVE for r, q in zip(res, reqs)))
    batch_roofline = {"bound": "alu", "achieved": flop / wall / 1e12, "peak": FP32_PEAK_TFLOPS,
                      "unit": "TFLOP/s", "frac": flop / wall / 1e12 / FP32_PEAK_TFLOPS,
                      "flop": flop, "issued_frac": steps * FLOP32_ISSUED_PER_STEP / wall / 1e12 / FP32_PEAK_TFLOPS,
                      "basis": f"{FLOP_PER_STEP} per RK4 step, {FLOP_PER_EPOCH} per epoch, {FLOP_PER_MOVE} per "
                               f"move, over the launch's wall time, against the derived FP32 peak (the "
                               f"iterations are FP32; issued_frac counts the {FLOP32_ISSUED_PER_STEP} FP32 "
                               f"operations the Encke form issues per step)"}
    err = np.array([pos_err_km(r["state"], dep) for r, (_, dep, _, _) in zip(res, inst)])
    err_pso = np.array([pos_err_km(r["pso_state"], dep) for r, (_, dep, _, _) in zip(res, inst)])
    le = err <= 1.0
    capacity = len(reqs) / wall
    fb = [int(i) for i, r in enumerate(res) if r.get("fallback")]
    out = {"instances": len(reqs), "noise": "none", "refine_iters": args.refine_iters,
           "refine_gate_per_epoch": gate, "fp64_fallbacks": len(fb), "fp64_fallback_indices": fb,
           "autotuned_dt_by_class": dict(zip([str(c) for c in classes], dt_tuned)),
           "autotune_dt_candidates": dt_cands, "autotune_dt_angle_err_rad": np.asarray(dt_err).tolist(),
           "autotune_dt_budget_rad": 0.1 * I.ARCSEC, "headline_form_on_variant_subset": same_subset,
           "fixed_dt_5e-4": fixed, "fp64_last_iters": last, "fp64_tail_50": tail50,
           "swarm_only_frac_within_1km": float((err_pso <= 1.0).mean()),
           "swarm_only_pos_err_km_median": float(np.median(err_pso)),
           "autotuned_block": tuned[0], "autotune_weighted_ms": tune_ms.tolist(),
           "threads_per_particle_by_class": {str(c): 1 for c in classes},
           "threads_per_particle_note": "one thread per particle in every class: the batch's iterations are "
                                        "FP32 (the two primaries already share packed FP32x2 instructions); "
                                        "lane pairs exist for FP64 circular problems, where each lane of a pair "
                                        "issues half the gravity instructions",
           "workload": "batched: 10-400 angle pairs over 1-7 d, swarms 1,024/4,096/16,384, "
                       f"100-500 iterations, mixed precision (FP32, the personal bests rescored "
                       f"in FP64, then {last} FP64 iterations), RK4 step autotuned per class, then "
                       f"Levenberg-Marquardt (up to {args.refine_iters} iterations, FP64); "
                       f"{len(reqs)} seeded noise-free instances",
           "batch_wall_s": wall, "batch_solves_per_s": capacity,
           "batch_solves_per_s_le_1km": float(le.sum()) / wall,
           "batch_rk_steps_per_s": steps / wall, "roofline": batch_roofline,
           "mem_high_water_bytes": int(st["bytes_high_water"]),
           "pos_err_km_median": float(np.median(err)), "pos_err_km_max": float(err.max()),
           "frac_within_1km": float(le.mean())}
    # the plain FP64 form one problem at a time (create, solve, read the result) on a
    # seeded uniform sample of the same instances
    k = min(args.fp64_sample, len(reqs))
    pick = np.sort(np.random.default_rng(17).choice(len(reqs), size=k, replace=False))
    fp64 = api.options(dt=5e-4)

    def fp64_solve(q, o=fp64):
        """The plain FP64 form of one solve: create, swarm, refine, result."""
        with api.Problem(q.mu, q.chief, q.t, q.angles, q.sigma, q.bounds, o) as G:
            G.run(q.m, q.iters, q.w, q.c1, q.c2, q.seed)
            r1 = G.result(trace=False)
            x = r1["state"]
            if args.refine_iters > 0:
                x, _, _ = G.refine(r1["state"], args.refine_iters)
        return r1["state"], x

    t_one, err1, diff, err1_pso = [], [], [], []
    states64 = {}
    for i in pick:
        q, dep = reqs[i], inst[i][1]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x_pso, x = fp64_solve(q)
        t_one.append(time.perf_counter() - t0)
        err1.append(pos_err_km(x, dep))
        err1_pso.append(pos_err_km(x_pso, dep))
        diff.append(float(np.linalg.norm(x[:3] - res[i]["state"][:3]) * I.L_KM))
        states64[int(i)] = x.tolist()
    t_one = np.array(t_one)
    err1 = np.array(err1)
    le1 = err1 <= 1.0
    # the same sample in plain FP64 at the batch's autotuned step of its size class (the
    # like-for-like comparison of precision and batching alone)
    dt_of = dict(zip(classes, dt_tuned))
    t_tuned, err_tuned = [], []
    for i in pick:
        q, dep = reqs[i], inst[i][1]
        o = api.options(dt=float(dt_of.get(q.m, 5e-4)))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, x = fp64_solve(q, o)
        t_tuned.append(time.perf_counter() - t0)
        err_tuned.append(pos_err_km(x, dep))
    t_tuned, err_tuned = np.array(t_tuned), np.array(err_tuned)
    work_tuned = np.array([q.m * (q.iters + 1) * rk4_steps_per_eval(q.t, dt_of.get(q.m, 5e-4))
                           for q in reqs], dtype=float)
    ratio_tuned = float(work_tuned[pick].mean() / work_tuned.mean())
    rate_tuned = k / t_tuned.sum() * ratio_tuned
    # a uniform sample's solve times, scaled to the whole set by its share of the set's
    # RK4 work (the ratio estimator of the set's total time); the plain sample rate beside
    work_ratio = float(work[pick].mean() / work.mean())
    fp64_rate_sample = k / t_one.sum()
    fp64_rate = fp64_rate_sample * work_ratio
    log(f"FP64 one at a time: {k} sampled solves in {t_one.sum():.1f} s")
    out.update({
        "fp64_one_at_a_time_solves_per_s": fp64_rate,
        "fp64_one_at_a_time_solves_per_s_le_1km": fp64_rate * float(le1.mean()),
        "fp64_one_at_a_time_frac_within_1km": float(le1.mean()),
        "fp64_one_at_a_time_sample": f"seeded uniform sample of {k} of {len(reqs)} instances "
                                     f"(indices {pick.tolist()}); sample mean work / set mean work = "
                                     f"{work_ratio:.3f}; each solve (create, swarm, refinement, "
                                     "result) timed on the host clock; the set's rate is the "
                                     "sample's rate times that work ratio",
        "fp64_one_at_a_time_solves_per_s_sample": fp64_rate_sample,
        "fp64_one_at_a_time_tuned_dt_solves_per_s": rate_tuned,
        "fp64_one_at_a_time_tuned_dt_frac_within_1km": float((err_tuned <= 1.0).mean()),
        "fp64_one_at_a_time_tuned_dt_work_ratio": ratio_tuned,
        "fp64_one_at_a_time_tuned_dt_s": t_tuned.tolist(),
        "speedup_batched_mixed_vs_fp64_tuned_dt": capacity / rate_tuned,
        "fp64_sample_indices": pick.tolist(),
        "fp64_sample_work_ratio": work_ratio,
        "fp64_sample_s": t_one.tolist(),
        "fp64_one_at_a_time_pos_err_km": err1.tolist(),
        "fp64_one_at_a_time_swarm_only_pos_err_km": err1_pso,
        "batched_pos_err_km_same_instances": err[pick].tolist(),
        "mixed_batch_vs_fp64_pos_km": diff,
        "fp64_states": states64,
        "speedup_batched_mixed_vs_fp64_one_at_a_time": capacity / fp64_rate,
        "speedup_le_1km": (float(le.sum()) / wall) / max(fp64_rate * float(le1.mean()), 1e-300),
    })
    lm_it = [r["refine_iters"] for r in res]
    out["instances_beyond_1km"] = [{"index": int(i), "m": reqs[i].m, "iters": reqs[i].iters,
                                    "n_obs": int(reqs[i].t.size), "arc_days": float(reqs[i].t[-1] / I.DAY_TU),
                                    "pos_err_km": float(err[i]), "swarm_pos_err_km": float(err_pso[i]),
                                    "lm_iters": int(lm_it[i])} for i in np.nonzero(~le)[0]]
    out["instance_records"] = [{"m": q.m, "iters": q.iters, "n_obs": int(q.t.size),
                                "arc_days": float(q.t[-1] / I.DAY_TU), "work": float(w),
                                "pos_err_km": float(e)} for q, (_, _, w, _), e in zip(reqs, inst, err)]
    # the cheapest instances, also solved in FP64 one at a time, for the oracle's
    # comparison in the CPU-baseline leg (the oracle solves them there from its own inputs)
    sub = np.argsort(work, kind="stable")[:args.oracle_subset]
    fp64_sub = {}
    for i in sub:
        fp64_sub[int(i)] = fp64_solve(reqs[i])[1]
    out["_oracle_subset"] = [{"index": int(i), "sc": inst[i][3], "deputy": inst[i][1],
                              "mixed_state": res[i]["state"], "fp64_state": fp64_sub[int(i)],
                              "work": float(work[i]), "refine_iters": args.refine_iters} for i in sub]
    # serving: fresh seeded instances, Poisson arrivals at fractions of the batch capacity
    serving = []
    loads = [(float(v) * capacity, float(v), "served_" + f"{float(v):.2f}x".replace(".", "p"))
             for v in args.serve_loads.split(",") if v]
    loads += [(float(v), float(v) / capacity, "served_rate" + f"{float(v):g}".replace(".", "p"))
              for v in args.serve_rates.split(",") if v]
    for j, (rate, frac, label) in enumerate(loads):
        n_req = min(args.serve_max_requests, max(8, int(rate * 20)))
        fresh = batched_instances(n_req, seed=100 + j, noise=False)
        sreq = [q for q, _, _, _ in fresh]
        arr = I.poisson_arrivals(rate, n_req, seed=11 + j)
        B = api.Batch(opts, budget_bytes=32 << 30, max_resident=1024)
        B.set_block_sizes([1 << 30], [tuned[0]])
        B.set_step_sizes(*dts)
        r = serve(B, sreq, arr, slice_s=0.05, timeout_s=600.0)
        B.close()
        results = r.pop("results")
        r["fp64_fallbacks"] = sum(int(x.get("fallback", 0)) for x in results)
        e_s = np.array([pos_err_km(x["state"], dep) for x, (_, dep, _, _) in zip(results, fresh)])
        e_sp = np.array([pos_err_km(x["pso_state"], dep) for x, (_, dep, _, _) in zip(results, fresh)])
        lat = np.array(r.pop("latencies_s"))
        log(f"serving at {rate:.2f}/s ({frac:.2f} x capacity): {n_req} requests in {r['wall_s']:.1f} s")
        # the floor: a seeded sample of the same requests, each run alone (a batch of one)
        ka = min(args.alone_sample, n_req)
        pa = np.sort(np.random.default_rng(23 + j).choice(n_req, size=ka, replace=False))
        alone = []
        for i in pa:
            _, w_alone, _ = run_batch([sreq[i]], opts, block=tuned[0], dts=dts)
            alone.append(w_alone)
        alone = np.array(alone)
        r.update({"label": label, "load_vs_capacity": frac, "arrival_rate_per_s": rate, "noise": "none",
                  "solves_per_s_le_1km": float((e_s <= 1.0).sum()) / r["wall_s"],
                  "frac_within_1km": float((e_s <= 1.0).mean()),
                  "swarm_only_frac_within_1km": float((e_sp <= 1.0).mean()),
                  "pos_err_km_median": float(np.median(e_s)),
                  "alone_sample": pa.tolist(), "alone_latency_s": alone.tolist(),
                  "alone_latency_p50_s": float(np.percentile(alone, 50)),
                  "alone_latency_p99_s": float(np.percentile(alone, 99)),
                  "served_over_alone_latency_median": float(np.median(lat[pa] / alone))})
        serving.append(r)
    out["serving"] = serving
    return out


# the paper's Table 1 (PSO, then its nonlinear least squares), for context: its swarm
# size, iteration count, noise level and cost weights are not stated
PAPER_TABLE1 = {1: {"pso_range_km": 0.3276, "nlsq_range_km": 0.0304, "pso_speed_kms": 2.84e-6,
                    "nlsq_speed_kms": 3.40e-8, "pso_min_cost": 0.0493, "nlsq_min_cost": 8.56e-11},
                2: {"pso_range_km": 6.072, "nlsq_range_km": 0.0177, "pso_speed_kms": 3.27e-5,
                    "nlsq_speed_kms": 5.77e-8, "pso_min_cost": 1.667, "nlsq_min_cost": 7.34e-11}}


def paper_table_leg(stream, dev, m=16384, iters=300):
    """The paper's two printed geometries (L2 southern halo deputy; chief on the L2 halo
    with 35 epochs, or on the L2 axial orbit with 10 epochs; 7 days; box +-250 km /
    +-0.1 km/s about the true deputy), noise-free and with 1 arcsec noise: one FP64
    swarm solve, then Levenberg-Marquardt refinement of its global best, with the
    truth errors beside the paper's Table 1."""
    import numpy as np
    import torch

    from paper_2207_13175_gb300 import api
    from paper_2207_13175_gb300 import inputs as I
    out = []
    for scen in (1, 2):
        for noise in (False, True):
            sc = I.paper_table(scen, noise=noise)
            ang, _ = api.simulate_obs(sc.mu, sc.chief, sc.deputy, sc.t, sc.noise)
            bounds = api.bounds_from_chief(sc.deputy, sc.r_max_km, sc.v_max_ms, I.L_KM, I.TU_S)
            opts = api.options(dt=sc.dt)
            with api.Problem(sc.mu, sc.chief, sc.t, ang, sc.sigma, bounds, opts, stream=stream) as G:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize(dev)
                e0.record(stream)
                G.run(m, iters, sc.w, sc.c1, sc.c2, sc.seed)
                e1.record(stream)
                r = G.result(trace=False)
                t_pso = e0.elapsed_time(e1) / 1e3
                t0 = time.perf_counter()
                x, c, it = G.refine(r["state"], 50)
                t_lm = time.perf_counter() - t0
                J_truth = float(G.eval(sc.deputy[None, :]).cpu()[0])

            def err(s):
                return (float(np.linalg.norm(s[:3] - sc.deputy[:3]) * I.L_KM),
                        float(np.linalg.norm(s[3:] - sc.deputy[3:]) * I.L_KM / I.TU_S))
            (rp, vp), (rl, vl) = err(r["state"]), err(x)
            log(f"paper scenario {scen}, noise {noise}: swarm {t_pso:.1f} s, {rp:.3f} km -> {rl:.4f} km")
            out.append({"scenario": scen, "noise_arcsec": 1.0 if noise else 0.0, "n_obs": sc.n_obs,
                        "particles": m, "iterations": iters,
                        "pso_range_km": rp, "pso_speed_kms": vp, "pso_min_cost": r["cost"],
                        "lm_range_km": rl, "lm_speed_kms": vl, "lm_cost": c, "lm_iterations": it,
                        "cost_at_truth": J_truth, "pso_s": t_pso, "lm_s": t_lm,
                        "paper": PAPER_TABLE1[scen]})
    return {"workload": "the paper's scenarios 1 and 2 (Tables 2-3), FP64 swarm of "
                        f"{m} particles x {iters} iterations, then Levenberg-Marquardt (50 at most); "
                        "costs use 1 arcsec weights", "runs": out}


def end_to_end(args, sc, ang, bounds, opts, stream, dev, world):
    """The same metric through the public API: pinned host inputs -> create ->
    initialise and one iteration -> result back to the host -> destroy, every step."""
    import numpy as np
    import torch

    from paper_2207_13175_gb300 import api
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).pin_memory().numpy()
    h_t, h_ang, h_chief = pin(sc.t), pin(ang), pin(sc.chief)
    h_sig, h_b = pin(np.asarray(sc.sigma)), pin(bounds)
    e2e_steps = max(1, min(args.steps, 10))
    G = api.Problem(sc.mu, h_chief, h_t, h_ang, h_sig, h_b, opts, stream=stream)
    G.run(sc.m, 1, sc.w, sc.c1, sc.c2, sc.seed)
    G.result(trace=False)
    G.close()
    barrier(world)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    done = 0
    for k in range(e2e_steps):
        G = api.Problem(sc.mu, h_chief, h_t, h_ang, h_sig, h_b, opts, stream=stream)
        G.run(sc.m, 1, sc.w, sc.c1, sc.c2, sc.seed + k)
        res = G.result(trace=False)
        done += res["rk_steps"]
        G.close()
    torch.cuda.synchronize(dev)
    barrier(world)
    e2e_s, e2e_units = aggregate(time.perf_counter() - t0, float(done), world)
    h2d = 8 * (h_t.size + h_ang.size + h_chief.size + h_sig.size + h_b.size)
    d2h = 96    # the device-side global best record read back by iod_result
    return {"value": e2e_units / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "steps": e2e_steps,
            "step": "create + initialise + 1 iteration + result + destroy"}


if __name__ == "__main__":
    sys.exit(main())
