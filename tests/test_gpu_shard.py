"""One swarm sharded by particle range over several problems reproduces the unsharded
swarm bit for bit: global best trace (cost and whole-swarm index), final state, step
counts and every particle's position, velocity and personal best, for even and ragged
splits, the swarm variants (stratified start, random start velocities, per-dimension
random numbers, Algorithm 1's lagged global best), DOPRI5, the balanced schedule, and
Algorithm 2's stopping test run by the driver on the exchanged costs.  The shards live in
one process here (the exchange is in-process); the same driver over torch.distributed
ranks is tested on CPU."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _case():
    import scenarios as S
    from paper_2207_13175_gb300 import inputs as I
    sc = I.tiny(1)
    pair = S.Pair(sc)
    return sc, pair.bounds, np.stack([pair.ra, pair.dec], 1)


def _unsharded(sc, bounds, ang, M, iters, seed, **kw):
    from paper_2207_13175_gb300 import api
    opts = api.options(dt=sc.dt, **kw)
    with api.Problem(sc.mu, sc.chief, sc.t, ang, sc.sigma, bounds, opts) as P:
        P.run(M, iters, w=sc.w, c1=sc.c1, c2=sc.c2, seed=seed)
        return P.result(), P.swarm_get()


def _sharded(sc, bounds, ang, M, world, iters, seed, tol=None, **kw):
    from paper_2207_13175_gb300 import api, shard
    probs, counts = [], []
    try:
        for r in range(world):
            off, cnt = shard.shard_range(M, world, r)
            opts = api.options(dt=sc.dt, shard_offset=off, shard_total=M, record_trace=0, **kw)
            probs.append(api.Problem(sc.mu, sc.chief, sc.t, ang, sc.sigma, bounds, opts))
            counts.append(cnt)
        extra = {} if tol is None else dict(tol_tau=tol[0], tol_window=tol[1])
        out = shard.ShardedSwarm(probs, counts).run(iters, w=sc.w, c1=sc.c1, c2=sc.c2, seed=seed,
                                                    **extra)
        swarms = [p.swarm_get() for p in probs]
        return out, swarms
    finally:
        for p in probs:
            p.close()


def _assert_same(ref, out, swarms):
    r, w = ref
    assert out["iters_done"] == r["iters_done"]
    assert np.array_equal(out["gcost_trace"], r["gcost_trace"])
    assert np.array_equal(out["gidx_trace"], r["gidx_trace"])
    assert np.array_equal(out["state"], r["state"]) and out["cost"] == r["cost"]
    assert out["gbest_index"] == r["gbest_index"]
    assert out["rk_steps"] == r["rk_steps"]
    for k in ("x", "v", "p"):
        assert np.array_equal(np.concatenate([s[k] for s in swarms], 1), w[k]), k
    for k in ("pJ", "J"):
        assert np.array_equal(np.concatenate([s[k] for s in swarms]), w[k]), k


@pytest.mark.parametrize("M,world", [(1000, 2), (1000, 3), (257, 4)])
def test_sharded_equals_unsharded(M, world):
    sc, bounds, ang = _case()
    ref = _unsharded(sc, bounds, ang, M, 6, 11)
    out, swarms = _sharded(sc, bounds, ang, M, world, 6, 11)
    _assert_same(ref, out, swarms)


@pytest.mark.parametrize("kw", [
    dict(init_grid=1, velocity_init=1, per_dim_random=1),
    dict(gbest_order=1),
    dict(integrator=1),
    dict(threads_per_particle=2),
])
def test_sharded_variants(kw):
    sc, bounds, ang = _case()
    ref = _unsharded(sc, bounds, ang, 600, 5, 3, **kw)
    out, swarms = _sharded(sc, bounds, ang, 600, 3, 5, 3, **kw)
    _assert_same(ref, out, swarms)


def test_sharded_constriction_and_quartic_cost():
    from paper_2207_13175_gb300 import api, shard
    sc, bounds, ang = _case()
    M, world, iters = 500, 2, 5
    coef = dict(w=1.0, c1=2.05, c2=2.05, seed=4)
    kw = dict(dt=sc.dt, cost_form=1, constriction=1)
    with api.Problem(sc.mu, sc.chief, sc.t, ang, sc.sigma, bounds, api.options(**kw)) as P:
        P.run(M, iters, **coef)
        ref = (P.result(), P.swarm_get())
    probs, counts = [], []
    for r in range(world):
        off, cnt = shard.shard_range(M, world, r)
        probs.append(api.Problem(sc.mu, sc.chief, sc.t, ang, sc.sigma, bounds,
                                 api.options(shard_offset=off, shard_total=M, record_trace=0, **kw)))
        counts.append(cnt)
    out = shard.ShardedSwarm(probs, counts).run(iters, **coef)
    swarms = [p.swarm_get() for p in probs]
    for p in probs:
        p.close()
    _assert_same(ref, out, swarms)


def test_sharded_balanced_schedule():
    """Shards large enough for the balanced FP64 schedule (one resident warp per FP64
    sub-partition); the unsharded swarm runs balanced too."""
    import torch
    from paper_2207_13175_gb300 import api
    sc, bounds, ang = _case()
    warps = 4 * torch.cuda.get_device_properties(0).multi_processor_count
    M = 2 * (32 * warps) + 2 * 77
    ref = _unsharded(sc, bounds, ang, M, 4, 8, schedule=api.SCHED_BALANCED)
    assert ref[0]["schedule"] == api.SCHED_BALANCED
    out, swarms = _sharded(sc, bounds, ang, M, 2, 4, 8, schedule=api.SCHED_BALANCED)
    _assert_same(ref, out, swarms)


def test_sharded_algorithm2_stop_matches_device_test():
    """The unsharded run's device test and the driver's host test on the exchanged costs
    stop at the same iteration."""
    sc, bounds, ang = _case()
    win = 3
    # tau just above the smallest relative change over iterations win+1..30 of the run
    # without the test, so that the test fires at the first iteration reaching it
    free = _unsharded(sc, bounds, ang, 400, 30, 2)[0]["gcost_trace"]
    K = [abs((free[n] - free[n - win]) / free[n]) for n in range(win + 1, 31)]
    tau = float(np.nextafter(min(K), np.inf))
    ref = _unsharded(sc, bounds, ang, 400, 60, 2, tol_tau=tau, tol_window=win)
    assert ref[0]["iters_done"] <= 30      # the test fired
    out, swarms = _sharded(sc, bounds, ang, 400, 2, 60, 2, tol=(tau, win))
    assert out["iters_done"] == ref[0]["iters_done"]
    n = out["iters_done"]
    assert np.array_equal(out["gcost_trace"], ref[0]["gcost_trace"][: n + 1])
    assert np.array_equal(out["state"], ref[0]["state"])


def test_gbest_set_is_what_the_next_move_uses():
    """A shard that is handed a global best moves towards it: one shard of a two-shard
    swarm continued with the other shard's best equals the unsharded swarm's particles of
    that range."""
    from paper_2207_13175_gb300 import api
    sc, bounds, ang = _case()
    M = 300
    ref = _unsharded(sc, bounds, ang, M, 1, 6)
    # the global best after initialisation, from the unsharded run's trace
    with api.Problem(sc.mu, sc.chief, sc.t, ang, sc.sigma, bounds, api.options(dt=sc.dt)) as P0:
        P0.run(M, 0, w=sc.w, c1=sc.c1, c2=sc.c2, seed=6)
        g0, gJ0, gi0, it0 = P0.gbest_get()
    assert it0 == 0 and gi0 == ref[0]["gidx_trace"][0] and gJ0 == ref[0]["gcost_trace"][0]
    opts = api.options(dt=sc.dt, shard_offset=100, shard_total=M, record_trace=0)
    with api.Problem(sc.mu, sc.chief, sc.t, ang, sc.sigma, bounds, opts) as Q:
        Q.run(200, 0, w=sc.w, c1=sc.c1, c2=sc.c2, seed=6)
        Q.gbest_set(g0, gJ0, gi0)
        Q.continue_(1)
        s = Q.swarm_get()
    for k in ("x", "v", "p"):
        assert np.array_equal(s[k], ref[1][k][:, 100:]), k
    assert np.array_equal(s["pJ"], ref[1]["pJ"][100:])


_NCCL_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, os.getcwd()); sys.path.insert(0, os.path.join(os.getcwd(), "tests"))
import numpy as np, torch, torch.distributed as dist
from paper_2207_13175_gb300 import api, shard
import scenarios as S
from paper_2207_13175_gb300 import inputs as I
torch.cuda.set_device(0)
dist.init_process_group("nccl", rank=0, world_size=1)
sc = I.tiny(1); pair = S.Pair(sc); ang = np.stack([pair.ra, pair.dec], 1)
M = 700
probs, counts = [], []
for r in range(2):
    off, cnt = shard.shard_range(M, 2, r)
    probs.append(api.Problem(sc.mu, sc.chief, sc.t, ang, sc.sigma, pair.bounds,
                             api.options(dt=sc.dt, shard_offset=off, shard_total=M, record_trace=0)))
    counts.append(cnt)
out = shard.ShardedSwarm(probs, counts, shard.torch_allgather()).run(5, w=sc.w, c1=sc.c1, c2=sc.c2, seed=4)
with api.Problem(sc.mu, sc.chief, sc.t, ang, sc.sigma, pair.bounds, api.options(dt=sc.dt)) as P:
    P.run(M, 5, w=sc.w, c1=sc.c1, c2=sc.c2, seed=4)
    ref = P.result()
dist.destroy_process_group()
same = (np.array_equal(out["gcost_trace"], ref["gcost_trace"]) and np.array_equal(out["gidx_trace"], ref["gidx_trace"])
        and np.array_equal(out["state"], ref["state"]) and out["rk_steps"] == ref["rk_steps"])
with open(os.environ["IOD_TEST_OUT"], "w") as f:
    json.dump({"same": bool(same)}, f)
"""


def test_sharded_exchange_over_nccl(tmp_path):
    """The driver's exchange through NCCL (CUDA tensors; a one-rank group, the only GPU
    count a test here has) with two shards on the rank: equal to the unsharded swarm."""
    import json
    import os
    import socket
    import subprocess
    import sys
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = tmp_path / "nccl_shard.json"
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), NCCL_NVLS_ENABLE="0",
               IOD_TEST_OUT=str(out))
    r = subprocess.run([sys.executable, "-c", _NCCL_SCRIPT], cwd=root, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-3000:]
    assert json.loads(out.read_text())["same"], r.stdout[-2000:]
