"""The sharded-swarm driver on CPU.

A swarm's particles interact only through the global best, so a swarm split by particle
range over several engines, with the best (cost, index) over the shards exchanged after
every iteration, must reproduce the unsharded swarm exactly.  The engine here is a small
numpy swarm with the library's rules (random numbers keyed by the whole-swarm index, the
lowest index winning equal costs, a record replaced only on a strict improvement) and a
coarsely quantised cost, so that equal costs across shards are common.  The driver runs it
in one process (several shards, in-process exchange) and as two gloo ranks (the exchange
over torch.distributed), and both must match the one-engine run bit for bit.  The option
checks of the library's sharded problems run here too (they precede any device work)."""
import ctypes as C
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TARGET = np.array([0.3, -0.2, 0.1, 0.05, -0.4, 0.25])
LO, HI = -np.ones(6), np.ones(6)


class ToyShard:
    """Particles offset .. offset+m-1 of a swarm of `total` (one engine = one problem)."""

    def __init__(self, offset=0, total=None):
        self.offset = offset
        self.total = total

    def _u(self, gi, n, stream, k):
        return np.random.default_rng([self.seed, gi, n, stream]).random(k)

    def _cost(self, X):
        return 1.0 + np.round(((X - TARGET) ** 2).sum(1) * 50.0) / 50.0   # quantised: frequent ties

    def _best_update(self, init):
        order = np.lexsort((np.arange(self.m), self.pJ))
        bj, bi = self.pJ[order[0]], order[0]
        if init or bj < self.gJ:
            self.gJ, self.gidx, self.g = bj, int(bi) + self.offset, self.P[bi].copy()
        self.trace.append((self.gJ, self.gidx))

    def run(self, m, iters, w, c1, c2, seed):
        self.m, self.w, self.c1, self.c2, self.seed, self.n = m, w, c1, c2, seed, 0
        gi = self.offset + np.arange(m)
        U = np.stack([self._u(i, 0, 2, 6) for i in gi])
        self.X = LO + U * (HI - LO)
        self.V = np.zeros_like(self.X)
        self.P = self.X.copy()
        self.pJ = self._cost(self.X)
        self.evals = m
        self.trace = []
        self._best_update(True)
        self.continue_(iters)

    def continue_(self, iters):
        gi = self.offset + np.arange(self.m)
        for _ in range(iters):
            self.n += 1
            R = np.stack([self._u(i, self.n, 3, 2) for i in gi])
            self.V = (self.w * self.V + self.c1 * R[:, :1] * (self.P - self.X)
                      + self.c2 * R[:, 1:] * (self.g - self.X))
            self.X = np.clip(self.X + self.V, LO, HI)
            J = self._cost(self.X)
            self.evals += self.m
            better = J < self.pJ
            self.P[better] = self.X[better]
            self.pJ[better] = J[better]
            self._best_update(False)

    def gbest_get(self):
        return self.g.copy(), float(self.gJ), int(self.gidx), self.n

    def gbest_set(self, g, gJ, gidx):
        self.g, self.gJ, self.gidx = np.array(g, dtype=np.float64), float(gJ), int(gidx)

    def result(self, trace=False):
        return {"rk_steps": self.evals}


COEF = dict(w=0.72, c1=1.49, c2=1.49, seed=5)


def _unsharded(M, iters):
    t = ToyShard(0, M)
    t.run(M, iters, **COEF)
    return t


def _sharded_local(M, iters, world):
    from paper_2207_13175_gb300 import shard
    shards, counts = [], []
    for r in range(world):
        off, cnt = shard.shard_range(M, world, r)
        shards.append(ToyShard(off, M))
        counts.append(cnt)
    return shard.ShardedSwarm(shards, counts).run(iters, **COEF)


def _assert_same(ref: ToyShard, out: dict):
    assert np.array_equal(out["gcost_trace"], np.array([t[0] for t in ref.trace]))
    assert np.array_equal(out["gidx_trace"], np.array([t[1] for t in ref.trace]))
    assert np.array_equal(out["state"], ref.g) and out["cost"] == ref.gJ
    assert out["gbest_index"] == ref.gidx and out["rk_steps"] == ref.evals


def test_shard_range_covers_the_swarm():
    from paper_2207_13175_gb300 import shard
    for M, world in [(10, 3), (7, 7), (1000, 8), (65536, 3)]:
        parts = [shard.shard_range(M, world, r) for r in range(world)]
        assert parts[0][0] == 0
        for (o0, c0), (o1, _) in zip(parts, parts[1:]):
            assert o1 == o0 + c0
        assert sum(c for _, c in parts) == M
        assert max(c for _, c in parts) - min(c for _, c in parts) <= 1
    with pytest.raises(ValueError):
        shard.shard_range(2, 3, 0)


def test_best_record_is_lowest_cost_then_lowest_index():
    from paper_2207_13175_gb300 import shard
    recs = np.array([[2.0, 5] + [0.0] * 6, [1.0, 9] + [1.0] * 6, [1.0, 3] + [2.0] * 6,
                     [np.nan, 0] + [3.0] * 6])
    b = shard.best_record(recs)
    assert b[0] == 1.0 and b[1] == 3 and np.all(b[2:] == 2.0)
    allnan = np.array([[np.nan, 4] + [0.0] * 6, [np.nan, 2] + [1.0] * 6])
    assert shard.best_record(allnan)[1] == 2     # +inf ties: the lowest index


@pytest.mark.parametrize("world", [1, 2, 3, 5])
def test_local_shards_equal_one_engine(world):
    ref = _unsharded(101, 12)
    ties = sum(1 for a, b in zip(ref.trace, ref.trace[1:]) if a[0] == b[0])
    assert ties > 0           # the quantised cost does produce repeated bests
    _assert_same(ref, _sharded_local(101, 12, world))


def test_driver_stops_on_algorithm2_test():
    from paper_2207_13175_gb300 import shard
    shards = [ToyShard(*shard.shard_range(64, 2, r)[:1], 64) for r in range(2)]
    counts = [shard.shard_range(64, 2, r)[1] for r in range(2)]
    out = shard.ShardedSwarm(shards, counts).run(200, tol_tau=1e-9, tol_window=5, **COEF)
    tr = out["gcost_trace"]
    n = out["iters_done"]
    assert 5 < n < 200
    assert abs((tr[n] - tr[n - 5]) / tr[n]) < 1e-9
    for k in range(6, n):    # no earlier iteration passed the test
        assert not abs((tr[k] - tr[k - 5]) / tr[k]) < 1e-9


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, M, iters, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist

    from paper_2207_13175_gb300 import shard
    from test_shard_host import ToyShard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    off, cnt = shard.shard_range(M, world, rank)
    out = shard.ShardedSwarm([ToyShard(off, M)], [cnt], shard.torch_allgather()).run(iters, **COEF)
    q.put((rank, out))
    dist.destroy_process_group()


def _rank_two_shards(rank, world, port, M, iters, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist

    from paper_2207_13175_gb300 import shard
    from test_shard_host import ToyShard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    shards, counts = [], []
    for r in (2 * rank, 2 * rank + 1):      # two shards per rank, four in all
        off, cnt = shard.shard_range(M, 2 * world, r)
        shards.append(ToyShard(off, M))
        counts.append(cnt)
    out = shard.ShardedSwarm(shards, counts, shard.torch_allgather()).run(iters, **COEF)
    q.put((rank, out))
    dist.destroy_process_group()


def test_two_gloo_ranks_with_two_shards_each():
    """Several shards per rank: each rank contributes its shards' records to the
    all-gather, and the result still equals the one-engine run."""
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    M, iters = 91, 8
    procs = [ctx.Process(target=_rank_two_shards, args=(r, 2, port, M, iters, q)) for r in range(2)]
    for p in procs:
        p.start()
    outs = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = _unsharded(M, iters)
    for r in range(2):
        _assert_same(ref, outs[r])


def test_two_gloo_ranks_equal_one_engine():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    M, iters = 77, 10
    procs = [ctx.Process(target=_rank, args=(r, 2, port, M, iters, q)) for r in range(2)]
    for p in procs:
        p.start()
    outs = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = _unsharded(M, iters)
    for r in range(2):
        _assert_same(ref, outs[r])


# ----------------------------------------------------------------- library option checks
def _create(**kw):
    from paper_2207_13175_gb300 import _native as N
    lib = N.lib()
    chief = np.array([0.85, 0, 0.17, 0, 0.26, 0.0])
    t = np.linspace(0.0, 0.23, 20)
    ang = np.tile([0.1, 0.2], (20, 1))
    sigma = np.array([4.8e-6, 4.8e-6])
    d = np.array([2.6e-4] * 3 + [9.8e-4] * 3)
    bounds = np.concatenate([chief - d, chief + d])
    D = C.POINTER(C.c_double)
    keep = [np.ascontiguousarray(a) for a in (chief, t, ang, sigma, bounds)]
    ptrs = [a.ctypes.data_as(D) for a in keep]
    o = N.Options()
    assert lib.iod_options_default(C.byref(o)) == 0
    assert o.shard_offset == 0 and o.shard_total == 0
    for k, v in kw.items():
        setattr(o, k, v)
    h = C.c_void_p(123)
    rc = lib.iod_create(0.01215058560962404, ptrs[0], 20, ptrs[1], ptrs[2], ptrs[3], ptrs[4],
                        C.byref(o), C.byref(h))
    return rc, h.value, lib.iod_last_error().decode()


@pytest.mark.parametrize("kw,word", [
    (dict(shard_offset=3), "shard_offset"),
    (dict(shard_total=-1), "shard_offset"),
    (dict(shard_offset=-1, shard_total=10), "shard_offset"),
    (dict(shard_offset=10, shard_total=10), "shard_offset"),
    (dict(shard_offset=0, shard_total=10, precision=1), "IOD_FP64"),
    (dict(shard_offset=0, shard_total=10, tol_tau=1e-6), "tol_tau"),
])
def test_sharded_options_refused(kw, word):
    rc, h, msg = _create(**kw)
    assert rc == -1 and not h and word in msg


def test_batch_refuses_sharded_options():
    from paper_2207_13175_gb300 import _native as N
    lib = N.lib()
    o = N.Options()
    lib.iod_options_default(C.byref(o))
    o.shard_total = 4
    b = C.c_void_p(7)
    rc = lib.iod_batch_create(C.byref(o), 1 << 30, 4, C.byref(b))
    assert rc == -1 and "sharded" in lib.iod_last_error().decode()
