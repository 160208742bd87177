"""One swarm sharded by particle range over several problems (ranks, GPUs or streams).

Algorithm 1's particles interact only through the global best g: every other quantity of
a particle (position, velocity, personal best, its random numbers) is its own.  A swarm of
M particles is therefore split into contiguous index ranges, one problem per range
(``iod_options.shard_offset`` / ``shard_total``: the library draws each particle's random
numbers and its init_grid stratum from its index in the whole swarm), and between
iterations the shards agree on g:

* after the initial evaluation and after every iteration each shard reports its own
  global best (cost J, whole-swarm index i, state);
* the whole swarm's best is the lexicographic minimum of (J, i) over the shards -- the
  rule one problem applies over its own particles (lowest index among equal costs), and a
  shard only replaces its record on a strict improvement, as one problem does;
* every shard takes that best before its next iteration.

With that exchange the sharded run reproduces the unsharded run bit for bit (same global
best trace, same final state).  Algorithm 2's stopping test needs the whole swarm's best,
so it runs here, on the exchanged costs, with the device's formula
|(J_n - J_{n-w}) / J_n| < tau for n > w.

The exchange is an all-gather of 8 doubles per shard: ``torch_allgather`` for ranks of a
``torch.distributed`` process group (NCCL or gloo), ``local_allgather`` for several shards
held by one process.
"""
from __future__ import annotations

from typing import Callable, List, Sequence

import numpy as np

# one record per shard: (J, whole-swarm index, g[0..5])
_REC = 8


def shard_range(m_total: int, world: int, rank: int):
    """(offset, count) of rank's contiguous slice of an m_total-particle swarm: the first
    m_total % world ranks hold one particle more."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    if m_total < world:
        raise ValueError("every shard needs at least one particle")
    base, extra = divmod(int(m_total), int(world))
    count = base + (1 if rank < extra else 0)
    offset = rank * base + min(rank, extra)
    return offset, count


def best_record(recs: np.ndarray) -> np.ndarray:
    """The record with the lowest (J, index): a NaN cost counts as +inf."""
    recs = np.asarray(recs, dtype=np.float64).reshape(-1, _REC)
    J = np.where(np.isnan(recs[:, 0]), np.inf, recs[:, 0])
    order = np.lexsort((recs[:, 1], J))
    return recs[order[0]].copy()


def local_allgather(recs: np.ndarray) -> np.ndarray:
    """The exchange when every shard of the swarm lives in this process."""
    return np.asarray(recs, dtype=np.float64).reshape(-1, _REC)


def torch_allgather(group=None) -> Callable[[np.ndarray], np.ndarray]:
    """The exchange over a torch.distributed process group: every rank contributes its
    local shards' records (the same number on every rank) and receives all of them."""
    import torch
    import torch.distributed as dist

    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    world = dist.get_world_size(group)

    def gather(recs: np.ndarray) -> np.ndarray:
        t = torch.from_numpy(np.ascontiguousarray(recs, dtype=np.float64).reshape(-1)).to(dev)
        out = [torch.empty_like(t) for _ in range(world)]
        dist.all_gather(out, t, group=group)
        return torch.cat(out).cpu().numpy().reshape(-1, _REC)

    return gather


class ShardedSwarm:
    """Drives the local shards of one swarm.

    ``shards`` are engines with ``run(m, iters, w, c1, c2, seed)``, ``continue_(iters)``,
    ``gbest_get() -> (g, J, index, iter)``, ``gbest_set(g, J, index)`` and
    ``result(trace=False)`` (``api.Problem`` is one), each created with its own
    shard_offset and the whole swarm's shard_total; ``counts`` their particle counts.
    ``allgather`` maps this process's records [n_local][8] to the whole swarm's.
    """

    def __init__(self, shards: Sequence, counts: Sequence[int],
                 allgather: Callable[[np.ndarray], np.ndarray] = local_allgather):
        if len(shards) != len(counts) or not shards:
            raise ValueError("one particle count per shard")
        self.shards = list(shards)
        self.counts = [int(c) for c in counts]
        self.allgather = allgather
        self.gcost_trace: List[float] = []
        self.gidx_trace: List[int] = []
        self.best = None

    def _exchange(self) -> np.ndarray:
        recs = np.empty((len(self.shards), _REC))
        for k, s in enumerate(self.shards):
            g, J, idx, _ = s.gbest_get()
            recs[k, 0] = J
            recs[k, 1] = idx
            recs[k, 2:] = g
        best = best_record(self.allgather(recs))
        for s in self.shards:
            s.gbest_set(best[2:], best[0], int(best[1]))
        self.best = best
        self.gcost_trace.append(float(best[0]))
        self.gidx_trace.append(int(best[1]))
        return best

    def run(self, iters: int, w=0.7, c1=1.5, c2=1.5, seed=0, tol_tau: float = 0.0,
            tol_window: int = 10) -> dict:
        """Initialise and evaluate every shard, then ``iters`` iterations with an exchange
        after each; stops early on Algorithm 2's test when tol_tau > 0."""
        if iters < 0:
            raise ValueError("iters must be >= 0")
        self.gcost_trace, self.gidx_trace = [], []
        for s, m in zip(self.shards, self.counts):
            s.run(m, 0, w, c1, c2, seed)
        self._exchange()
        done = 0
        for n in range(1, iters + 1):
            for s in self.shards:
                s.continue_(1)
            best = self._exchange()
            done = n
            if tol_tau > 0 and n > tol_window:
                old = np.float64(self.gcost_trace[n - tol_window])
                with np.errstate(divide="ignore", invalid="ignore"):
                    K = abs((np.float64(best[0]) - old) / np.float64(best[0]))
                if K < tol_tau:
                    break
        steps = np.array([[float(s.result(trace=False)["rk_steps"])] + [0.0] * (_REC - 1)
                          for s in self.shards])
        total_steps = int(self.allgather(steps)[:, 0].sum())
        return {"state": self.best[2:].copy(), "cost": float(self.best[0]),
                "gbest_index": int(self.best[1]), "iters_done": done, "rk_steps": total_steps,
                "gcost_trace": np.array(self.gcost_trace),
                "gidx_trace": np.array(self.gidx_trace, dtype=np.int32)}
