"""Serving loop over a batch: requests arrive on a schedule, are submitted as their time
comes, run while others are on the GPU (continuous batching: admitted as memory and
slots free up, retired as they finish) and are reported with their latencies.

The scheduling itself (admission by memory, rounds, retirement) is the library's
batch interface; this loop only feeds it on the wall clock and collects results.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np

from . import api


@dataclass
class Request:
    mu: float
    chief: np.ndarray
    t: np.ndarray
    angles: np.ndarray
    sigma: tuple
    bounds: np.ndarray
    m: int
    iters: int
    seed: int = 0
    w: float = 0.7
    c1: float = 1.5
    c2: float = 1.5


def serve(batch: "api.Batch", requests, arrivals, slice_s: float = 0.05, rounds_per_step: int = 0,
          timeout_s: float = 600.0) -> dict:
    """Submit requests[i] at wall-clock offset arrivals[i] (seconds after the start), keep
    the batch running until every request has finished, and report per-request
    latencies (finish - arrival) with their p50/p99, solves/s over the whole run, the
    batch's device-memory high-water mark and the most requests seen queued (waiting for
    memory or a slot) and resident at once.  The batch runs in persistent slices of
    `slice_s` device seconds (new arrivals join between slices), or in steps of
    `rounds_per_step` lockstep rounds when that is set."""
    order = np.argsort(arrivals)
    tickets = {}
    results = {}
    t0 = time.perf_counter()
    nxt = 0
    queued_max = resident_max = 0
    while len(results) < len(requests):
        now = time.perf_counter() - t0
        if now > timeout_s:
            raise TimeoutError("serving run exceeded its time limit")
        while nxt < len(order) and arrivals[order[nxt]] <= now:
            i = int(order[nxt])
            q = requests[i]
            tickets[i] = batch.submit(q.mu, q.chief, q.t, q.angles, q.sigma, q.bounds, q.m, q.iters,
                                      q.w, q.c1, q.c2, q.seed)
            nxt += 1
        if not tickets or len(tickets) == len(results):
            # nothing in flight: wait for the next arrival
            if nxt < len(order):
                time.sleep(max(0.0, min(0.01, arrivals[order[nxt]] - now)))
            continue
        st = batch.stats()
        queued_max = max(queued_max, st["queued"])
        resident_max = max(resident_max, st["resident"])
        if rounds_per_step:
            batch.step(rounds_per_step)
        else:
            batch.run(slice_s)
        for i, tk in tickets.items():
            if i in results:
                continue
            r = batch.poll(tk)
            if r is not None:
                r["t_done"] = time.perf_counter() - t0
                results[i] = r
    wall = time.perf_counter() - t0
    lat = np.array([results[i]["t_done"] - arrivals[i] for i in range(len(requests))])
    st = batch.stats()
    return {"n": len(requests), "wall_s": wall, "solves_per_s": len(requests) / wall,
            "latency_p50_s": float(np.percentile(lat, 50)),
            "latency_p99_s": float(np.percentile(lat, 99)),
            "latency_max_s": float(lat.max()), "latencies_s": lat.tolist(),
            "mem_high_water_bytes": int(st["bytes_high_water"]), "budget_bytes": int(st["budget"]),
            "queued_max": queued_max, "resident_max": resident_max,
            "results": [results[i] for i in range(len(requests))]}
