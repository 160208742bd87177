"""Host logic of the serving loop, without a GPU: a stand-in batch that finishes each
request a fixed number of slices after its submission checks that requests are submitted
at their arrival times, polled until done, and that the reported latencies, percentiles,
throughput and queue/residency maxima follow from that schedule."""
import numpy as np

from paper_2207_13175_gb300.serve import Request, serve


class FakeBatch:
    """Each submitted request finishes after `slices` run() calls; at most `slots` run
    at once, the rest wait queued (as the library's admission would keep them)."""

    def __init__(self, slices=3, slots=2):
        self.slices, self.slots = slices, slots
        self.left = {}            # ticket -> remaining slices (running)
        self.queue = []           # tickets waiting for a slot
        self.done = set()
        self.submitted = []
        self.runs = 0

    def submit(self, mu, chief, t, angles, sigma, bounds, m, iters, w, c1, c2, seed):
        tk = len(self.submitted)
        self.submitted.append((tk, m))
        self.queue.append(tk)
        return tk

    def _admit(self):
        while self.queue and len(self.left) < self.slots:
            self.left[self.queue.pop(0)] = self.slices

    def run(self, seconds):
        self.runs += 1
        self._admit()
        for tk in list(self.left):
            self.left[tk] -= 1
            if self.left[tk] == 0:
                del self.left[tk]
                self.done.add(tk)

    def poll(self, tk):
        return {"state": np.zeros(6), "cost": float(tk)} if tk in self.done else None

    def stats(self):
        return {"queued": len(self.queue), "resident": len(self.left), "bytes_high_water": 123,
                "budget": 456}


def _requests(n):
    z = np.zeros(6)
    return [Request(0.01, z, np.array([0.0, 1.0]), np.zeros((2, 2)), (1e-5, 1e-5), np.zeros(12),
                    64 + i, 10) for i in range(n)]


def test_every_request_is_served_with_its_latency():
    B = FakeBatch(slices=3, slots=2)
    reqs = _requests(6)
    arrivals = np.array([0.0, 0.0, 0.01, 0.02, 0.03, 0.2])
    out = serve(B, reqs, arrivals, slice_s=0.0)
    assert out["n"] == 6 and len(out["results"]) == 6
    assert [m for _, m in B.submitted] == [64 + i for i in np.argsort(arrivals, kind="stable")]
    assert all(r is not None for r in out["results"])
    lat = np.array([r["t_done"] for r in out["results"]]) - arrivals
    assert np.all(lat > 0)
    assert out["latency_p50_s"] == np.percentile(lat, 50)
    assert out["latency_p99_s"] == np.percentile(lat, 99)
    assert out["solves_per_s"] == 6 / out["wall_s"]
    assert out["resident_max"] <= 2 and out["queued_max"] >= 1
    assert out["mem_high_water_bytes"] == 123 and out["budget_bytes"] == 456


def test_requests_are_not_submitted_before_they_arrive():
    B = FakeBatch(slices=1, slots=8)
    reqs = _requests(2)
    arrivals = np.array([0.0, 0.15])
    out = serve(B, reqs, arrivals, slice_s=0.0)
    # the second request's completion cannot precede its arrival
    assert out["results"][1]["t_done"] >= 0.15
