"""Batches: every problem's result in a batch of uneven problems (observation counts,
swarm sizes, iteration counts, size classes, arrival times) equals the result of the
same problem run alone through iod_run, and admission respects the memory budget."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def make_requests(n, seed=0, m_choices=(64, 200, 333, 700), k_range=(8, 60)):
    """Seeded uneven problems: chiefs from the corrected orbits and the tiny chief, 8-60
    epochs over 0.5-2 days, swarms of 64-700, 3-12 iterations."""
    from paper_2207_13175_gb300 import api
    from paper_2207_13175_gb300 import inputs as I
    rng = np.random.default_rng(seed)
    orbits = I.chief_orbits()
    chiefs = [np.array(orbits[k]["state"]) for k in ("halo", "dro", "lyapunov")]
    chiefs.append(np.array([0.85, 0, 0.17, 0, 0.26, 0]))
    out = []
    for j in range(n):
        chief = chiefs[j % len(chiefs)]
        off, _, _ = I.truth_offset(rng, 5.0, 200.0, 0.0, 2.0)
        deputy = chief + off
        K = int(rng.integers(*k_range))
        T = rng.uniform(0.5, 2.0) * I.DAY_TU
        t = np.linspace(0.0, T, K)
        noise = rng.normal(0, I.ARCSEC, (K, 2))
        ang, _ = api.simulate_obs(I.MU, chief, deputy, t, noise)
        bounds = api.bounds_from_chief(chief, 250.0, 2.0, I.L_KM, I.TU_S)
        out.append(dict(mu=I.MU, chief=chief, t=t, angles=ang, sigma=(I.ARCSEC, I.ARCSEC),
                        bounds=bounds, m=int(rng.choice(m_choices)), iters=int(rng.integers(3, 13)),
                        seed=int(rng.integers(0, 2 ** 31))))
    return out


def alone(req, opts):
    from paper_2207_13175_gb300 import api
    with api.Problem(req["mu"], req["chief"], req["t"], req["angles"], req["sigma"], req["bounds"],
                     opts) as G:
        G.run(req["m"], req["iters"], seed=req["seed"])
        return G.result()


def submit(B, req):
    return B.submit(req["mu"], req["chief"], req["t"], req["angles"], req["sigma"], req["bounds"],
                    req["m"], req["iters"], seed=req["seed"])


def run_staggered(B, reqs, rounds=2):
    """Submit a third of the requests, run a step, then the rest, stepping until done."""
    tickets = [submit(B, r) for r in reqs[: len(reqs) // 3]]
    B.step(rounds)
    tickets += [submit(B, r) for r in reqs[len(reqs) // 3:]]
    for _ in range(500):
        if all(B.poll(t) is not None for t in tickets):
            break
        B.step(rounds)
    return [B.poll(t, trace=True) for t in tickets]


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_results_equal_alone(precision):
    from paper_2207_13175_gb300 import api
    opts = api.options(dt=1e-3, precision=precision, fp64_last_iters=3)
    reqs = make_requests(14, seed=3 + precision)
    B = api.Batch(api.options(dt=1e-3, precision=precision, fp64_last_iters=3),
                  budget_bytes=1 << 30, max_resident=64)
    B.set_block_sizes([128, 400, 1 << 30], [64, 128, 256])
    got = run_staggered(B, reqs)
    for req, r in zip(reqs, got):
        ref = alone(req, opts)
        assert r is not None
        assert r["iters_done"] == ref["iters_done"] == req["iters"]
        assert np.array_equal(r["state"], ref["state"]), (req["m"], req["iters"])
        assert r["cost"] == ref["cost"] and r["gbest_index"] == ref["gbest_index"]
        assert r["rk_steps"] == ref["rk_steps"]
        assert np.array_equal(r["gidx_trace"], ref["gidx_trace"])
        assert np.array_equal(r["gcost_trace"], ref["gcost_trace"])
    st = B.stats()
    assert st["resident"] == 0 and st["finished"] == len(reqs)
    B.close()


def test_batch_budget_queueing_and_cancel():
    from paper_2207_13175_gb300 import api
    reqs = make_requests(10, seed=11, m_choices=(512,), k_range=(20, 21))
    for r in reqs:                   # equal sizes and arcs: equal device footprints
        r["iters"] = 6
        r["t"] = reqs[0]["t"]
    opts = api.options(dt=1e-3, precision=api.MIXED, fp64_last_iters=2)
    B = api.Batch(opts, budget_bytes=1 << 30, max_resident=64)
    # size the budget for three resident problems
    submit(B, reqs[0])
    B.step(0)
    one = B.stats()["bytes_in_use"]
    assert one > 0
    B.close()
    B = api.Batch(opts, budget_bytes=3 * one + one // 2, max_resident=64)
    tickets = [submit(B, r) for r in reqs]
    B.step(1)
    st = B.stats()
    assert st["resident"] == 3 and st["queued"] == 7
    B.cancel(tickets[1])            # resident
    B.cancel(tickets[9])            # queued
    for _ in range(400):
        if all(B.poll(t) is not None for i, t in enumerate(tickets) if i not in (1, 9)):
            break
        B.step(2)
    st = B.stats()
    assert st["bytes_high_water"] <= B.stats()["budget"]
    for i, t in enumerate(tickets):
        if i in (1, 9):
            with pytest.raises(api.IodError) as e:
                B.poll(t)
            assert e.value.code == -6
        else:
            ref = alone(reqs[i], opts)
            r = B.poll(t)
            assert np.array_equal(r["state"], ref["state"]) and r["cost"] == ref["cost"]
            ts, ta, td = B.times(t)
            assert 0 <= ts <= ta <= td
    B.close()


@pytest.mark.parametrize("precision,slice_s", [(0, 0.0), (1, 0.0), (1, 0.02)])
def test_persistent_scheduler_results_equal_alone(precision, slice_s):
    """The dependency-driven scheduler (problems advance independently inside one
    launch), run to completion or in short device-time slices with arrivals in
    between, gives every problem the same result as running it alone."""
    from paper_2207_13175_gb300 import api
    opts = api.options(dt=1e-3, precision=precision, fp64_last_iters=3)
    reqs = make_requests(12, seed=21 + precision)
    B = api.Batch(opts, budget_bytes=1 << 30, max_resident=64)
    tickets = [submit(B, r) for r in reqs[:5]]
    B.run(slice_s)
    tickets += [submit(B, r) for r in reqs[5:]]
    for _ in range(2000):
        if all(B.poll(t) is not None for t in tickets):
            break
        B.run(slice_s)
    for req, t in zip(reqs, tickets):
        r = B.poll(t, trace=True)
        ref = alone(req, opts)
        assert r is not None and r["iters_done"] == req["iters"]
        assert np.array_equal(r["state"], ref["state"]) and r["cost"] == ref["cost"]
        assert r["rk_steps"] == ref["rk_steps"]
        assert np.array_equal(r["gidx_trace"], ref["gidx_trace"])
    assert B.stats()["resident"] == 0
    B.close()


def test_autotuner_sets_block_sizes():
    """The autotuner times the candidates, sets the chosen sizes, and results do not
    depend on the block size chosen."""
    from paper_2207_13175_gb300 import api
    opts = api.options(dt=1e-3, precision=api.MIXED, fp64_last_iters=2)
    reqs = make_requests(3, seed=31, m_choices=(100, 300, 700))
    B = api.Batch(opts, budget_bytes=1 << 30, max_resident=16)
    samples = [(r["mu"], r["chief"], r["t"], r["angles"], r["sigma"], r["bounds"], r["m"], 6)
               for r in reqs]
    chosen, ms = B.autotune([128, 400, 1 << 30], samples, candidates=(64, 128, 256), uniform=True)
    assert len(set(chosen)) == 1 and chosen[0] in (64, 128, 256)
    assert ms.shape == (3, 3) and np.all(ms > 0)
    tickets = [submit(B, r) for r in reqs]
    B.run(0.0)
    for r, t in zip(reqs, tickets):
        ref = alone(r, opts)
        got = B.poll(t)
        assert np.array_equal(got["state"], ref["state"]) and got["cost"] == ref["cost"]
    B.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_slot_reuse_under_short_persistent_slices(precision):
    """Few resident slots, many requests, persistent runs of a few milliseconds: slots
    retire and are reused by later requests between runs (their freed descriptors must
    stay inactive), and every result still equals the problem run alone."""
    from paper_2207_13175_gb300 import api
    opts = api.options(dt=1e-3, precision=precision, fp64_last_iters=3)
    reqs = make_requests(12, seed=41 + precision)
    B = api.Batch(opts, budget_bytes=1 << 30, max_resident=3)
    tickets = [submit(B, r) for r in reqs]
    for _ in range(2000):
        if all(B.poll(t) is not None for t in tickets):
            break
        B.run(0.002)
    for req, t in zip(reqs, tickets):
        got = B.poll(t, trace=True)
        ref = alone(req, opts)
        assert got is not None and got["iters_done"] == ref["iters_done"]
        assert np.array_equal(got["state"], ref["state"]) and got["cost"] == ref["cost"]
        assert np.array_equal(got["gcost_trace"], ref["gcost_trace"])
    assert B.stats()["finished"] == len(reqs)
    B.close()


@pytest.mark.parametrize("precision,persistent", [(0, True), (1, True), (1, False)])
def test_batch_refinement_equals_swarm_then_iod_refine(precision, persistent):
    """With refine_iters set, a batch request ends with Levenberg-Marquardt from its
    global best (the paper's local minimisation, Eqs. 14-16): its swarm result (pso_state,
    pso_cost) equals the request run alone, and its refined state and cost equal
    iod_refine started from that swarm result, bit for bit, under the persistent
    scheduler and in lockstep rounds."""
    from paper_2207_13175_gb300 import api
    base = dict(dt=1e-3, precision=precision, fp64_last_iters=3)
    reqs = make_requests(6, seed=51 + precision)
    B = api.Batch(api.options(refine_iters=25, **base), budget_bytes=1 << 30, max_resident=64)
    tickets = [submit(B, r) for r in reqs]
    for _ in range(2000):
        if all(B.poll(t) is not None for t in tickets):
            break
        if persistent:
            B.run(0.0)
        else:
            B.step(2)
    for req, t in zip(reqs, tickets):
        got = B.poll(t)
        ref = alone(req, api.options(**base))
        assert np.array_equal(got["pso_state"], ref["state"]) and got["pso_cost"] == ref["cost"]
        with api.Problem(req["mu"], req["chief"], req["t"], req["angles"], req["sigma"],
                         req["bounds"], api.options(dt=1e-3)) as G:
            x, c, it = G.refine(ref["state"], 25)
        assert np.array_equal(got["state"], x) and got["cost"] == c, (got["state"] - x, got["cost"], c)
        assert got["refine_iters"] == it and got["cost"] <= got["pso_cost"]
    B.close()


def _solve_all(B, reqs, persistent):
    tickets = [submit(B, r) for r in reqs]
    for _ in range(4000):
        if all(B.poll(t) is not None for t in tickets):
            break
        if persistent:
            B.run(0.0)
        else:
            B.step(2)
    return [B.poll(t) for t in tickets]


@pytest.mark.parametrize("persistent", [True, False])
def test_refinement_gate_falls_back_to_fp64(persistent):
    """refine_gate: a request whose refined cost is above the gate is solved again in FP64
    from the same initial swarm.  With a gate below every cost, every result equals the
    same request in an FP64 batch with the same refinement, bit for bit (swarm best,
    refined state and cost, LM iterations), with fallback = 1 and both solves' steps
    counted; with a gate above every cost nothing changes."""
    from paper_2207_13175_gb300 import api
    base = dict(dt=1e-3, fp64_last_iters=3, refine_iters=25)
    reqs = make_requests(4, seed=91)
    B = api.Batch(api.options(precision=1, refine_gate=1e-300, **base), budget_bytes=1 << 30, max_resident=64)
    got = _solve_all(B, reqs, persistent)
    B.close()
    B = api.Batch(api.options(precision=0, **base), budget_bytes=1 << 30, max_resident=64)
    ref = _solve_all(B, reqs, persistent)
    B.close()
    for g, r in zip(got, ref):
        assert g["fallback"] == 1 and r["fallback"] == 0
        assert np.array_equal(g["state"], r["state"]) and g["cost"] == r["cost"]
        assert np.array_equal(g["pso_state"], r["pso_state"]) and g["pso_cost"] == r["pso_cost"]
        assert g["refine_iters"] == r["refine_iters"] and g["iters_done"] == r["iters_done"]
        assert g["rk_steps"] > r["rk_steps"]
    B = api.Batch(api.options(precision=1, refine_gate=1e300, **base), budget_bytes=1 << 30, max_resident=64)
    high = _solve_all(B, reqs, persistent)
    B.close()
    B = api.Batch(api.options(precision=1, **base), budget_bytes=1 << 30, max_resident=64)
    off = _solve_all(B, reqs, persistent)
    B.close()
    for h, o in zip(high, off):
        assert h["fallback"] == 0
        assert np.array_equal(h["state"], o["state"]) and h["cost"] == o["cost"] and h["rk_steps"] == o["rk_steps"]


def test_refine_iters_rejected_for_single_problems():
    from paper_2207_13175_gb300 import api
    req = make_requests(1, seed=61)[0]
    with pytest.raises(api.IodError) as e:
        api.Problem(req["mu"], req["chief"], req["t"], req["angles"], req["sigma"], req["bounds"],
                    api.options(dt=1e-3, refine_iters=5))
    assert e.value.code == -1


def test_autotuner_with_refinement_enabled():
    """The autotuner times samples as swarms, also for a batch that refines."""
    from paper_2207_13175_gb300 import api
    reqs = make_requests(2, seed=71, m_choices=(100, 300))
    B = api.Batch(api.options(dt=1e-3, refine_iters=10), budget_bytes=1 << 30, max_resident=8)
    samples = [(r["mu"], r["chief"], r["t"], r["angles"], r["sigma"], r["bounds"], r["m"], 4) for r in reqs]
    chosen, ms = B.autotune([200, 1 << 30], samples, candidates=(64, 128), uniform=True)
    assert len(set(chosen)) == 1 and np.all(ms > 0)
    B.close()


def test_step_sizes_by_class_equal_alone():
    """Per-class RK4 step bounds: every request integrates with its class's dt and its
    result equals the same problem run alone at that dt."""
    from paper_2207_13175_gb300 import api
    reqs = make_requests(8, seed=81)
    classes, dts = [128, 400, 1 << 30], [2e-3, 1e-3, 5e-4]
    B = api.Batch(api.options(dt=1e-3), budget_bytes=1 << 30, max_resident=64)
    B.set_step_sizes(classes, dts)
    tickets = [submit(B, r) for r in reqs]
    B.run(0.0)
    for req, t in zip(reqs, tickets):
        dt = next(d for c, d in zip(classes, dts) if req["m"] <= c)
        ref = alone(req, api.options(dt=dt))
        got = B.poll(t)
        assert np.array_equal(got["state"], ref["state"]) and got["cost"] == ref["cost"]
        assert got["rk_steps"] == ref["rk_steps"]
    B.close()


def test_step_size_autotuner():
    """The step-size autotuner: a generous budget takes the largest candidate, a budget
    below every error the smallest, and otherwise the largest candidate within the
    budget.  (For deputies within a few hundred km the chief's and the deputy's RK4
    errors nearly cancel in the line of sight, so the errors sit near the DOPRI5
    reference's own floor, ~1e-10 rad, for every candidate.)"""
    from paper_2207_13175_gb300 import api
    from paper_2207_13175_gb300 import inputs as I
    reqs = make_requests(2, seed=91, m_choices=(100, 300))
    samples = [(r["mu"], r["chief"], r["t"], r["angles"], r["sigma"], r["bounds"], r["m"], 4, r["seed"])
               for r in reqs]
    cands = [4e-3, 2e-3, 1e-3, 5e-4]
    B = api.Batch(api.options(dt=1e-3), budget_bytes=1 << 30, max_resident=8)
    dt, err = B.autotune_dt([200, 1 << 30], samples, cands, 1.0, n_probe=32)
    assert dt == [4e-3, 4e-3]
    assert np.all(np.isfinite(err)) and np.all(err > 0) and np.all(err < 1e-7), err
    budget = 0.1 * I.ARCSEC
    dt, err = B.autotune_dt([200, 1 << 30], samples, cands, budget, n_probe=32)
    for c in range(2):
        ok = [d for d, e in zip(cands, err[c]) if e <= budget]
        assert dt[c] == (max(ok) if ok else min(cands))
    dt, _ = B.autotune_dt([200, 1 << 30], samples, cands, 1e-300, n_probe=32)
    assert dt == [5e-4, 5e-4]
    B.close()
