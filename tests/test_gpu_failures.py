"""Host-side failure paths, made on the host (no GPU fault): an allocator hook that
returns NULL gives IOD_ENOMEM with every earlier allocation released; a batch whose
admission allocation fails while other problems are resident backs off and admits the
request on a later call, with the result of the request run alone; with nothing
resident the request fails with IOD_ENOMEM; non-finite or misordered requests are
refused by iod_batch_submit."""
import ctypes as C
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


class FlakyAllocator:
    """Allocator hooks over PyTorch's caching allocator that fail while `failing` is set,
    counting live allocations."""

    def __init__(self):
        import torch
        from paper_2207_13175_gb300 import _native as N
        self.failing = False
        self.live = {}

        def alloc(nbytes, ctx):
            if self.failing:
                return None
            dev = torch.cuda.current_device()
            p = torch.cuda.caching_allocator_alloc(int(nbytes), dev, torch.cuda.current_stream(dev))
            self.live[p] = int(nbytes)
            return p

        def release(ptr, ctx):
            self.live.pop(ptr, None)
            torch.cuda.caching_allocator_delete(ptr)

        self.refs = (N.ALLOC_FN(alloc), N.RELEASE_FN(release))

    def __enter__(self):
        from paper_2207_13175_gb300 import _native as N
        assert N.lib().iod_set_allocator(self.refs[0], self.refs[1], None) == 0
        return self

    def __exit__(self, *exc):
        from paper_2207_13175_gb300 import _native as N
        from paper_2207_13175_gb300 import api
        api.use_torch_allocator()
        torch_refs = api._allocator_refs
        assert N.lib().iod_set_allocator(torch_refs[0], torch_refs[1], None) == 0


def test_create_enomem_releases_everything():
    from paper_2207_13175_gb300 import api
    from paper_2207_13175_gb300 import inputs as I
    sc = I.tiny(0)
    ang = np.zeros((sc.n_obs, 2)) + 0.1
    bounds = api.bounds_from_chief(sc.chief, 100.0, 1.0, I.L_KM, I.TU_S)
    with FlakyAllocator() as A:
        A.failing = True
        with pytest.raises(api.IodError) as e:
            api.Problem(sc.mu, sc.chief, sc.t, ang, sc.sigma, bounds, api.options(dt=sc.dt),
                        torch_allocator=False)
        assert e.value.code == -2 and "allocator hook returned NULL" in str(e.value)
        assert A.live == {}
        # fail at the swarm's allocation instead (the problem itself was created)
        A.failing = False
        G = api.Problem(sc.mu, sc.chief, sc.t, ang, sc.sigma, bounds, api.options(dt=sc.dt),
                        torch_allocator=False)
        held = dict(A.live)
        A.failing = True
        with pytest.raises(api.IodError) as e:
            G.run(256, 2)
        assert e.value.code == -2
        assert A.live == held                  # the failed run left nothing behind
        A.failing = False
        G.run(64, 1)
        assert G.result(trace=False)["iters_done"] == 1
        G.close()
        assert A.live == {}


def _reqs():
    import test_gpu_batch as TB
    return TB.make_requests(3, seed=21, m_choices=(200,), k_range=(20, 21))


def test_batch_admission_backs_off_and_recovers():
    import test_gpu_batch as TB
    from paper_2207_13175_gb300 import api
    reqs = _reqs()
    opts = api.options(dt=1e-3)
    with FlakyAllocator() as A:
        B = api.Batch(opts, budget_bytes=1 << 30, max_resident=8, torch_allocator=False)
        t0 = TB.submit(B, reqs[0])
        B.step(1)                                   # request 0 resident
        assert B.stats()["resident"] == 1
        A.failing = True
        t1 = TB.submit(B, reqs[1])
        B.step(1)                                   # its allocation fails: deferred
        st = B.stats()
        assert st["deferred_admissions"] >= 1 and st["queued"] == 1 and st["resident"] == 1
        assert B.poll(t1) is None
        A.failing = False
        for _ in range(200):
            if B.poll(t0) is not None and B.poll(t1) is not None:
                break
            B.step(2)
        for req, tk in ((reqs[0], t0), (reqs[1], t1)):
            r = B.poll(tk)
            ref = TB.alone(req, opts)
            assert np.array_equal(r["state"], ref["state"]) and r["cost"] == ref["cost"]
        assert B.stats()["bytes_in_use"] == 0
        # nothing resident: an allocation failure fails the request
        A.failing = True
        t2 = TB.submit(B, reqs[2])
        B.step(1)
        with pytest.raises(api.IodError) as e:
            B.poll(t2)
        assert e.value.code == -2
        A.failing = False
        st = B.stats()
        assert st["resident"] == 0 and st["queued"] == 0 and st["bytes_in_use"] == 0
        B.close()
        assert A.live == {}


@pytest.mark.parametrize("field,value", [
    ("angles_nan", math.nan), ("angles_inf", math.inf), ("sigma_nan", math.nan),
    ("times_unsorted", None), ("times_negative", None), ("bounds_inverted", None)])
def test_batch_submit_rejects(field, value):
    import test_gpu_batch as TB
    from paper_2207_13175_gb300 import api
    req = dict(_reqs()[0])
    if field.startswith("angles"):
        a = np.array(req["angles"], dtype=float)
        a[4, 1] = value
        req["angles"] = a
    elif field == "sigma_nan":
        req["sigma"] = (value, req["sigma"][1])
    elif field == "times_unsorted":
        t = np.array(req["t"])
        t[[3, 4]] = t[[4, 3]]
        req["t"] = t
    elif field == "times_negative":
        req["t"] = np.array(req["t"]) - 0.01
    else:
        b = np.array(req["bounds"])
        req["bounds"] = np.concatenate([b[6:], b[:6]])
    B = api.Batch(api.options(dt=1e-3), budget_bytes=1 << 28, max_resident=4)
    with pytest.raises(api.IodError) as e:
        TB.submit(B, req)
    assert e.value.code == -1, field
    assert B.stats()["queued"] == 0
    B.close()
