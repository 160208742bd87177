"""Argument validation of iod_create (the problem statement's inputs, checked before any
device work, so this runs without a GPU): non-finite angles, times, chief state, sigma
or bounds, unsorted or negative times, an empty or inverted box and a mass parameter out
of range are refused with IOD_EINVAL and a message, and no problem is returned."""
import ctypes as C
import math

import numpy as np
import pytest

IOD_EINVAL = -1


def _create(lib, mu=0.01215058560962404, chief=None, t=None, ang=None, sigma=None, bounds=None,
            n_obs=None):
    from paper_2207_13175_gb300 import _native as N
    chief = np.array([0.85, 0, 0.17, 0, 0.26, 0.0]) if chief is None else np.asarray(chief, float)
    t = np.linspace(0.0, 0.23, 20) if t is None else np.asarray(t, float)
    ang = np.tile([0.1, 0.2], (t.size, 1)) if ang is None else np.asarray(ang, float)
    sigma = np.array([4.8e-6, 4.8e-6]) if sigma is None else np.asarray(sigma, float)
    if bounds is None:
        d = np.array([2.6e-4] * 3 + [9.8e-4] * 3)
        bounds = np.concatenate([chief - d, chief + d])
    bounds = np.asarray(bounds, float)
    D = C.POINTER(C.c_double)
    keep = [np.ascontiguousarray(a) for a in (chief, t, ang, sigma, bounds)]
    ptrs = [a.ctypes.data_as(D) for a in keep]
    o = N.Options()
    assert lib.iod_options_default(C.byref(o)) == 0
    h = C.c_void_p(123)
    rc = lib.iod_create(mu, ptrs[0], t.size if n_obs is None else n_obs, ptrs[1], ptrs[2], ptrs[3],
                        ptrs[4], C.byref(o), C.byref(h))
    return rc, h.value, lib.iod_last_error().decode()


@pytest.fixture(scope="module")
def lib():
    from paper_2207_13175_gb300 import _native
    return _native.lib()


def _with(arr, idx, val):
    a = np.array(arr, dtype=float)
    a[idx] = val
    return a


T = np.linspace(0.0, 0.23, 20)
ANG = np.tile([0.1, 0.2], (20, 1))


@pytest.mark.parametrize("case,kw,word", [
    ("nan angle", dict(ang=_with(ANG, (3, 0), math.nan)), "angles"),
    ("inf angle", dict(ang=_with(ANG, (7, 1), math.inf)), "angles"),
    ("nan time", dict(t=_with(T, 5, math.nan)), "obs_times"),
    ("unsorted times", dict(t=_with(T, 5, T[3])), "increasing"),
    ("repeated time", dict(t=_with(T, 6, T[5])), "increasing"),
    ("negative first time", dict(t=T - 0.01), ">= 0"),
    ("nan sigma", dict(sigma=[math.nan, 4.8e-6]), "sigma"),
    ("zero sigma", dict(sigma=[4.8e-6, 0.0]), "sigma"),
    ("negative sigma", dict(sigma=[-1e-6, 4.8e-6]), "sigma"),
    ("inf chief", dict(chief=[0.85, 0, math.inf, 0, 0.26, 0]), "chief"),
    ("nan bound", dict(bounds=_with(np.zeros(12) + np.r_[-np.ones(6), np.ones(6)], 4, math.nan)), "bounds"),
    ("inverted box", dict(bounds=np.r_[np.ones(6), -np.ones(6)]), "lo must be < hi"),
    ("empty box", dict(bounds=np.zeros(12)), "lo must be < hi"),
    ("no epochs", dict(n_obs=0), "n_obs"),
    ("mu zero", dict(mu=0.0), "mu"),
    ("mu nan", dict(mu=math.nan), "mu"),
])
def test_create_rejects(lib, case, kw, word):
    rc, h, msg = _create(lib, **kw)
    assert rc == IOD_EINVAL, (case, rc, msg)
    assert h is None, case                     # *out is cleared: no problem handed back
    assert word in msg, (case, msg)


def test_strerror_names_every_code(lib):
    for code in range(0, -9, -1):
        assert lib.iod_strerror(code)


@pytest.mark.parametrize("args", [(0, 1, 10), (33, 1, 10), (1, 0, 10), (1, 33, 10), (1, 1, 0),
                                  (1, 1, 2000000)])
def test_fp64_issue_probe_arguments(lib, args):
    """The FP64 issue diagnostic refuses bad shapes before any device work."""
    out = C.c_double(0.0)
    assert lib.iod_selftest_fp64_issue(*args, C.byref(out)) == IOD_EINVAL
    assert lib.iod_selftest_fp64_issue(1, 1, 10, None) == IOD_EINVAL


@pytest.mark.parametrize("gate,iters", [(-1.0, 5), (float("nan"), 5), (float("inf"), 5), (2.0, 0)])
def test_refine_gate_checked_by_batch_create(lib, gate, iters):
    """The refinement gate must be finite and non-negative, and needs refine_iters."""
    from paper_2207_13175_gb300 import _native as N
    o = N.Options()
    lib.iod_options_default(C.byref(o))
    o.refine_gate = gate
    o.refine_iters = iters
    b = C.c_void_p(7)
    assert lib.iod_batch_create(C.byref(o), 1 << 30, 4, C.byref(b)) == IOD_EINVAL
    assert "refine_gate" in lib.iod_last_error().decode()


def test_refine_gate_refused_for_single_problems(lib):
    rc, h, msg = _create_with(lib, refine_gate=3.0)
    assert rc == IOD_EINVAL and not h and "refine_gate" in msg


def _create_with(lib, **kw):
    from paper_2207_13175_gb300 import _native as N
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
    lib.iod_options_default(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    h = C.c_void_p(123)
    rc = lib.iod_create(0.01215058560962404, ptrs[0], 20, ptrs[1], ptrs[2], ptrs[3], ptrs[4],
                        C.byref(o), C.byref(h))
    return rc, h.value, lib.iod_last_error().decode()
