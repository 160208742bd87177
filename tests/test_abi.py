"""The C-ABI library builds for sm_103a, loads without a GPU and exports every entry
point that include/iod.h declares; the Python binding declares each of them.  No
compute calls are made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "iod.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(iod_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def native():
    from paper_2207_13175_gb300 import build
    build.build()
    from paper_2207_13175_gb300 import _native
    return _native


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ("iod_create", "iod_run", "iod_result", "iod_destroy", "iod_set_stream",
                     "iod_set_allocator", "iod_snapshot", "iod_restore", "iod_strerror",
                     "iod_bounds_from_chief", "iod_eval", "iod_options_default"):
        assert required in names


def test_library_exports_every_declared_symbol(native):
    lib = ctypes.CDLL(native.LIB_PATH)
    missing = [n for n in header_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(native):
    assert sorted(native.SIGNATURES) == header_functions()
    native.lib()


def test_host_only_entry_points(native):
    """Entry points that touch no device: strerror and argument validation paths."""
    L = native.lib()
    assert L.iod_strerror(0) == b"ok"
    assert L.iod_strerror(-1) == b"invalid argument"
    o = native.Options()
    assert L.iod_options_default(ctypes.byref(o)) == 0
    assert o.integrator == 0 and o.dt == 1e-3 and o.rtol == 1e-12 and o.record_trace == 1
    assert L.iod_options_default(None) == -1
    b = (ctypes.c_double * 12)()
    chief = (ctypes.c_double * 6)(0.85, 0, 0.17, 0, 0.26, 0)
    assert L.iod_bounds_from_chief(chief, 100.0, 1.0, 384400.0, 375190.0, b) == 0
    assert b[0] == pytest.approx(0.85 - 100 / 384400.0) and b[9] == pytest.approx(1e-3 / (384400 / 375190))
    assert L.iod_bounds_from_chief(chief, -1.0, 1.0, 384400.0, 375190.0, b) == -1
    # invalid create arguments are rejected before any device work
    h = ctypes.c_void_p()
    t = (ctypes.c_double * 2)(0.0, 0.1)
    ang = (ctypes.c_double * 4)(0, 0, 0, 0)
    sig = (ctypes.c_double * 2)(1e-5, 1e-5)
    assert L.iod_create(0.0121, chief, 0, t, ang, sig, b, None, ctypes.byref(h)) == -1
    t_bad = (ctypes.c_double * 2)(0.1, 0.1)
    assert L.iod_create(0.0121, chief, 2, t_bad, ang, sig, b, None, ctypes.byref(h)) == -1
    assert b"increasing" in L.iod_last_error()
    sig_bad = (ctypes.c_double * 2)(0.0, 1e-5)
    assert L.iod_create(0.0121, chief, 2, t, ang, sig_bad, b, None, ctypes.byref(h)) == -1
    assert L.iod_run(None, 10, 1, 0.7, 1.5, 1.5, 0) == -1


def test_oracle_does_not_enter_the_package():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2207_13175_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), f
                assert "iod_oracle" not in text, f


def test_check_build_exports_every_declared_symbol():
    """The IOD_CHECK variant (argument checks compiled into the swarm kernels) builds and
    exports the same entry points."""
    from paper_2207_13175_gb300 import build
    path = build.build(check=True)
    lib = ctypes.CDLL(path)
    missing = [n for n in header_functions() if not hasattr(lib, n)]
    assert not missing, missing
