"""The IOD_CHECK build (argument and launch-shape checks at the entry of every swarm
kernel body, reported as a status instead of a fault): the parity tests of single runs,
edge sizes, lane pairs, the balanced schedule, batches and sharded swarms pass unchanged with it loaded,
so no check fires on any launch they make and the checked library computes the same
results.  Run in a child process, which loads libiod_gb300_check.so (IOD_CHECK=1)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parity_tests_pass_under_the_check_build():
    from paper_2207_13175_gb300 import build
    build.build(check=True)
    env = dict(os.environ, IOD_CHECK="1")
    sel = ("trace_parity_tiny or edge_sizes or lockstep or pairs or balanced_equals_grid "
           "or results_equal_alone or refinement_equals or sharded_equals_unsharded")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-m", "gpu", "-p", "no:cacheprovider",
                        "tests/test_gpu_parity.py", "tests/test_gpu_pairs.py", "tests/test_gpu_balanced.py",
                        "tests/test_gpu_batch.py", "tests/test_gpu_shard.py", "-k", sel],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    assert " passed" in r.stdout and "error" not in r.stdout.split("\n")[-2].lower(), r.stdout[-500:]


def test_check_build_is_the_loaded_library():
    env = dict(os.environ, IOD_CHECK="1")
    code = ("from paper_2207_13175_gb300 import _native as N; import os; "
            "print(os.path.basename(N.LIB_PATH))")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True)
    assert r.stdout.strip() == "libiod_gb300_check.so", r.stdout + r.stderr
