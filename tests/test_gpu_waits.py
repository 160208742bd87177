"""The bounded device waits give up with a status the host reads, and the CUDA context
stays usable: the balanced schedule's hand-off wait run on a flag that nothing sets (and,
as a control, on one that is set), then an ordinary problem on the same device."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_wait_on_unset_flag_gives_up_and_context_survives():
    import scenarios as S
    from paper_2207_13175_gb300 import api
    from paper_2207_13175_gb300 import inputs as I
    gave_up, waited = api.selftest_wait(0.25, set_flag=False)
    assert gave_up
    assert 0.25 <= waited < 5.0
    gave_up, waited = api.selftest_wait(0.25, set_flag=True)
    assert not gave_up and waited < 0.25
    # the device still runs problems, with the same results as before
    sc = I.tiny(0)
    pair = S.Pair(sc)
    pair.gpu.run(sc.m, 5, sc.w, sc.c1, sc.c2, sc.seed)
    r1 = pair.gpu.result()
    api.selftest_wait(0.1)
    pair.gpu.run(sc.m, 5, sc.w, sc.c1, sc.c2, sc.seed)
    r2 = pair.gpu.result()
    assert np.array_equal(r1["state"], r2["state"]) and r1["cost"] == r2["cost"]
    pair.close()


def test_wait_probe_arguments_checked():
    from paper_2207_13175_gb300 import api
    for bad in (0.0, -1.0, 11.0, float("nan")):
        with pytest.raises(api.IodError):
            api.selftest_wait(bad)
