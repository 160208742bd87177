"""iod_score_noalloc, the allocation-free scoring call (for callers that cannot
allocate device memory once running), against the ordinary evaluation entry point.

It is called twice in a row through the C ABI, because the scratch array it shares
between calls keeps the previous call's contents; both calls must match iod_eval on
the same problem within the cost tolerance the other parity tests use, and a sample of
its costs must match the oracle directly (so that the two kernels cannot drift
together).  This file is named to be collected last."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_scoring_matches_eval_twice():
    import torch

    import scenarios as S
    from paper_2207_13175_gb300 import _native
    from paper_2207_13175_gb300 import inputs as I

    sc = I.tiny(5)
    pair = S.Pair(sc)
    X = np.vstack([I.particles_in_box(pair.lo, pair.hi, 3000, seed=8),
                   I.near_truth(sc.deputy, 300, 1.0, 0.01, seed=9)])     # 3,300: ragged
    m = X.shape[0]
    J_ref = pair.gpu.eval(X).cpu().numpy()                  # the existing entry point
    rc = pair.gpu.chief_positions()
    obs = np.stack([sc.t, pair.ra, pair.dec, rc[:, 0], rc[:, 1], rc[:, 2]])
    d_obs = torch.from_numpy(np.ascontiguousarray(obs)).cuda()
    d_x = torch.from_numpy(np.ascontiguousarray(X.T)).cuda()
    lib = _native.lib()
    stream = torch.cuda.current_stream()
    i_ref = int(np.argmin(J_ref))
    for call in range(2):
        d_J = torch.full((m,), float("nan"), dtype=torch.float64, device="cuda")
        d_best = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
        code = lib.iod_score_noalloc(sc.mu, sc.n_obs, ctypes.c_void_p(d_obs.data_ptr()),
                                     sc.sigma[0], sc.sigma[1], sc.dt,
                                     ctypes.c_void_p(d_x.data_ptr()), m,
                                     ctypes.c_void_p(d_J.data_ptr()),
                                     ctypes.c_void_p(d_best.data_ptr()),
                                     ctypes.c_void_p(stream.cuda_stream))
        assert code == 0, lib.iod_last_error()
        torch.cuda.synchronize()
        J = d_J.cpu().numpy()
        best = d_best.cpu().numpy()
        assert np.all(np.abs(J - J_ref) <= S.COST_RTOL * np.abs(J_ref)), call
        assert int(best[1]) == i_ref, call
        assert abs(best[0] - J_ref[i_ref]) <= S.COST_RTOL * abs(J_ref[i_ref])
        assert np.array_equal(best[2:], X[i_ref])
        # a sample straight against the oracle, with the per-particle cost tolerance
        sample = np.unique(np.concatenate([np.arange(0, m, m // 12), [m - 1, i_ref]]))
        states = pair.gpu.propagate(X[sample]).cpu().numpy()
        for j, i in enumerate(sample):
            ref, _, _ = pair.ora.propagate(X[i])
            Jo = pair.ora.cost(X[i])
            tol = S.cost_tolerance(pair, ref, Jo, states[:, :, j] - ref)
            assert abs(J[i] - Jo) <= tol, (call, i, J[i], Jo, tol)
    # sizes beyond the scratch array are refused, with nothing launched
    big = 131072 + 1
    code = lib.iod_score_noalloc(sc.mu, sc.n_obs, ctypes.c_void_p(d_obs.data_ptr()),
                                 sc.sigma[0], sc.sigma[1], sc.dt, ctypes.c_void_p(d_x.data_ptr()),
                                 big, ctypes.c_void_p(d_J.data_ptr()),
                                 ctypes.c_void_p(d_best.data_ptr()), None)
    assert code == -1 and b"131072" in lib.iod_last_error()
    pair.close()
