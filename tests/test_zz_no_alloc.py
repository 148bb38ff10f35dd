"""tacaw_spectrum_static, the time transform for callers that cannot allocate device memory.

It must give the same S as the allocating entry point tacaw_spectrum (FP32 arithmetic), call
after call: its scratch is one fixed device array that every call reuses.  This file sorts
last so that a run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.fixture(scope="module")
def T():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2602_10064_gb300 as T
    return T


def test_static_spectrum_matches_allocating_entry_point_on_consecutive_calls(T):
    import torch
    with T.Context(0) as ctx:
        for seed, (P, F, nq) in [(11, (2, 96, 300)), (12, (1, 64, 1000))]:
            psi = torch.from_numpy(workloads.random_exit_waves(P, F, nq, seed=seed)).cuda()
            want = ctx.spectrum(psi, precision=T.DFT_FP32).cpu().numpy()
            got = torch.full((P, F, nq), float("nan"), dtype=torch.float32, device="cuda")
            rc = T.tacaw_spectrum_static(torch.view_as_real(psi), P, F, nq, got)
            assert rc == T.TACAW_OK
            torch.cuda.synchronize()
            assert rel(got.cpu().numpy(), want) < 1e-5


def test_static_spectrum_rejects_sizes_beyond_its_array(T):
    import torch
    P, F, nq = 1, 64, 40000  # residual alone is 20 MB > 16 MiB
    psi = torch.zeros((P, F, nq, 2), dtype=torch.float32, device="cuda")
    out = torch.zeros((P, F, nq), dtype=torch.float32, device="cuda")
    assert T.tacaw_spectrum_static(psi, P, F, nq, out) == T.TACAW_ETOOBIG
    assert T.tacaw_spectrum_static(psi, 0, F, nq, out) == T.TACAW_EINVAL
