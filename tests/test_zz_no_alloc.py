"""tacaw_spectrum_static, the time transform for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc: an application that has already reserved the device's
memory for its own allocator, or that gives this library only its input and output buffers
under a fixed budget.  This entry point serves them from a fixed device array inside the
library.  It must give the same S as the allocating entry point tacaw_spectrum (FP32
arithmetic) and as the FP64 oracle, call after call, on any stream, without allocating: its
scratch is one fixed array that every call reuses.  This file sorts last so that a run
stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

import oracle
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
    side = torch.cuda.Stream()
    with T.Context(0) as ctx:
        for k, (seed, (P, F, nq)) in enumerate([(11, (2, 96, 300)), (12, (1, 64, 1000))]):
            psi_np = workloads.random_exit_waves(P, F, nq, seed=seed)
            psi = torch.from_numpy(psi_np).cuda()
            want = ctx.spectrum(psi, precision=T.DFT_FP32).cpu().numpy()
            got = torch.full((P, F, nq), float("nan"), dtype=torch.float32, device="cuda")
            torch.cuda.synchronize()
            if k == 0:
                rc = T.tacaw_spectrum_static(torch.view_as_real(psi), P, F, nq, got)
                torch.cuda.synchronize()
            else:
                # the second call on a non-default stream, passed explicitly
                with torch.cuda.stream(side):
                    rc = T.tacaw_spectrum_static(torch.view_as_real(psi), P, F, nq, got, side)
                side.synchronize()
            assert rc == T.TACAW_OK
            out = got.cpu().numpy()
            assert rel(out, want) < 1e-5
            # against the FP64 oracle, at the tolerance of the FP32 spectrum parity tests
            assert rel(out, oracle.spectrum(psi_np)) < 1e-5


def test_static_spectrum_allocates_nothing(T):
    import torch
    P, F, nq = 1, 128, 2000
    psi = torch.from_numpy(workloads.random_exit_waves(P, F, nq, seed=13)).cuda()
    out = torch.empty((P, F, nq), dtype=torch.float32, device="cuda")
    args = (torch.view_as_real(psi), P, F, nq, out)
    assert T.tacaw_spectrum_static(*args) == T.TACAW_OK  # warm-up: device code loaded
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    for _ in range(3):
        assert T.tacaw_spectrum_static(*args) == T.TACAW_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0


def test_static_spectrum_rejects_sizes_beyond_its_array(T):
    import torch
    P, F, nq = 1, 64, 40000  # residual alone is 20 MB > 16 MiB
    psi = torch.zeros((P, F, nq, 2), dtype=torch.float32, device="cuda")
    out = torch.zeros((P, F, nq), dtype=torch.float32, device="cuda")
    assert T.tacaw_spectrum_static(psi, P, F, nq, out) == T.TACAW_ETOOBIG
    assert T.tacaw_spectrum_static(psi, 0, F, nq, out) == T.TACAW_EINVAL
    host = torch.zeros((P, 8, 16, 2), dtype=torch.float32)
    assert T.tacaw_spectrum_static(host, P, 8, 16, torch.zeros((P, 8, 16), device="cuda")) == T.TACAW_EINVAL
