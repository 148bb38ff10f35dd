"""One trajectory split by frames (tacaw_spectrum_partial, tacaw_intensity) on one GPU: the
partial transforms of two frame ranges against the first frame's exit wave, summed as the
all-reduce across two ranks would, equal the single-process spectrum and the oracle."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm((np.asarray(a) - b).ravel()) / max(np.linalg.norm(np.ravel(b)), 1e-300))


@pytest.fixture(scope="module")
def T():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2602_10064_gb300 as T
    return T


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("scan", [False, True])
def test_two_frame_ranges_sum_to_the_whole_spectrum(T, scan):
    import torch
    from paper_2602_10064_gb300 import sharded
    w = workloads.diamond_si(n_frames=12, grid=64, n_slices=4, seed=81)
    if scan:
        w.alpha_mrad, w.probes = 30.0, workloads.probe_grid(w.cell[0], w.cell[1], 2)
    with T.Context(0) as ctx:
        ctx.load_form_factors(w.form_Z, w.form_coef)
        p, pr, Z = T.params_of(w), T.probe_of(w), dev(w.Z)
        P, F, nq = pr.n_probes, w.n_frames, w.nx * w.ny
        q = torch.from_numpy(T.tacaw_band_points(ctx.h, p)).cuda()
        nsel = q.numel()
        ref = ctx.propagate(p, ctx.build_potential(p, dev(w.pos[:1]), Z), pr)[:, 0].contiguous()
        total = torch.zeros((P, F, nsel, 2), dtype=torch.float32, device="cuda")
        for f0, f1 in (sharded.frame_range(F, r, 2) for r in range(2)):
            psi = ctx.propagate(p, ctx.build_potential(p, dev(w.pos[f0:f1]), Z), pr)
            part = torch.empty_like(total)
            T.tacaw_spectrum_partial(ctx.h, torch.view_as_real(psi), P, f1 - f0, f0, F, nq,
                                     torch.view_as_real(ref), q, nsel, part)
            total += part  # what the all-reduce across the two ranks computes
        S = torch.empty((P, F, w.ny, w.nx), dtype=torch.float32, device="cuda")
        T.tacaw_intensity(ctx.h, total, P, F, nsel, q, nq, T.REDUCE_NONE, S)
        SI = torch.empty((P, F), dtype=torch.float32, device="cuda")
        T.tacaw_intensity(ctx.h, total, P, F, nsel, q, nq, T.REDUCE_DETECTOR, SI)
        single = ctx.run(p, dev(w.pos), Z, pr, precision=T.DFT_FP32).cpu().numpy()
        # one rank holding every frame: the same entry points, no collective
        whole = sharded.run_frames_sharded(ctx, p, dev(w.pos), dev(w.pos[:1]), Z, pr, 0, F).cpu().numpy()
        ctx.check()
    S, SI = S.cpu().numpy(), SI.cpu().numpy()
    ref_S = oracle.tacaw(w)
    assert rel(S, single) < 1e-5
    assert rel(S, ref_S) < 1e-4
    assert rel(SI, ref_S.sum(axis=(2, 3))) < 1e-4
    assert rel(whole, ref_S) < 1e-4
    assert np.abs(S[:, 0]).max() == 0.0
