"""The benchmark's workloads at full size, in the launch configuration that bench.py times:
one tacaw_run over the whole trajectory, the BF16x3 time transform, the default tiling, the
full S on the device.  The result is checked element by element against the oracle.

The oracle cannot run 1024-2048 frames of these grids within a test, so each trajectory
repeats its first R = 8 frames.  The shapes, sizes, atom counts and tiling are the
benchmark's own; only the frame contents repeat.  For a sequence x_t of period R over F
frames (R divides F):
- the mean over the F frames is the mean over one period;
- the DFT over t vanishes except at omega = m F / R;
- at those bins it is F / R times the R-point DFT of one period.

So S_F(m F/R) = (F/R)^2 S_R(m), and S_F = 0 at every other omega, where S_R is the oracle's
spectrum (|DFT_t(psi - mean)|^2, Sec. 2) of the R distinct exit waves.  The relative L2 error
of S against that reference counts the off-peak bins too, summed on the device.
"""
import math

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

TOL_S = 1e-4
R = 8


@pytest.fixture(scope="module")
def T():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2602_10064_gb300 as T
    return T


@pytest.fixture(scope="module")
def ctx(T):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    c = T.Context(0)
    yield c
    c.close()


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def periodic(w):
    """The workload with frames t and t mod R made identical."""
    assert w.n_frames % R == 0
    w.pos = np.ascontiguousarray(np.tile(w.pos[:R], (w.n_frames // R, 1, 1)))
    return w


def periodic_error(S, ref_R, probes):
    """Relative L2 error of the device spectrum S [P][F][ny][nx] (rows `probes`) against the
    periodic reference built from ref_R [len(probes)][R][ny][nx]."""
    F = S.shape[1]
    k = F // R
    ref = float(k * k) * ref_R
    num = 0.0
    for i, p in enumerate(probes):
        peaks = S[p, ::k].double().cpu().numpy()
        num += float(((peaks - ref[i]) ** 2).sum())
        for m in range(R):  # the off-peak bins between two peaks, on the device
            band = S[p, m * k + 1:(m + 1) * k].double()
            num += float((band * band).sum())
    return math.sqrt(num / float((ref ** 2).sum()))


def run_full(ctx, T, w):
    ctx.load_form_factors(w.form_Z, w.form_coef)
    S = ctx.run(T.params_of(w), dev(w.pos), dev(w.Z), T.probe_of(w), precision=T.DFT_BF16X3)
    ctx.check()
    return S


def oracle_spectrum(w, probes=None):
    op = oracle.params_of(w)
    pr = None if w.alpha_mrad <= 0 else np.asarray(w.probes)[probes]
    psi = oracle.multislice(op, w.pos[:R], w.Z, w.form_Z, w.form_coef, w.alpha_mrad, pr)
    return oracle.spectrum(psi)


def test_config2_full_size(ctx, T):
    """1024 frames of 8000-atom rocksalt, 512^2, 20 slices, plane wave."""
    w = periodic(workloads.config2())
    assert (w.n_frames, w.n_atoms, w.nx, w.n_slices) == (1024, 8000, 512, 20)
    S = run_full(ctx, T, w)
    err = periodic_error(S, oracle_spectrum(w), [0])
    print(f"c2 full size: S rel L2 {err:.2e}")
    assert err < TOL_S, err


def test_config4_full_size(ctx, T):
    """2048 frames of the 64-atom diamond cell, 1024^2, 20 slices, plane wave (S is 8 GiB)."""
    w = periodic(workloads.config4())
    assert (w.n_frames, w.nx, w.n_slices) == (2048, 1024, 20)
    S = run_full(ctx, T, w)
    err = periodic_error(S, oracle_spectrum(w), [0])
    print(f"c4 full size: S rel L2 {err:.2e}")
    assert err < TOL_S, err


def test_config3_full_size_sampled_probes(ctx, T):
    """256 frames x 256 probe positions of 576-atom diamond, 256^2, 20 slices, 30 mrad probe
    (S is 16 GiB); three probe positions, first, inner and last, against the oracle."""
    w = periodic(workloads.config3())
    assert (w.n_frames, w.n_probes, w.nx) == (256, 256, 256)
    S = run_full(ctx, T, w)
    probes = [0, 137, 255]
    err = periodic_error(S, oracle_spectrum(w, probes), probes)
    print(f"c3 full size, probes {probes}: S rel L2 {err:.2e}")
    assert err < TOL_S, err
