"""The paper-shaped workloads at full geometry against the FP64 oracle.

- The precision configuration (1024^2 grid, 20 slices, frames 2 fs apart) on a real,
  non-periodic trajectory: relative L2 error of S per energy band for every time-transform
  arithmetic (Methods, "Workflow Architecture": the mean-subtracted time transform).  The oracle
  propagates every frame in full and keeps every 4th kx and ky for the spectrum.
- The minimal example's geometry (Supplement, "Minimal Working Example": 16,000 Si atoms,
  0.1 A sampling padded to 1152^2, 54 slices): exit waves of sampled frames.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

TOL_FIELD = 2e-5
TOL_S = 1e-4


def rel(a, b):
    return float(np.linalg.norm((np.asarray(a) - b).ravel()) / max(np.linalg.norm(np.ravel(b)), 1e-300))


@pytest.fixture(scope="module")
def T():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2602_10064_gb300 as T
    return T


@pytest.fixture(scope="module")
def ctx(T):
    c = T.Context(0)
    yield c
    c.close()


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


BANDS_MEV = ((0, 25), (25, 50), (50, 100), (100, None))


def band_errors(S, ref, F, dt_fs):
    """Relative L2 error of S[F][...] per band of |E| = h |f| (meV), and over all bins."""
    f = np.fft.fftfreq(F, d=dt_fs * 1e-3)  # THz
    E = np.abs(f) * workloads.H_MEV_PS
    out = {}
    for lo, hi in BANDS_MEV:
        m = (E >= lo) & ((E < hi) if hi is not None else True)
        out[f"{lo}-{hi if hi is not None else 'inf'} meV"] = rel(S[m], ref[m])
    out["all"] = rel(S, ref)
    return out


def test_precision_per_energy_band_on_a_1024sq_trajectory(ctx, T):
    F, sub = 128, 4
    w = workloads.config4(n_frames=F, seed=14)
    ctx.load_form_factors(w.form_Z, w.form_coef)
    p, pr, pos, Z = T.params_of(w), T.probe_of(w), dev(w.pos), dev(w.Z)
    got = {}
    for name, code in (("fp32", T.DFT_FP32), ("bf16x3", T.DFT_BF16X3), ("tf32x3", T.DFT_TF32X3),
                       ("bf16", T.DFT_BF16), ("tf32", T.DFT_TF32)):
        S = ctx.run(p, pos, Z, pr, precision=code)
        got[name] = S[0, :, ::sub, ::sub].cpu().numpy().astype(np.float64)
        del S
    ctx.check()
    psi = oracle.multislice(oracle.params_of(w), w.pos, w.Z, w.form_Z, w.form_coef)
    ref = oracle.spectrum(np.ascontiguousarray(psi[:, :, ::sub, ::sub]))[0]
    del psi
    rows = {name: band_errors(S, ref, F, w.dt_fs) for name, S in got.items()}
    for name, r in rows.items():
        print(name, " ".join(f"{k}: {v:.2e}" for k, v in r.items()))
    for name in ("fp32", "bf16x3", "tf32x3"):
        for band, err in rows[name].items():
            assert err < TOL_S, (name, band, err)
    assert rows["bf16"]["all"] > 3 * rows["bf16x3"]["all"]


def test_minimal_example_geometry_sampled_frames(ctx, T):
    w = workloads.minimal_example_si(n_frames=8)
    assert (w.nx, w.ny, w.n_slices, w.n_atoms) == (1152, 1152, 54, 16000)
    ctx.load_form_factors(w.form_Z, w.form_coef)
    p = T.params_of(w)
    frames = [0, 5]
    V = ctx.build_potential(p, dev(w.pos[frames]), dev(w.Z))
    psi = ctx.propagate(p, V, T.probe_of(w)).cpu().numpy()[0]
    refs = oracle.multislice(oracle.params_of(w), w.pos[frames], w.Z, w.form_Z, w.form_coef)[0]
    for i in range(len(frames)):
        err = rel(psi[i], refs[i])
        print(f"minimal example, frame {frames[i]}: exit wave rel L2 = {err:.2e}")
        assert err < TOL_FIELD, err


def test_minimal_example_scan_sampled_probes(ctx, T):
    # the minimal example's 32 x 32 scan at 30 mrad: two of its probes, two frames
    w = workloads.minimal_example_si(n_frames=8, n_scan=32)
    assert w.n_probes == 1024 and w.alpha_mrad == 30.0
    ctx.load_form_factors(w.form_Z, w.form_coef)
    p = T.params_of(w)
    frames, sel = [1, 6], [0, 529]
    xy = w.probes[sel]
    V = ctx.build_potential(p, dev(w.pos[frames]), dev(w.Z))
    psi = ctx.propagate(p, V, T.ProbeSpec(w.alpha_mrad, xy)).cpu().numpy()
    refs = oracle.multislice(oracle.params_of(w), w.pos[frames], w.Z, w.form_Z, w.form_coef,
                             alpha_mrad=w.alpha_mrad, probes=xy)
    for j in range(len(sel)):
        for i in range(len(frames)):
            err = rel(psi[j, i], refs[j, i])
            print(f"minimal example scan, probe {sel[j]}, frame {frames[i]}: exit wave rel L2 = {err:.2e}")
            assert err < TOL_FIELD, err
