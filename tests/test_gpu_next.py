"""GPU parity of the rows beyond the core path: TACAW accessors, trajectory averaging,
aberrated and user-supplied probes, against the oracle on the same seeded inputs."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


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


def synthetic_S(P=2, F=20, ny=16, nx=32, seed=6):
    return np.random.default_rng(seed).random((P, F, ny, nx)).astype(np.float32)


@pytest.mark.parametrize("fold", [False, True])
def test_spectral_diffraction_parity(ctx, T, fold):
    S = synthetic_S()
    for f in (0.0, 5.0, 31.25, -60.0, 212.5):
        got = ctx.spectral_diffraction(dev(S), 5.0, f, fold).cpu().numpy()
        want = oracle.spectral_diffraction(S.astype(np.float64), 5.0, f, fold)
        assert np.array_equal(got, want.astype(np.float32)) or rel(got, want) < 1e-7


def test_spectrum_image_from_detector_sum(ctx, T):
    SI = np.random.default_rng(7).random((9, 40)).astype(np.float32)
    got = ctx.spectral_diffraction(dev(SI), 10.0, 15.0).cpu().numpy()
    want = oracle.spectral_diffraction(SI[:, :, None].astype(np.float64), 10.0, 15.0)[:, 0]
    assert np.allclose(got, want, rtol=1e-7, atol=0)


def test_dispersion_parity(ctx, T):
    S = synthetic_S(P=1, F=6, ny=16, nx=32)
    cell = (21.7, 10.86, 5.43)
    kx = np.linspace(0, 1 / (2 * 5.43), 17)  # Gamma -> X as in the paper's minimal example
    ky = np.linspace(-0.3, 0.41, 17)
    got = ctx.dispersion(dev(S), cell, kx, ky).cpu().numpy()
    want = oracle.dispersion(S.astype(np.float64), cell, kx, ky)
    assert rel(got, want) < 1e-6


def test_trajectory_averaging(ctx, T):
    import torch
    ws = [workloads.diamond_si(n_frames=16, grid=32, n_slices=4, reps=(1, 1, 1), seed=s) for s in (61, 62, 63)]
    ctx.load_form_factors(ws[0].form_Z, ws[0].form_coef)
    acc = torch.zeros((1, 16, 32, 32), dtype=torch.float64, device="cuda")
    for w in ws:
        S = ctx.run(T.params_of(w), dev(w.pos), dev(w.Z), T.probe_of(w))
        ctx.accumulate(S, acc, 1.0 / len(ws))
    ref = np.mean([oracle.tacaw(w) for w in ws], axis=0)
    assert rel(acc.cpu().numpy(), ref) < 1e-4


def test_aberrated_probe_scan(ctx, T):
    w = workloads.diamond_si(n_frames=2, grid=64, n_slices=4, seed=64)
    xy = np.array([[0.5, 1.0], [3.0, 6.5]])
    ab = dict(defocus=25.0, cs_mm=1.2, astig=15.0, astig_angle=0.4, coma=900.0, coma_angle=1.1)
    ctx.load_form_factors(w.form_Z, w.form_coef)
    p = T.params_of(w)
    V = ctx.build_potential(p, dev(w.pos), dev(w.Z))
    psi = ctx.propagate(p, V, T.ProbeSpec(30.0, xy, **ab)).cpu().numpy()
    op = oracle.params_of(w)
    psi0 = np.stack([oracle.probe_aberrated(op, 30.0, x, y, df=ab["defocus"], cs_mm=ab["cs_mm"], a1=ab["astig"],
                                            phi_a=ab["astig_angle"], b2=ab["coma"], phi_b=ab["coma_angle"])
                     for x, y in xy])
    for f in range(2):
        ref = oracle.multislice_frame_init(op, w.pos[f], w.Z, w.form_Z, w.form_coef, psi0)
        assert rel(psi[:, f], ref) < 2e-5


def test_user_wavefront_vortex(ctx, T):
    import torch
    w = workloads.diamond_si(n_frames=2, grid=64, n_slices=4, seed=65)
    N, L = w.nx, w.cell[0]
    k = np.fft.fftfreq(N, d=L / N)
    kx, ky = np.meshgrid(k, k)
    kmax = 25e-3 / oracle.wavelength(100e3)
    psik = np.where(kx ** 2 + ky ** 2 <= kmax ** 2, np.exp(2j * np.arctan2(ky, kx)), 0)  # l = 2 vortex
    psi_r = np.fft.ifft2(psik) * N
    psi_r /= np.sqrt(np.sum(np.abs(psi_r) ** 2))
    psi0 = psi_r[None].astype(np.complex64)
    ctx.load_form_factors(w.form_Z, w.form_coef)
    p = T.params_of(w)
    V = ctx.build_potential(p, dev(w.pos), dev(w.Z))
    d_psi0 = torch.from_numpy(psi0).cuda()
    psi = ctx.propagate(p, V, T.ProbeSpec(psi0=d_psi0)).cpu().numpy()
    op = oracle.params_of(w)
    for f in range(2):
        ref = oracle.multislice_frame_init(op, w.pos[f], w.Z, w.form_Z, w.form_coef, psi0.astype(np.complex128))
        assert rel(psi[:, f], ref) < 2e-5
