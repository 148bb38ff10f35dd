"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a brute-force transform,
a closed form, a special case, an exact invariant.  The choice is such that a dropped term,
a flipped sign, a wrong index or a transposed operand anywhere in the oracle fails one of them.
"""
import math

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.filterwarnings("ignore")


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


# ---------------------------------------------------------------------------------------
# transforms: the in-house FFT equals the O(N^2) / O(N^4) DFT
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 8, 12, 16, 32, 64])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft_equals_brute_force_dft(n, sign):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    assert rel(oracle.fft(x, sign), oracle.dft(x, sign)) < 1e-12


@pytest.mark.parametrize("n", [6, 7, 9, 15, 45, 96, 100, 192, 384, 768, 1152])
@pytest.mark.parametrize("sign", [-1, 1])
def test_mixed_radix_fft_equals_brute_force_dft(n, sign):
    # the lengths 3 * 2^k and 9 * 2^7 of the grids, plus odd and prime lengths
    rng = np.random.default_rng(1000 + n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    assert rel(oracle.fft(x, sign), oracle.dft(x, sign)) < 1e-12


def test_brute_dft_definition_small():
    # n = 4, forward: the matrix exp(-2 pi i jk/4) has entries 1, -i, -1, i.
    x = np.array([1.0, 2.0, 3.0, 4.0], dtype=complex)
    want = np.array([10, -2 + 2j, -2, -2 - 2j])
    assert np.abs(oracle.dft(x, -1) - want).max() < 1e-13


@pytest.mark.parametrize("shape", [(8, 8), (16, 16), (8, 16), (16, 4), (12, 24), (24, 9)])
def test_fft2_equals_brute_force_2d(shape):
    rng = np.random.default_rng(sum(shape))
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    for sign in (-1, 1):
        assert rel(oracle.fft2(x, sign), oracle.dft2_brute(x, sign)) < 1e-12


def test_fft_round_trip_and_delta():
    n = 64
    x = np.zeros(n, complex)
    x[5] = 1.0
    X = oracle.fft(x, -1)
    assert np.allclose(X, np.exp(-2j * np.pi * 5 * np.arange(n) / n), atol=1e-14)
    assert rel(oracle.fft(X, +1) / n, x) < 1e-14


# ---------------------------------------------------------------------------------------
# electron optics: closed forms
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("V,lam", [(100e3, 0.037014), (200e3, 0.025079), (300e3, 0.019687)])
def test_wavelength_textbook(V, lam):
    assert abs(oracle.wavelength(V) - lam) < 5e-7


@pytest.mark.parametrize("V", [60e3, 100e3, 200e3, 300e3])
def test_sigma_equivalent_closed_form(V):
    # sigma = (2 pi / (lambda V)) (m0 c^2 + eV) / (2 m0 c^2 + eV), m0 c^2 = 510998.95 eV
    mc2 = 510998.95000
    want = 2 * math.pi / (oracle.wavelength(V) * V) * (mc2 + V) / (2 * mc2 + V)
    assert abs(oracle.sigma(V) / want - 1) < 1e-8


def test_sigma_100kv_value():
    assert abs(oracle.sigma(100e3) - 9.2440e-4) < 5e-8


def test_kirkland_prefactor():
    # 2 pi a0 e with a0 = 0.529177 A and e = 14.39965 V A
    assert abs(oracle.kirkland_prefactor() - 2 * math.pi * 0.529177210903 * 14.399645) < 1e-4
    assert abs(oracle.kirkland_prefactor() - 47.8776) < 1e-4


# ---------------------------------------------------------------------------------------
# form factor: each of the six terms alone at a point where its value is known
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("i", [0, 1, 2])
def test_form_factor_lorentzian_terms(i):
    c = np.zeros(12)
    c[1:6:2] = 1.0  # unused Lorentzians: a = 0, b = 1
    c[2 * i], c[2 * i + 1] = 1.7, 0.9  # a_i, b_i
    q = math.sqrt(0.9)
    assert abs(oracle.form_factor(c, q) - 1.7 / 1.8) < 1e-14
    assert abs(oracle.form_factor(c, 0.0) - 1.7 / 0.9) < 1e-14


@pytest.mark.parametrize("i", [0, 1, 2])
def test_form_factor_gaussian_terms(i):
    c = np.zeros(12)
    c[1:6:2] = 1.0  # Lorentzians off: a = 0, b = 1
    c[6 + 2 * i], c[7 + 2 * i] = 0.3, 2.5  # c_i, d_i
    q = math.sqrt(math.log(2.0) / 2.5)
    assert abs(oracle.form_factor(c, q) - 0.15) < 1e-14
    assert abs(oracle.form_factor(c, 0.0) - 0.3) < 1e-14


# ---------------------------------------------------------------------------------------
# grids
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("n", [7, 8, 128])
def test_kfreq_is_fftfreq(n):
    L = 10.86
    want = np.fft.fftfreq(n, d=L / n)
    got = np.array([oracle.kfreq(i, n, L) for i in range(n)])
    assert np.abs(got - want).max() < 1e-15


@pytest.mark.parametrize("N", [16, 32, 64])
def test_mask_counts_integer_disc(N):
    # square cell: |k| <= (2/3)(N/2)/L  <=>  9 (m^2 + n^2) <= N^2
    p = oracle.params(N, N, 1, (10.86, 10.86, 5.0))
    m = oracle.mask(p)
    idx = np.fft.fftfreq(N, d=1.0 / N).astype(int)
    want = (9 * (idx[:, None] ** 2 + idx[None, :] ** 2) <= N * N).astype(np.int32)
    assert np.array_equal(m, want)
    assert oracle.mask(oracle.params(N, N, 1, (10.86, 10.86, 5.0), bandlimit=0.0)).all()


def test_slice_index_rule():
    Lz, S = 10.0, 4  # dz = 2.5
    cases = [(0.0, 0), (2.4999999, 0), (2.5, 1), (9.9999, 3), (10.0, 0), (-1e-6, 3), (12.6, 1),
             (-7.5, 1), (25.0, 2)]
    for z, s in cases:
        assert oracle.slice_index(z, Lz, S) == s, (z, s)


# ---------------------------------------------------------------------------------------
# projected potential
# ---------------------------------------------------------------------------------------
def _one_atom(x, y, Z=14, N=32, L=8.0, bandlimit=2.0 / 3.0):
    p = oracle.params(N, N, 1, (L, L, 4.0), bandlimit=bandlimit)
    fz, fc = workloads.placeholder_form_factors([Z])
    pos = np.array([[x, y, 1.0]], dtype=np.float32)
    return p, fz, fc, oracle.potential_slice(p, pos, [Z], 0, fz, fc)


def test_potential_single_atom_fourier_coefficients():
    p, fz, fc, V = _one_atom(0.0, 0.0)
    N, L = p.nx, p.Lx
    ck = oracle.fft2(V, -1) / (N * N)  # Fourier coefficients of v
    k = np.fft.fftfreq(N, d=L / N)
    q = np.sqrt(k[:, None] ** 2 + k[None, :] ** 2)
    f = np.vectorize(lambda qq: oracle.form_factor(fc[0], qq))(q)
    want = oracle.kirkland_prefactor() / (L * L) * f * oracle.mask(p)
    assert np.abs(ck - want).max() < 1e-12 * np.abs(want).max()


def test_potential_translation_by_grid_vector():
    _, _, _, V0 = _one_atom(0.0, 0.0)
    p, _, _, V1 = _one_atom(3 * 8.0 / 32, 5 * 8.0 / 32)
    assert np.abs(V1 - np.roll(V0, (5, 3), axis=(0, 1))).max() < 1e-10 * np.abs(V0).max()


def test_potential_inversion_symmetry_and_mean():
    p, fz, fc, V = _one_atom(0.0, 0.0)
    Vm = np.roll(V[::-1, ::-1], (1, 1), axis=(0, 1))  # v(-r)
    assert np.abs(V - Vm).max() < 1e-10 * np.abs(V).max()
    want_mean = oracle.kirkland_prefactor() / (p.Lx * p.Ly) * oracle.form_factor(fc[0], 0.0)
    assert abs(V.mean() - want_mean) < 1e-12 * abs(want_mean)


def test_potential_brute_force_two_species_tiny():
    N, L = 8, 4.0
    p = oracle.params(N, N, 2, (L, L, 4.0))
    fz, fc = workloads.placeholder_form_factors([8, 12])
    pos = np.array([[0.7, 1.9, 0.5], [2.3, 0.4, 1.2], [1.1, 3.3, 3.0]], dtype=np.float32)
    Z = np.array([8, 12, 12], dtype=np.int32)
    V = oracle.potential_slice(p, pos, Z, 0, fz, fc)  # slice 0 = z in [0, 2): atoms 0 and 1
    k = np.fft.fftfreq(N, d=L / N)
    mk = oracle.mask(p)
    want = np.zeros((N, N))
    pre = oracle.kirkland_prefactor() / (L * L)
    for iy in range(N):
        for ix in range(N):
            r = np.array([ix * L / N, iy * L / N])
            acc = 0j
            for j in (0, 1):
                c = fc[list(fz).index(Z[j])]
                rj = pos[j, :2].astype(np.float64)
                for a in range(N):
                    for b in range(N):
                        if not mk[a, b]:
                            continue
                        kv = np.array([k[b], k[a]])
                        acc += pre * oracle.form_factor(c, np.hypot(*kv)) * np.exp(2j * np.pi * kv @ (r - rj))
            want[iy, ix] = acc.real
    assert np.abs(V - want).max() < 1e-11 * np.abs(want).max()


def test_potential_missing_species_is_an_error():
    p = oracle.params(8, 8, 1, (4.0, 4.0, 4.0))
    fz, fc = workloads.placeholder_form_factors([14])
    with pytest.raises(ValueError):
        oracle.potential_slice(p, np.zeros((1, 3), np.float32), [8], 0, fz, fc)


# ---------------------------------------------------------------------------------------
# probe
# ---------------------------------------------------------------------------------------
def test_probe_norm_aperture_and_shift():
    N, L = 64, 16.0
    p = oracle.params(N, N, 1, (L, L, 2.0))
    psi = oracle.probe(p, 30.0)
    assert abs(np.sum(np.abs(psi) ** 2) - 1) < 1e-12
    ck = oracle.fft2(psi, -1) / N  # unitary
    k = np.fft.fftfreq(N, d=L / N)
    kmax = 30e-3 / oracle.wavelength(100e3)
    inside = (k[:, None] ** 2 + k[None, :] ** 2) <= kmax ** 2
    assert np.abs(ck[~inside]).max() < 1e-12
    assert np.allclose(np.abs(ck[inside]), 1 / math.sqrt(inside.sum()), atol=1e-12)
    shifted = oracle.probe(p, 30.0, 3 * L / N, 7 * L / N)
    assert np.abs(shifted - np.roll(psi, (7, 3), axis=(0, 1))).max() < 1e-12
    pw = oracle.probe(p, 0.0)
    assert np.allclose(pw, 1 / N)


# ---------------------------------------------------------------------------------------
# propagation
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("S", [1, 3, 7])
def test_vacuum_is_fresnel_free_propagation(S):
    N, L, Lz = 32, 12.0, 21.0
    p = oracle.params(N, N, S, (L, L, Lz))
    fz, fc = workloads.placeholder_form_factors([14])
    psi_k = oracle.multislice_frame(p, np.zeros((0, 3), np.float32), np.zeros(0, np.int32), fz, fc,
                                    alpha_mrad=40.0, probes=np.array([[1.3, 2.9]]))[0]
    psi0 = oracle.fft2(oracle.probe(p, 40.0, 1.3, 2.9), -1) / N
    k = np.fft.fftfreq(N, d=L / N)
    k2 = k[:, None] ** 2 + k[None, :] ** 2
    want = psi0 * oracle.mask(p) * np.exp(-1j * np.pi * oracle.wavelength(100e3) * Lz * k2)
    assert np.abs(psi_k - want).max() < 1e-12


def test_plane_wave_vacuum_stays_unscattered():
    p = oracle.params(16, 16, 4, (5.0, 5.0, 8.0))
    fz, fc = workloads.placeholder_form_factors([14])
    psi_k = oracle.multislice_frame(p, np.zeros((0, 3), np.float32), np.zeros(0, np.int32), fz, fc)[0]
    want = np.zeros((16, 16), complex)
    want[0, 0] = 1.0
    assert np.abs(psi_k - want).max() < 1e-13


def test_thin_slice_weak_phase_object():
    # One slice without the final propagator: psi(k) = M(k) c_k(t), and for weak sigma V
    # c_k(t) = delta_k0 + i sigma c_k(V) + R_k with |R_k| <= (sigma ||V||_inf)^2 / 2.
    N, L = 32, 8.0
    scale = 1e-3
    p = oracle.params(N, N, 1, (L, L, 3.0), final_propagator=0, sigma_scale=scale)
    fz, fc = workloads.placeholder_form_factors([14])
    pos = np.array([[2.1, 3.7, 1.0], [5.5, 6.1, 2.0]], np.float32)
    psi_k, V = oracle.multislice_frame(p, pos, [14, 14], fz, fc, want_V=True)
    psi_k = psi_k[0]
    ckV = oracle.fft2(V[0], -1) / (N * N)
    sig = oracle.sigma(100e3) * scale
    delta = np.zeros((N, N))
    delta[0, 0] = 1
    lin = (delta + 1j * sig * ckV) * oracle.mask(p)
    bound = 0.5 * (sig * np.abs(V).max()) ** 2
    err = np.abs(psi_k - lin).max()
    assert err <= bound
    # the first-order term is far above the bound, so a sign error in exp(i sigma V) fails
    assert np.abs(sig * ckV).max() > 20 * bound


def test_thin_slice_exact_transmission():
    N, L = 16, 6.0
    p = oracle.params(N, N, 1, (L, L, 3.0), final_propagator=0)
    fz, fc = workloads.placeholder_form_factors([14])
    pos = np.array([[1.0, 2.0, 1.0]], np.float32)
    psi_k, V = oracle.multislice_frame(p, pos, [14], fz, fc, want_V=True)
    t = np.exp(1j * oracle.sigma(100e3) * V[0])
    want = oracle.fft2(t, -1) / (N * N) * oracle.mask(p)
    assert np.abs(psi_k[0] - want).max() < 1e-13


def test_norm_conserved_without_mask_and_not_increased_with():
    # Without masks every step is unitary.  With the propagator mask but an unfiltered
    # (unimodular) t, each slice can only lose norm.  A band-limited t is not unimodular,
    # so there the norm is only close to 1.
    w = workloads.diamond_si(n_frames=1, grid=32, n_slices=4)
    fr = w.pos[0]
    p0 = oracle.params_of(w, bandlimit=0.0)
    psi = oracle.multislice_frame(p0, fr, w.Z, w.form_Z, w.form_coef)[0]
    assert abs(np.sum(np.abs(psi) ** 2) - 1) < 1e-13
    for S in (1, 2, 4, 8):
        p = oracle.params(w.nx, w.ny, S, w.cell, bandlimit_transmission=0)
        n = np.sum(np.abs(oracle.multislice_frame(p, fr, w.Z, w.form_Z, w.form_coef)[0]) ** 2)
        assert n <= 1 + 1e-13
        p1 = oracle.params(w.nx, w.ny, S, w.cell, bandlimit_transmission=1)
        n1 = np.sum(np.abs(oracle.multislice_frame(p1, fr, w.Z, w.form_Z, w.form_coef)[0]) ** 2)
        assert abs(n1 - 1) < 1e-3


def test_slices_compose_in_vacuum():
    p1 = oracle.params(16, 16, 1, (6.0, 6.0, 10.0))
    p5 = oracle.params(16, 16, 5, (6.0, 6.0, 10.0))
    fz, fc = workloads.placeholder_form_factors([14])
    e = np.zeros((0, 3), np.float32)
    a = oracle.multislice_frame(p1, e, np.zeros(0, np.int32), fz, fc, 25.0, np.array([[1.0, 1.0]]))
    b = oracle.multislice_frame(p5, e, np.zeros(0, np.int32), fz, fc, 25.0, np.array([[1.0, 1.0]]))
    assert np.abs(a - b).max() < 1e-13


# ---------------------------------------------------------------------------------------
# time transform
# ---------------------------------------------------------------------------------------
def test_spectrum_fft_equals_direct_and_parseval():
    psi = workloads.random_exit_waves(2, 16, 10)
    S_fft = oracle.spectrum(psi)
    S_dir = oracle.spectrum(psi, direct=True)
    assert rel(S_fft, S_dir) < 1e-12
    r = psi.astype(np.complex128) - psi.astype(np.complex128).mean(axis=1, keepdims=True)
    assert rel(S_fft.sum(axis=1), 16 * np.sum(np.abs(r) ** 2, axis=1)) < 1e-12
    assert np.abs(S_fft[:, 0]).max() < 1e-20


def test_spectrum_sign_convention():
    F, m0 = 16, 3
    n = np.arange(F)
    psi = np.exp(2j * np.pi * m0 * n / F)[None, :, None] * np.ones((1, 1, 2))
    S = oracle.spectrum(psi, subtract_mean=False)
    assert np.argmax(S[0, :, 0]) == m0
    assert abs(S[0, m0, 0] - F * F) < 1e-9


def test_mean_subtraction_changes_only_bin_zero():
    psi = workloads.random_exit_waves(1, 32, 12, elastic=5.0)
    a = oracle.spectrum(psi, subtract_mean=True)
    b = oracle.spectrum(psi, subtract_mean=False)
    assert rel(a[:, 1:], b[:, 1:]) < 1e-10
    assert np.abs(a[:, 0]).max() < 1e-20 * np.abs(b[:, 0]).max()


def test_mean_is_arithmetic_mean():
    psi = workloads.random_exit_waves(2, 8, 5)
    assert rel(oracle.mean(psi), psi.astype(np.complex128).mean(axis=1)) < 1e-14


# ---------------------------------------------------------------------------------------
# end to end: physics invariants of multislice + TACAW
# ---------------------------------------------------------------------------------------
def test_static_trajectory_has_no_inelastic_signal():
    w = workloads.static_si()
    S = oracle.tacaw(w)
    p = oracle.params_of(w)
    psi = oracle.multislice(p, w.pos, w.Z, w.form_Z, w.form_coef)
    S_nomean = oracle.spectrum(psi, subtract_mean=False)
    assert S.max() <= 1e-24 * S_nomean.max()
    assert S_nomean[:, 1:].max() <= 1e-24 * S_nomean[:, 0].max()


def test_single_mode_on_bin_peaks_at_the_mode():
    m0, F = 2, 32
    w = workloads.single_mode_si(n_frames=F, m0=m0)
    S = oracle.tacaw(w)[0].reshape(F, -1)
    per_bin = S.sum(axis=1)
    off = [m for m in range(F) if m % m0 != 0]
    assert per_bin[off].max() <= 1e-18 * per_bin.max()
    nz = [m for m in range(1, F)]
    best = nz[int(np.argmax(per_bin[1:]))]
    assert best in (m0, F - m0)


def test_single_mode_amplitude_scaling():
    m0, F = 2, 32
    tot = {}
    for A in (0.004, 0.002):
        w = workloads.single_mode_si(n_frames=F, m0=m0, amp=A)
        S = oracle.tacaw(w)[0].reshape(F, -1).sum(axis=1)
        tot[A] = (S[m0] + S[F - m0], S[2 * m0] + S[F - 2 * m0])
    r1 = tot[0.004][0] / tot[0.002][0]
    r2 = tot[0.004][1] / tot[0.002][1]
    assert abs(r1 / 4 - 1) < 0.02
    assert abs(r2 / 16 - 1) < 0.1


def test_time_roll_and_reversal():
    w = workloads.diamond_si(n_frames=16, grid=32, n_slices=4, seed=11)
    p = oracle.params_of(w)
    psi = oracle.multislice(p, w.pos, w.Z, w.form_Z, w.form_coef)
    S = oracle.spectrum(psi)
    S_roll = oracle.spectrum(np.roll(psi, 5, axis=1))
    S_rev = oracle.spectrum(psi[:, ::-1])
    assert rel(S_roll, S) < 1e-12
    neg = (-np.arange(16)) % 16
    assert rel(S_rev, S[:, neg]) < 1e-12


def test_periodic_trajectory_spectrum():
    """A trajectory that repeats every R frames: S over F = k R frames is k^2 times the R-frame
    spectrum at omega = m k and zero elsewhere (the DFT of a periodic sequence).  The full-size
    GPU tests build their reference this way."""
    w = workloads.diamond_si(n_frames=4, grid=32, n_slices=4, seed=12)
    p = oracle.params_of(w)
    psi = oracle.multislice(p, w.pos, w.Z, w.form_Z, w.form_coef)
    R, k = 4, 6
    S_R = oracle.spectrum(psi)
    S_F = oracle.spectrum(np.tile(psi, (1, k, 1, 1)))
    assert rel(S_F[:, ::k], k * k * S_R) < 1e-12
    off = np.delete(S_F, np.arange(0, R * k, k), axis=1)
    assert np.abs(off).max() < 1e-12 * S_F.max()


def test_lattice_translation_invariance():
    w = workloads.diamond_si(n_frames=8, grid=32, n_slices=4, seed=12)
    p = oracle.params_of(w)
    S = oracle.spectrum(oracle.multislice(p, w.pos, w.Z, w.form_Z, w.form_coef))
    pos2 = (w.pos.astype(np.float64) + np.array([5.43, 0.0, 0.0])).astype(np.float32)
    S2 = oracle.spectrum(oracle.multislice(p, pos2, w.Z, w.form_Z, w.form_coef))
    assert rel(S2, S) < 1e-4


def test_final_propagator_does_not_change_spectrum():
    w = workloads.diamond_si(n_frames=8, grid=32, n_slices=4, seed=13)
    S1 = oracle.tacaw(w)
    S0 = oracle.tacaw(w, final_propagator=0)
    assert rel(S0, S1) < 1e-10


# ---------------------------------------------------------------------------------------
# accessors, averaging, aberrated probe
# ---------------------------------------------------------------------------------------
def test_freq_bin_and_spectral_diffraction():
    # 200 frames at 10 fs: bins of 0.5 THz (Supplement, "Minimal Working Example")
    assert oracle.freq_bin(15.0, 200, 10.0) == 30
    assert oracle.freq_bin(-15.0, 200, 10.0) == 170
    S = np.random.default_rng(3).random((2, 8, 4, 5))
    m = oracle.spectral_diffraction(S, 10.0, 2 * 12.5, fold=False)  # F = 8, dt 10 fs: 12.5 THz bins
    assert np.array_equal(m, S[:, 2])
    mf = oracle.spectral_diffraction(S, 10.0, 2 * 12.5, fold=True)
    assert np.allclose(mf, S[:, 2] + S[:, 6])


def test_dispersion_interpolation():
    rng = np.random.default_rng(4)
    S = rng.random((1, 3, 8, 16))
    cell = (16.0, 8.0, 1.0)  # dk = 1/16, 1/8
    # on grid points: exact values, including the periodic wrap
    kx = np.array([0.0, 3 / 16, -1 / 16, 15 / 16])
    ky = np.array([0.0, 2 / 8, 0.0, 1 / 8])
    out = oracle.dispersion(S, cell, kx, ky)
    want = np.stack([S[0, :, 0, 0], S[0, :, 2, 3], S[0, :, 0, 15], S[0, :, 1, 15]], axis=-1)
    assert np.allclose(out[0], want)
    # half-way between two columns: the mean
    mid = oracle.dispersion(S, cell, np.array([2.5 / 16]), np.array([1 / 8]))
    assert np.allclose(mid[0, :, 0], 0.5 * (S[0, :, 1, 2] + S[0, :, 1, 3]))


def test_defocus_is_free_propagation():
    # chi = pi lambda df k^2 applied at the aperture equals vacuum propagation over df
    N, L, df = 64, 16.0, 35.0
    p = oracle.params(N, N, 1, (L, L, 2.0), bandlimit=0.0)
    focused = oracle.probe(p, 25.0, 3.0, 5.0)
    defoc = oracle.probe_aberrated(p, 25.0, 3.0, 5.0, df=df)
    k = np.fft.fftfreq(N, d=L / N)
    P = np.exp(-1j * np.pi * oracle.wavelength(100e3) * df * (k[:, None] ** 2 + k[None, :] ** 2))
    prop = oracle.fft2(P * oracle.fft2(focused, -1), +1) / (N * N)
    assert np.abs(defoc - prop).max() < 1e-12
    assert np.abs(oracle.probe_aberrated(p, 25.0, 3.0, 5.0) - focused).max() < 1e-13
    assert abs(np.sum(np.abs(oracle.probe_aberrated(p, 25.0, cs_mm=1.2, a1=40.0, phi_a=0.3)) ** 2) - 1) < 1e-12


def _unitary_k(psi):
    return oracle.fft2(psi, -1) / math.sqrt(psi.size)


def _aperture_coefficients(N, L, alpha_mrad, lam):
    """Focused aperture in k-space (uniform amplitude inside alpha/lambda) and the k grid."""
    k = np.fft.fftfreq(N, d=L / N)
    KX, KY = np.meshgrid(k, k, indexing="xy")  # KX[iy, ix] = k[ix]
    inside = KX ** 2 + KY ** 2 <= (alpha_mrad * 1e-3 / lam) ** 2
    return KX, KY, inside


@pytest.mark.parametrize("a1,df", [(40.0, 0.0), (-25.0, 15.0)])
def test_astigmatism_is_separable_fresnel_along_the_axes(a1, df):
    # With phi_a = 0, a1 cos(2 phi) k^2 = a1 (kx^2 - ky^2): the probe equals the focused probe
    # propagated by exp(-i pi lambda (df + a1) kx^2) along x and exp(-i pi lambda (df - a1) ky^2)
    # along y.  A cos(phi) in place of cos(2 phi), or a flipped sign of a1, fails this.
    N, L = 64, 16.0
    p = oracle.params(N, N, 1, (L, L, 2.0), bandlimit=0.0)
    lam = oracle.wavelength(100e3)
    KX, KY, inside = _aperture_coefficients(N, L, 28.0, lam)
    focused = _unitary_k(oracle.probe(p, 28.0, 2.5, 4.0))
    want = focused * np.exp(-1j * np.pi * lam * ((df + a1) * KX ** 2 + (df - a1) * KY ** 2))
    got = _unitary_k(oracle.probe_aberrated(p, 28.0, 2.5, 4.0, df=df, a1=a1, phi_a=0.0))
    assert np.abs(got - want).max() < 1e-12
    # the astigmatic phase is far from negligible at the aperture edge
    assert np.pi * lam * abs(a1) * (28e-3 / lam) ** 2 > 1.0


@pytest.mark.parametrize("phi_a", [np.pi / 4, 0.3])
def test_astigmatism_rotated_axes_cartesian_form(phi_a):
    # a1 cos 2(phi - phi_a) k^2 = a1 [cos(2 phi_a) (kx^2 - ky^2) + sin(2 phi_a) 2 kx ky]
    N, L, a1 = 64, 16.0, 30.0
    p = oracle.params(N, N, 1, (L, L, 2.0), bandlimit=0.0)
    lam = oracle.wavelength(100e3)
    KX, KY, inside = _aperture_coefficients(N, L, 28.0, lam)
    focused = _unitary_k(oracle.probe(p, 28.0))
    chi = np.pi * lam * a1 * (np.cos(2 * phi_a) * (KX ** 2 - KY ** 2) + np.sin(2 * phi_a) * 2 * KX * KY)
    got = _unitary_k(oracle.probe_aberrated(p, 28.0, a1=a1, phi_a=phi_a))
    assert np.abs(got - focused * np.exp(-1j * chi)).max() < 1e-12


@pytest.mark.parametrize("cs_mm", [0.5, 1.2, -0.8])
def test_spherical_aberration_textbook_angular_form(cs_mm):
    # The spherical-aberration phase in angular form: chi(theta) = pi Cs theta^4 / (2 lambda),
    # theta = lambda |k|, Cs converted from mm to A (1 mm = 1e7 A).  Compare the phase of every
    # k inside the aperture of a centred probe with it.  lambda^2 in place of lambda^3, or a
    # wrong mm -> A factor, fails this.
    N, L, alpha = 96, 24.0, 30.0
    p = oracle.params(N, N, 1, (L, L, 2.0), bandlimit=0.0)
    lam = oracle.wavelength(100e3)
    KX, KY, inside = _aperture_coefficients(N, L, alpha, lam)
    theta = lam * np.sqrt(KX ** 2 + KY ** 2)
    chi = np.pi * (cs_mm * 1e7) * theta ** 4 / (2.0 * lam)
    got = _unitary_k(oracle.probe_aberrated(p, alpha, cs_mm=cs_mm))
    amp = 1.0 / math.sqrt(inside.sum())
    assert np.abs(got[inside] - amp * np.exp(-1j * chi[inside])).max() < 1e-11
    assert np.abs(got[~inside]).max() < 1e-12
    # at the aperture edge the phase spans many radians, so each factor is tested
    assert np.abs(chi[inside]).max() / abs(cs_mm) > 50.0


@pytest.mark.parametrize("b2,phi_b", [(2000.0, 0.0), (-3000.0, 0.7), (5000.0, 2.5)])
def test_coma_cartesian_form(b2, phi_b):
    # Axial coma, (2 pi / lambda) C21 theta^3 cos(phi - phi_b) / 3 at theta = lambda |k|, written
    # without angles: (2 pi / 3) C21 lambda^2 |k|^2 (kx cos phi_b + ky sin phi_b).  A 1/2 in place
    # of 1/3, a power of |k| off by one, cos(2 phi) in place of cos(phi), or a flipped sign fails.
    N, L, alpha = 96, 24.0, 30.0
    p = oracle.params(N, N, 1, (L, L, 2.0), bandlimit=0.0)
    lam = oracle.wavelength(100e3)
    KX, KY, inside = _aperture_coefficients(N, L, alpha, lam)
    chi = (2 * np.pi / 3) * b2 * lam ** 2 * (KX ** 2 + KY ** 2) * (KX * np.cos(phi_b) + KY * np.sin(phi_b))
    got = _unitary_k(oracle.probe_aberrated(p, alpha, b2=b2, phi_b=phi_b))
    amp = 1.0 / math.sqrt(inside.sum())
    assert np.abs(got[inside] - amp * np.exp(-1j * chi[inside])).max() < 1e-11
    assert np.abs(got[~inside]).max() < 1e-12
    # the coma phase spans radians across the aperture
    assert np.abs(chi[inside]).max() > 1.0


def test_coma_is_odd_and_the_other_terms_even():
    # chi(-k) = -chi(k) for coma and +chi(k) for defocus, astigmatism and Cs, so for a centred
    # probe c(k) c(-k) = amp^2 exp(-2 i chi_even(k)): the coma term cancels from the product and
    # the even terms remain.
    N, L, alpha = 64, 16.0, 28.0
    p = oracle.params(N, N, 1, (L, L, 2.0), bandlimit=0.0)
    lam = oracle.wavelength(100e3)
    ab = dict(df=20.0, cs_mm=0.9, a1=12.0, phi_a=0.4)
    even = _unitary_k(oracle.probe_aberrated(p, alpha, **ab))
    both = _unitary_k(oracle.probe_aberrated(p, alpha, b2=1200.0, phi_b=1.1, **ab))
    flip = lambda c: np.roll(c[::-1, ::-1], 1, axis=(0, 1))  # c(-k) on the fftfreq grid
    assert np.abs(both * flip(both) - even * flip(even)).max() < 1e-14
    # and the coma does change the probe
    assert np.abs(both - even).max() > 1e-3
    # coma alone: c(-k) = conj(c(k))
    coma = _unitary_k(oracle.probe_aberrated(p, alpha, b2=1200.0, phi_b=1.1))
    assert np.abs(flip(coma) - np.conj(coma)).max() < 1e-14


def test_multislice_from_initial_waves_matches_probe_path():
    w = workloads.diamond_si(n_frames=1, grid=32, n_slices=3)
    p = oracle.params_of(w)
    xy = np.array([[1.0, 2.0], [4.5, 0.5]])
    a = oracle.multislice_frame(p, w.pos[0], w.Z, w.form_Z, w.form_coef, 30.0, xy)
    psi0 = np.stack([oracle.probe(p, 30.0, *r) for r in xy])
    b = oracle.multislice_frame_init(p, w.pos[0], w.Z, w.form_Z, w.form_coef, psi0)
    assert np.abs(a - b).max() < 1e-14
