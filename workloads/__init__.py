"""Seeded synthetic inputs for the TACAW hot path.

This module builds the inputs that both the FP64 oracle and the CUDA path consume:
crystals (diamond and rocksalt cells), harmonic-mode trajectories standing in for the
paper's MLIP molecular dynamics, probe-position grids, a placeholder form-factor table
and serving request streams.  It computes no step of the method itself: no projected
potential, no transmission, no propagation and no time transform.

Randomness comes from SplitMix64 (Steele, Lea & Flood 2014, the constants as published by
Vigna) turned into uniform doubles from the top 53 bits and into normals by Box-Muller, so
a seed fixes every array byte for byte on any host.

Units: lengths in Angstrom, times in fs (frame spacing) and ps (inside the mode phase),
frequencies in THz, energies in meV.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_MASK64 = (1 << 64) - 1
# h in meV * ps: E[meV] = H_MEV_PS * f[THz]
H_MEV_PS = 4.135667696


class SplitMix64:
    """SplitMix64 generator with uniform and normal draws."""

    def __init__(self, seed: int):
        self.state = int(seed) & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (inclusive)."""
        return lo + int(self.uniform() * (hi - lo + 1))

    def normal(self) -> float:
        u1 = self.uniform()
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(1.0 - u1)) * math.cos(2.0 * math.pi * u2)


# --------------------------------------------------------------------------------------
# crystals
# --------------------------------------------------------------------------------------
_FCC = np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])


def _replicate(basis_frac, basis_Z, a, reps):
    nx, ny, nz = reps
    pos, Z = [], []
    for ix in range(nx):
        for iy in range(ny):
            for iz in range(nz):
                off = np.array([ix, iy, iz], dtype=np.float64)
                for b, z in zip(basis_frac, basis_Z):
                    pos.append((off + b) * a)
                    Z.append(z)
    cell = np.array([nx * a, ny * a, nz * a], dtype=np.float64)
    return np.array(pos, dtype=np.float64), np.array(Z, dtype=np.int32), cell


def diamond(a: float, reps, Z: int = 14):
    """Diamond-cubic crystal: fcc sites plus the same sites shifted by (1/4,1/4,1/4)."""
    basis = np.concatenate([_FCC, _FCC + 0.25])
    return _replicate(basis, [Z] * 8, a, reps)


def rocksalt(a: float, reps, Zc: int = 12, Za: int = 8):
    """Rocksalt crystal: cation on fcc sites, anion on fcc + (1/2,0,0)."""
    basis = np.concatenate([_FCC, (_FCC + np.array([0.5, 0.0, 0.0])) % 1.0])
    return _replicate(basis, [Zc] * 4 + [Za] * 4, a, reps)


# --------------------------------------------------------------------------------------
# harmonic-mode trajectories
# --------------------------------------------------------------------------------------
@dataclass
class Modes:
    """Plane-wave displacement modes u_j(t) = sum_m A_m e_m cos(2 pi Q_m.R_j - 2 pi f_m t + phi_m)."""

    Q: np.ndarray  # [M,3] cycles/A
    eps: np.ndarray  # [M,3] unit polarisation
    phase: np.ndarray  # [M] rad
    f_thz: np.ndarray  # [M] THz
    amp: np.ndarray  # [M] A


def random_modes(rng: SplitMix64, n_modes: int, cell, reps, e_mev=(5.0, 60.0),
                 amp: float | None = 0.05) -> Modes:
    """Draw modes commensurate with the supercell.

    Q_m = (n1,n2,n3)/L with n_i uniform in [-reps_i, reps_i]; polarisation uniform on the
    sphere; phase uniform in [0, 2 pi); energy uniform in e_mev.  amp=None draws Gaussian
    amplitudes (to be rescaled to a target RMS by the caller)."""
    Q, E, P, F, A = [], [], [], [], []
    for _ in range(n_modes):
        n = [rng.randint(-reps[i], reps[i]) for i in range(3)]
        Q.append([n[i] / cell[i] for i in range(3)])
        v = np.array([rng.normal(), rng.normal(), rng.normal()])
        E.append(v / np.linalg.norm(v))
        P.append(2.0 * math.pi * rng.uniform())
        e = e_mev[0] + (e_mev[1] - e_mev[0]) * rng.uniform()
        F.append(e / H_MEV_PS)
        A.append(amp if amp is not None else rng.normal())
    return Modes(np.array(Q), np.array(E), np.array(P), np.array(F), np.array(A))


def displacements(R: np.ndarray, modes: Modes, n_frames: int, dt_fs: float) -> np.ndarray:
    """u[F][A][3] in A (float64) for frames t_n = n * dt."""
    t_ps = np.arange(n_frames, dtype=np.float64) * (dt_fs * 1e-3)
    u = np.zeros((n_frames, R.shape[0], 3))
    for m in range(len(modes.amp)):
        arg = (2.0 * math.pi * (R @ modes.Q[m]))[None, :] - 2.0 * math.pi * modes.f_thz[m] * t_ps[:, None] \
            + modes.phase[m]
        u += modes.amp[m] * np.cos(arg)[:, :, None] * modes.eps[m][None, None, :]
    return u


def trajectory(R: np.ndarray, modes: Modes, n_frames: int, dt_fs: float, shift=(0.0, 0.0, 0.0),
               rms: float | None = None) -> np.ndarray:
    """Positions [F][A][3] float32: R + shift + u(t); with rms set, u is rescaled so its
    per-component RMS over (frame, atom, axis) is exactly rms."""
    u = displacements(R, modes, n_frames, dt_fs)
    if rms is not None:
        u *= rms / math.sqrt(float(np.mean(u * u)))
    pos = R[None, :, :] + np.asarray(shift, dtype=np.float64)[None, None, :] + u
    return pos.astype(np.float32)


# --------------------------------------------------------------------------------------
# form factors
# --------------------------------------------------------------------------------------
def placeholder_form_factors(Zs) -> tuple[np.ndarray, np.ndarray]:
    """SYNTHETIC placeholder coefficients in Kirkland's functional form.

    Row layout per Z: a1 b1 a2 b2 a3 b3 c1 d1 c2 d2 c3 d3 with
    f(q) = sum_i a_i/(q^2+b_i) + c_i exp(-d_i q^2), q in 1/A (no 2 pi), f in A.
    These are NOT Kirkland's fitted values: they have the same form and plausible
    magnitudes (f(0) of a few A), so absolute intensities are not physical."""
    Zs = np.asarray(sorted(set(int(z) for z in Zs)), dtype=np.int32)
    coef = np.zeros((len(Zs), 12))
    for i, z in enumerate(Zs):
        s = (z / 14.0) ** 0.7
        a = np.array([0.5, 1.5, 0.8]) * s
        b = np.array([0.12, 1.1, 9.0]) * (14.0 / z) ** 0.2
        c = np.array([0.06, 0.02, 0.005]) * s
        d = np.array([0.6, 3.0, 18.0])
        coef[i, 0:6:2], coef[i, 1:6:2] = a, b
        coef[i, 6:12:2], coef[i, 7:12:2] = c, d
    return Zs, coef


# --------------------------------------------------------------------------------------
# probes
# --------------------------------------------------------------------------------------
def probe_grid(Lx: float, Ly: float, n: int) -> np.ndarray:
    """n x n periodic scan positions (i L/n), no duplicated edge; p = iy * n + ix."""
    xy = np.zeros((n * n, 2))
    for iy in range(n):
        for ix in range(n):
            xy[iy * n + ix] = (ix * Lx / n, iy * Ly / n)
    return xy


# --------------------------------------------------------------------------------------
# the workloads
# --------------------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    pos: np.ndarray  # [F][A][3] float32, A
    Z: np.ndarray  # [A] int32
    cell: np.ndarray  # [3] A
    nx: int
    ny: int
    n_slices: int
    dt_fs: float
    voltage_ev: float = 100e3
    alpha_mrad: float = 0.0
    probes: np.ndarray = field(default_factory=lambda: np.zeros((1, 2)))  # [P][2] A
    form_Z: np.ndarray = None
    form_coef: np.ndarray = None
    bandlimit: float = 2.0 / 3.0
    bandlimit_transmission: int = 1

    @property
    def n_frames(self):
        return self.pos.shape[0]

    @property
    def n_atoms(self):
        return self.pos.shape[1]

    @property
    def n_probes(self):
        return self.probes.shape[0]


def _finish(name, R, Z, cell, modes, F, dt, S, n, shift_frac, rms=None, **kw):
    dz = cell[2] / S
    pos = trajectory(R, modes, F, dt, shift=(0.0, 0.0, shift_frac * dz), rms=rms)
    fz, fc = placeholder_form_factors(Z)
    return Workload(name=name, pos=pos, Z=Z, cell=cell, nx=n, ny=n, n_slices=S, dt_fs=dt,
                    form_Z=fz, form_coef=fc, **kw)


def diamond_si(n_frames=64, dt_fs=5.0, grid=128, n_slices=8, seed=1, n_modes=4, amp=0.05,
               reps=(2, 2, 2), shift_frac=0.5, name="diamond-si"):
    """Diamond Z=14, a=5.43 A; harmonic modes of fixed amplitude; planes shifted by
    shift_frac * dz so atomic planes sit inside slices."""
    R, Z, cell = diamond(5.43, reps)
    rng = SplitMix64(seed)
    modes = random_modes(rng, n_modes, cell, reps, amp=amp)
    return _finish(name, R, Z, cell, modes, n_frames, dt_fs, n_slices, grid, shift_frac)


def config1():
    """Diamond Si 2x2x2 (64 atoms, 10.86 A), 64 frames at 5 fs, 4 modes of 0.05 A,
    100 keV plane wave, 128^2, 8 slices, 2/3 band limit."""
    return diamond_si(name="c1-diamond-si-64x128sq")


def config2(n_frames=1024, seed=2):
    """Rocksalt Z=12/8, a=4.21 A, 10x10x10 (8000 atoms, 42.1 A), 1024 frames at 5 fs,
    32 Gaussian-amplitude modes rescaled to 0.06 A RMS, 100 keV plane wave, 512^2, 20 slices."""
    reps = (10, 10, 10)
    R, Z, cell = rocksalt(4.21, reps)
    rng = SplitMix64(seed)
    modes = random_modes(rng, 32, cell, reps, amp=None)
    return _finish(f"c2-rocksalt-mgo-{n_frames}x512sq", R, Z, cell, modes, n_frames, 5.0, 20, 512,
                   0.5, rms=0.06)


def config3(n_frames=256, n_scan=16, seed=3):
    """3x3x1 of the 64-atom diamond cell (576 atoms, 32.58 x 32.58 x 10.86 A), 256 frames at
    5 fs, 30 mrad probe on a 16x16 periodic scan, 256^2, 20 slices (planes shifted dz/4)."""
    reps = (6, 6, 2)
    R, Z, cell = diamond(5.43, reps)
    rng = SplitMix64(seed)
    modes = random_modes(rng, 4, cell, reps, amp=0.05)
    w = _finish(f"c3-diamond-si-scan{n_scan}-{n_frames}x256sq", R, Z, cell, modes, n_frames, 5.0,
                20, 256, 0.25, alpha_mrad=30.0, probes=probe_grid(cell[0], cell[1], n_scan))
    return w


def config4(n_frames=2048, grid=1024, seed=4):
    """The 64-atom diamond cell, 2048 frames at 2 fs, 1024^2, 20 slices (planes shifted dz/4)."""
    return diamond_si(n_frames=n_frames, dt_fs=2.0, grid=grid, n_slices=20, seed=seed, shift_frac=0.25,
                      name=f"c4-diamond-si-{n_frames}x{grid}sq")


def minimal_example_si(n_frames=200, grid=1152, n_slices=54, seed=6, n_scan=0):
    """The shape of the paper's minimal example (Supplement, "Minimal Working Example"):
    diamond Si a = 5.431 A, 20 x 20 x 5 cells (16,000 atoms, 108.62 x 108.62 x 27.155 A), 200
    frames 10 fs apart, 100 keV, 0.1 A sampling (1086 points, padded to 1152^2: 0.094 A),
    slices of ~0.5 A (54).  Thermal-like seeded displacements (32 modes, 0.06 A RMS) stand in
    for the MLIP MD."""
    reps = (20, 20, 5)
    R, Z, cell = diamond(5.431, reps)
    rng = SplitMix64(seed)
    modes = random_modes(rng, 32, cell, reps, amp=None)
    kw = {}
    if n_scan:
        kw = dict(alpha_mrad=30.0, probes=probe_grid(cell[0], cell[1], n_scan))
    return _finish(f"minimal-example-si-{n_frames}x{grid}sq", R, Z, cell, modes, n_frames, 10.0, n_slices, grid,
                   0.5, rms=0.06, **kw)


def single_mode_si(n_frames=32, m0=2, dt_fs=5.0, grid=32, n_slices=4, amp=0.05, q=(1, 0, 0),
                   reps=(1, 1, 1), phase=0.3, eps=(0.0, 0.6, 0.8)):
    """One mode whose frequency sits exactly on DFT bin m0: f = m0 / (F dt)."""
    R, Z, cell = diamond(5.43, reps)
    f_thz = m0 / (n_frames * dt_fs * 1e-3)
    e = np.asarray(eps, dtype=np.float64)
    modes = Modes(Q=np.array([[q[i] / cell[i] for i in range(3)]]), eps=(e / np.linalg.norm(e))[None],
                  phase=np.array([phase]), f_thz=np.array([f_thz]), amp=np.array([amp]))
    return _finish(f"single-mode-m{m0}", R, Z, cell, modes, n_frames, dt_fs, n_slices, grid, 0.5)


def static_si(n_frames=8, grid=32, n_slices=4):
    R, Z, cell = diamond(5.43, (1, 1, 1))
    modes = Modes(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0), np.zeros(0), np.zeros(0))
    return _finish("static", R, Z, cell, modes, n_frames, 5.0, n_slices, grid, 0.5)


def random_exit_waves(P, F, nq, seed=7, elastic=1.0, inelastic=0.01):
    """A seeded exit-wave stack psi[P][F][nq] (complex64) with a large time-independent part
    and a small fluctuating part, shaped like multislice output, for time-transform tests."""
    rng = np.random.default_rng(seed)
    base = elastic * (rng.standard_normal((P, 1, nq)) + 1j * rng.standard_normal((P, 1, nq)))
    fl = inelastic * (rng.standard_normal((P, F, nq)) + 1j * rng.standard_normal((P, F, nq)))
    return (base + fl).astype(np.complex64)


# --------------------------------------------------------------------------------------
# serving request stream
# --------------------------------------------------------------------------------------
@dataclass
class RequestSpec:
    rid: int
    arrival_s: float
    crystal: str  # "diamond" | "rocksalt"
    reps: int
    grid: int
    n_frames: int
    n_slices: int
    n_scan: int  # 0 = plane wave
    seed: int


def request_stream(n_requests=200, seed=5, rate_hz=10.0, grids=(128, 256, 512, 1024),
                   frames=(64, 128, 256, 512, 1024), slices=(8, 40), reps=(2, 13), scans=(4, 16),
                   p_plane=0.5, n_geometries=None):
    """Poisson arrivals of random cubic-cell requests (diamond Si or rocksalt Mg/O).  With
    n_geometries, every request takes one of that many seeded geometries (crystal, size, grid,
    frames, slices, probes) and its own trajectory seed: repeated screening of a few systems."""
    rng = SplitMix64(seed)

    def geometry():
        crystal = "diamond" if rng.uniform() < 0.5 else "rocksalt"
        r = rng.randint(reps[0], reps[1])
        g = grids[rng.randint(0, len(grids) - 1)]
        F = frames[rng.randint(0, len(frames) - 1)]
        S = rng.randint(slices[0], slices[1])
        scan = 0 if rng.uniform() < p_plane else rng.randint(scans[0], scans[1])
        return crystal, r, g, F, S, scan

    pool = [geometry() for _ in range(n_geometries)] if n_geometries else None
    t = 0.0
    out = []
    for i in range(n_requests):
        t += -math.log(1.0 - rng.uniform()) / rate_hz
        geo = pool[rng.randint(0, len(pool) - 1)] if pool else geometry()
        out.append(RequestSpec(i, t, *geo, rng.next_u64() & 0xFFFFFFFF))
    return out


def request_workload(spec: RequestSpec) -> Workload:
    """Materialise one serving request as a Workload."""
    reps = (spec.reps, spec.reps, spec.reps)
    rng = SplitMix64(spec.seed)
    if spec.crystal == "diamond":
        R, Z, cell = diamond(5.43, reps)
    else:
        R, Z, cell = rocksalt(4.21, reps)
    modes = random_modes(rng, 4, cell, reps, amp=0.05)
    kw = {}
    if spec.n_scan:
        kw = dict(alpha_mrad=30.0, probes=probe_grid(cell[0], cell[1], spec.n_scan))
    return _finish(f"req{spec.rid}", R, Z, cell, modes, spec.n_frames, 5.0, spec.n_slices, spec.grid,
                   0.5, **kw)


def harmonic_exit_waves(P, F, nq, bins=(3, 40, 90, 300), amps=(1e-2, 3e-3, 1e-3, 3e-4), elastic=1.0,
                        noise=1e-5, seed=8):
    """A seeded exit-wave stack whose time dependence is a few complex exponentials on given
    DFT bins (one per energy band) over a large static part plus white noise: the shape of
    a multislice stack with a handful of phonon modes, for per-band precision studies."""
    rng = np.random.default_rng(seed)
    n = np.arange(F)
    base = elastic * (rng.standard_normal((P, 1, nq)) + 1j * rng.standard_normal((P, 1, nq)))
    psi = np.repeat(base, F, axis=1).astype(np.complex128)
    for b, a in zip(bins, amps):
        c = a * (rng.standard_normal((P, 1, nq)) + 1j * rng.standard_normal((P, 1, nq)))
        psi += c * np.exp(2j * np.pi * b * n / F)[None, :, None]
    psi += noise * (rng.standard_normal((P, F, nq)) + 1j * rng.standard_normal((P, F, nq)))
    return psi.astype(np.complex64)
