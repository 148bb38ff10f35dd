"""FP64 CPU oracle for the TACAW hot path -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  The CUDA library and its Python binding never import it; the two
implementations share nothing but the seeded inputs from ``workloads``.

The arithmetic lives in ``tacaw_oracle.c`` (plain C, FP64, in-house FFT); this module only
compiles it with gcc and marshals numpy arrays through ctypes.  See the C file's header for
the paper passages each function follows and the readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tacaw_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so next to the source (gcc, OpenMP, -O2; no -march flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        # no FP contraction: the FP64 integer decisions (slice index, masks) must round exactly
        # as written, on every host architecture.  Complex products are formed inline as
        # (ac - bd) + i(ad + bc), without the runtime's recovery of infinite or NaN operands,
        # which the finite values here never reach.
        subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11", "-ffp-contract=off",
                        "-fcx-limited-range", "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("n_slices", C.c_int32),
                ("bandlimit_transmission", C.c_int32), ("final_propagator", C.c_int32),
                ("pad_", C.c_int32), ("Lx", C.c_double), ("Ly", C.c_double), ("Lz", C.c_double),
                ("voltage_ev", C.c_double), ("bandlimit", C.c_double), ("sigma_scale", C.c_double)]


def params(nx, ny, n_slices, cell, voltage_ev=100e3, bandlimit=2.0 / 3.0, bandlimit_transmission=1,
           final_propagator=1, sigma_scale=1.0) -> Params:
    return Params(nx, ny, n_slices, bandlimit_transmission, final_propagator, 0, float(cell[0]),
                  float(cell[1]), float(cell[2]), float(voltage_ev), float(bandlimit), float(sigma_scale))


def params_of(w, **kw) -> Params:
    """Oracle parameters of a workloads.Workload (keyword overrides allowed)."""
    d = dict(nx=w.nx, ny=w.ny, n_slices=w.n_slices, cell=w.cell, voltage_ev=w.voltage_ev,
             bandlimit=w.bandlimit, bandlimit_transmission=w.bandlimit_transmission)
    d.update(kw)
    return params(**d)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp, fp, ip, vp = C.POINTER(C.c_double), C.POINTER(C.c_float), C.POINTER(C.c_int32), C.c_void_p
            pp = C.POINTER(Params)
            sig = {
                "oracle_num_threads": (C.c_int, []),
                "oracle_wavelength": (C.c_double, [C.c_double]),
                "oracle_sigma": (C.c_double, [C.c_double]),
                "oracle_kirkland_prefactor": (C.c_double, []),
                "oracle_form_factor": (C.c_double, [dp, C.c_double]),
                "oracle_kfreq": (C.c_double, [C.c_int, C.c_int, C.c_double]),
                "oracle_kbl": (C.c_double, [pp]),
                "oracle_mask": (C.c_int, [pp, C.c_int, C.c_int]),
                "oracle_slice_index": (C.c_int, [C.c_double, C.c_double, C.c_int]),
                "oracle_dft": (None, [vp, vp, C.c_int, C.c_int]),
                "oracle_dft2_brute": (None, [vp, vp, C.c_int, C.c_int, C.c_int]),
                "oracle_fft": (None, [vp, C.c_int, C.c_int]),
                "oracle_fft2": (None, [vp, C.c_int, C.c_int, C.c_int]),
                "oracle_potential_slice": (C.c_int, [pp, fp, ip, C.c_int, C.c_int, ip, dp, C.c_int, dp]),
                "oracle_transmission": (None, [pp, dp, vp]),
                "oracle_probe": (None, [pp, C.c_double, C.c_double, C.c_double, vp]),
                "oracle_multislice_frame": (C.c_int, [pp, fp, ip, C.c_int, ip, dp, C.c_int, C.c_double, dp,
                                                      C.c_int, vp, dp]),
                "oracle_multislice": (C.c_int, [pp, fp, C.c_int, ip, C.c_int, ip, dp, C.c_int, C.c_double, dp,
                                                C.c_int, vp]),
                "oracle_spectrum": (None, [vp, C.c_int, C.c_int, C.c_long, C.c_int, C.c_int, dp]),
                "oracle_mean": (None, [vp, C.c_int, C.c_int, C.c_long, vp]),
                "oracle_freq_bin": (C.c_int, [C.c_double, C.c_int, C.c_double]),
                "oracle_spectral_diffraction": (None, [dp, C.c_int, C.c_int, C.c_long, C.c_double, C.c_double,
                                                       C.c_int, dp]),
                "oracle_dispersion": (None, [dp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, dp,
                                             dp, C.c_int, dp]),
                "oracle_probe_aberrated": (None, [pp, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                                  C.c_double, C.c_double, C.c_double, C.c_double, vp]),
                "oracle_multislice_frame_init": (C.c_int, [pp, fp, ip, C.c_int, ip, dp, C.c_int, vp, C.c_int, vp]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype, fn.argtypes = res, args
            _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def num_threads() -> int:
    return lib().oracle_num_threads()


def wavelength(V):
    return lib().oracle_wavelength(float(V))


def sigma(V):
    return lib().oracle_sigma(float(V))


def kirkland_prefactor():
    return lib().oracle_kirkland_prefactor()


def form_factor(coef, q):
    c = np.ascontiguousarray(coef, dtype=np.float64)
    return lib().oracle_form_factor(_p(c, C.c_double), float(q))


def kfreq(i, n, L):
    return lib().oracle_kfreq(int(i), int(n), float(L))


def kbl(p: Params):
    return lib().oracle_kbl(C.byref(p))


def mask(p: Params) -> np.ndarray:
    L = lib()
    return np.array([[L.oracle_mask(C.byref(p), iy, ix) for ix in range(p.nx)] for iy in range(p.ny)],
                    dtype=np.int32)


def slice_index(z, Lz, S):
    return lib().oracle_slice_index(float(z), float(Lz), int(S))


def dft(x, sign=-1):
    x = _c128(x)
    out = np.empty_like(x)
    lib().oracle_dft(x.ctypes.data, out.ctypes.data, x.size, sign)
    return out


def dft2_brute(x, sign=-1):
    x = _c128(x)
    out = np.empty_like(x)
    lib().oracle_dft2_brute(x.ctypes.data, out.ctypes.data, x.shape[0], x.shape[1], sign)
    return out


def fft(x, sign=-1):
    x = _c128(x).copy()
    lib().oracle_fft(x.ctypes.data, x.size, sign)
    return x


def fft2(x, sign=-1):
    x = _c128(x).copy()
    lib().oracle_fft2(x.ctypes.data, x.shape[0], x.shape[1], sign)
    return x


def _table(form_Z, form_coef):
    return (np.ascontiguousarray(form_Z, dtype=np.int32), np.ascontiguousarray(form_coef, dtype=np.float64))


def potential_slice(p: Params, pos, Z, s, form_Z, form_coef):
    """V[ny][nx] (V A) of slice s for one frame's positions pos[A][3] (float32)."""
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    Z = np.ascontiguousarray(Z, dtype=np.int32)
    tz, tc = _table(form_Z, form_coef)
    V = np.zeros((p.ny, p.nx))
    n = lib().oracle_potential_slice(C.byref(p), _p(pos, C.c_float), _p(Z, C.c_int32), pos.shape[0], int(s),
                                     _p(tz, C.c_int32), _p(tc, C.c_double), len(tz), _p(V, C.c_double))
    if n < 0:
        raise ValueError("species missing from the form-factor table")
    return V


def transmission(p: Params, V):
    V = np.ascontiguousarray(V, dtype=np.float64)
    t = np.zeros(V.shape, dtype=np.complex128)
    lib().oracle_transmission(C.byref(p), _p(V, C.c_double), t.ctypes.data)
    return t


def probe(p: Params, alpha_mrad, xp=0.0, yp=0.0):
    psi = np.zeros((p.ny, p.nx), dtype=np.complex128)
    lib().oracle_probe(C.byref(p), float(alpha_mrad), float(xp), float(yp), psi.ctypes.data)
    return psi


def multislice_frame(p: Params, pos, Z, form_Z, form_coef, alpha_mrad=0.0, probes=None, want_V=False):
    """psi_k[P][ny][nx] (complex128) for one frame; with want_V also V[S][ny][nx]."""
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    Z = np.ascontiguousarray(Z, dtype=np.int32)
    tz, tc = _table(form_Z, form_coef)
    pr = np.ascontiguousarray(np.zeros((1, 2)) if probes is None else probes, dtype=np.float64)
    out = np.zeros((pr.shape[0], p.ny, p.nx), dtype=np.complex128)
    V = np.zeros((p.n_slices, p.ny, p.nx)) if want_V else None
    rc = lib().oracle_multislice_frame(C.byref(p), _p(pos, C.c_float), _p(Z, C.c_int32), pos.shape[0],
                                       _p(tz, C.c_int32), _p(tc, C.c_double), len(tz), float(alpha_mrad),
                                       _p(pr, C.c_double), pr.shape[0], out.ctypes.data,
                                       _p(V, C.c_double) if want_V else None)
    if rc < 0:
        raise ValueError("species missing from the form-factor table")
    return (out, V) if want_V else out


def multislice(p: Params, pos, Z, form_Z, form_coef, alpha_mrad=0.0, probes=None):
    """psi_k[P][F][ny][nx] (complex128) for all frames of pos[F][A][3] (OpenMP over frames)."""
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    Z = np.ascontiguousarray(Z, dtype=np.int32)
    tz, tc = _table(form_Z, form_coef)
    pr = np.ascontiguousarray(np.zeros((1, 2)) if probes is None else probes, dtype=np.float64)
    F, A = pos.shape[0], pos.shape[1]
    out = np.zeros((pr.shape[0], F, p.ny, p.nx), dtype=np.complex128)
    rc = lib().oracle_multislice(C.byref(p), _p(pos, C.c_float), F, _p(Z, C.c_int32), A, _p(tz, C.c_int32),
                                 _p(tc, C.c_double), len(tz), float(alpha_mrad), _p(pr, C.c_double),
                                 pr.shape[0], out.ctypes.data)
    if rc < 0:
        raise ValueError("species missing from the form-factor table")
    return out


def spectrum(psi, subtract_mean=True, direct=False):
    """S[P][F][nq] (float64) from psi[P][F][nq]: |DFT_t(psi - mean_t psi)|^2."""
    psi = _c128(psi)
    P, F = psi.shape[0], psi.shape[1]
    nq = int(np.prod(psi.shape[2:]))
    S = np.zeros((P, F, nq))
    lib().oracle_spectrum(psi.ctypes.data, P, F, nq, int(bool(subtract_mean)), int(bool(direct)),
                          _p(S, C.c_double))
    return S.reshape(psi.shape)


def mean(psi):
    psi = _c128(psi)
    P, F = psi.shape[0], psi.shape[1]
    nq = int(np.prod(psi.shape[2:]))
    m = np.zeros((P, nq), dtype=np.complex128)
    lib().oracle_mean(psi.ctypes.data, P, F, nq, m.ctypes.data)
    return m.reshape((P,) + psi.shape[2:])


def freq_bin(f_thz, F, dt_fs):
    return lib().oracle_freq_bin(float(f_thz), int(F), float(dt_fs))


def spectral_diffraction(S, dt_fs, f_thz, fold=False):
    """map[P][...] = S at the bin of f (plus the bin of -f when fold)."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    P, F = S.shape[0], S.shape[1]
    nq = int(np.prod(S.shape[2:]))
    out = np.zeros((P, nq))
    lib().oracle_spectral_diffraction(_p(S, C.c_double), P, F, nq, float(dt_fs), float(f_thz), int(bool(fold)),
                                      _p(out, C.c_double))
    return out.reshape((P,) + S.shape[2:])


def dispersion(S, cell, kx, ky):
    """out[P][F][npts]: S[P][F][ny][nx] bilinearly interpolated at the k points (1/A)."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    P, F, ny, nx = S.shape
    kx = np.ascontiguousarray(kx, dtype=np.float64)
    ky = np.ascontiguousarray(ky, dtype=np.float64)
    out = np.zeros((P, F, kx.size))
    lib().oracle_dispersion(_p(S, C.c_double), P, F, ny, nx, float(cell[0]), float(cell[1]), _p(kx, C.c_double),
                            _p(ky, C.c_double), kx.size, _p(out, C.c_double))
    return out


def probe_aberrated(p: Params, alpha_mrad, xp=0.0, yp=0.0, df=0.0, cs_mm=0.0, a1=0.0, phi_a=0.0, b2=0.0, phi_b=0.0):
    psi = np.zeros((p.ny, p.nx), dtype=np.complex128)
    lib().oracle_probe_aberrated(C.byref(p), float(alpha_mrad), float(xp), float(yp), float(df), float(cs_mm),
                                 float(a1), float(phi_a), float(b2), float(phi_b), psi.ctypes.data)
    return psi


def multislice_frame_init(p: Params, pos, Z, form_Z, form_coef, psi0):
    """psi_k[P][ny][nx] for one frame from real-space initial waves psi0[P][ny][nx]."""
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    Z = np.ascontiguousarray(Z, dtype=np.int32)
    tz, tc = _table(form_Z, form_coef)
    psi0 = _c128(psi0).reshape(-1, p.ny, p.nx)
    out = np.zeros_like(psi0)
    rc = lib().oracle_multislice_frame_init(C.byref(p), _p(pos, C.c_float), _p(Z, C.c_int32), pos.shape[0],
                                            _p(tz, C.c_int32), _p(tc, C.c_double), len(tz), psi0.ctypes.data,
                                            psi0.shape[0], out.ctypes.data)
    if rc < 0:
        raise ValueError("species missing from the form-factor table")
    return out


def tacaw(w, **kw):
    """S[P][F][ny][nx] (float64) of a workloads.Workload: multislice then the time transform."""
    p = params_of(w, **kw)
    psi = multislice(p, w.pos, w.Z, w.form_Z, w.form_coef, w.alpha_mrad, w.probes)
    return spectrum(psi)
