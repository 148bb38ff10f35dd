"""GB300 (sm_103a) TACAW hot path: Python binding of libtacaw.so.

Argument marshalling only: every step of the path runs in the CUDA kernels of libtacaw.so,
whose C ABI is declared in include/tacaw.h.  torch tensors supply device memory and streams.
The module-level functions carry the C names (tacaw_build_potential, ...); ``Context`` wraps
a context handle.  There is no CPU fallback: without the built library every call raises.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

from ._build import LIB as _LIB_PATH

TACAW_OK = 0
TACAW_PENDING = 1
TACAW_EINVAL = -1
TACAW_ENOMEM = -2
TACAW_ETOOBIG = -3
TACAW_ETIMEOUT = -4
TACAW_ECUDA = -5
TACAW_ECANCELED = -6
TACAW_ENOTFOUND = -7

DFT_FP32, DFT_BF16X3, DFT_TF32X3, DFT_BF16, DFT_TF32 = 0, 1, 2, 3, 4
REDUCE_NONE, REDUCE_DETECTOR = 0, 1

_CODES = {-1: "EINVAL", -2: "ENOMEM", -3: "ETOOBIG", -4: "ETIMEOUT", -5: "ECUDA", -6: "ECANCELED", -7: "ENOTFOUND"}


class TacawError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"tacaw {_CODES.get(code, code)}: {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("n_slices", C.c_int32),
                ("bandlimit_transmission", C.c_int32), ("cell", C.c_double * 3), ("voltage_ev", C.c_double),
                ("bandlimit", C.c_double), ("dt_fs", C.c_double)]


class Probe(C.Structure):
    _fields_ = [("alpha_mrad", C.c_double), ("n_probes", C.c_int32), ("pad_", C.c_int32), ("xy", C.c_void_p),
                ("defocus", C.c_double), ("cs_mm", C.c_double), ("astig", C.c_double), ("astig_angle", C.c_double),
                ("psi0", C.c_void_p), ("coma", C.c_double), ("coma_angle", C.c_double)]


def make_params(nx, ny, n_slices, cell, voltage_ev=100e3, bandlimit=2.0 / 3.0, bandlimit_transmission=1,
                dt_fs=1.0) -> Params:
    p = Params()
    p.nx, p.ny, p.n_slices, p.bandlimit_transmission = int(nx), int(ny), int(n_slices), int(bandlimit_transmission)
    p.cell[0], p.cell[1], p.cell[2] = (float(c) for c in cell)
    p.voltage_ev, p.bandlimit, p.dt_fs = float(voltage_ev), float(bandlimit), float(dt_fs)
    return p


def params_of(w, **kw) -> Params:
    """Parameters of a workloads.Workload (keyword overrides allowed)."""
    d = dict(nx=w.nx, ny=w.ny, n_slices=w.n_slices, cell=w.cell, voltage_ev=w.voltage_ev, bandlimit=w.bandlimit,
             bandlimit_transmission=w.bandlimit_transmission, dt_fs=w.dt_fs)
    d.update(kw)
    return make_params(**d)


class Request(C.Structure):
    _fields_ = [("params", Params), ("probe", Probe), ("pos", C.c_void_p), ("Z", C.c_void_p),
                ("n_atoms", C.c_int64), ("n_frames", C.c_int64), ("precision", C.c_int32), ("reduce", C.c_int32),
                ("S_out", C.c_void_p)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("batched", C.c_int32), ("footprint_bytes", C.c_uint64),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double)]


class ProbeSpec:
    """A tacaw_probe plus the buffers its pointers refer to.  psi0: optional device complex64
    tensor [P][ny][nx] of real-space initial waves used instead of the aperture probe."""

    def __init__(self, alpha_mrad=0.0, xy=None, defocus=0.0, cs_mm=0.0, astig=0.0, astig_angle=0.0, psi0=None,
                 coma=0.0, coma_angle=0.0):
        self.xy = None if xy is None else np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
        self.psi0 = psi0
        n = 1 if self.xy is None else self.xy.shape[0]
        if psi0 is not None:
            n = psi0.shape[0]
        self.c = Probe(float(alpha_mrad), n, 0, None if self.xy is None else self.xy.ctypes.data, float(defocus),
                       float(cs_mm), float(astig), float(astig_angle),
                       None if psi0 is None else _ptr(psi0), float(coma), float(coma_angle))

    @property
    def n_probes(self):
        return self.c.n_probes


def probe_of(w) -> ProbeSpec:
    return ProbeSpec(w.alpha_mrad, w.probes if w.alpha_mrad > 0 else None)


# ------------------------------------------------------------------------------------------
# library loading
# ------------------------------------------------------------------------------------------
_lib = None


def lib():
    """The loaded libtacaw.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"libtacaw.so is not built ({_LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(_LIB_PATH)
        vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int32
        pp, prp = C.POINTER(Params), C.POINTER(Probe)
        sig = {
            "tacaw_version": (C.c_char_p, []),
            "tacaw_axes": (C.c_int, [pp, i64, vp, vp, vp, vp]),
            "tacaw_create": (C.c_int, [C.POINTER(vp), i32, C.c_uint64]),
            "tacaw_destroy": (C.c_int, [vp]),
            "tacaw_last_error": (C.c_char_p, [vp]),
            "tacaw_load_form_factors": (C.c_int, [vp, vp, vp, i32]),
            "tacaw_bin_slices": (C.c_int, [vp, pp, vp, i64, i64, vp, vp]),
            "tacaw_build_potential": (C.c_int, [vp, pp, vp, vp, i64, i64, vp, vp]),
            "tacaw_transmission": (C.c_int, [vp, pp, vp, i64, vp, vp]),
            "tacaw_propagate": (C.c_int, [vp, pp, vp, i64, prp, vp, vp]),
            "tacaw_spectrum": (C.c_int, [vp, vp, i64, i64, i64, i32, i32, vp, i64, vp, vp]),
            "tacaw_run": (C.c_int, [vp, pp, vp, vp, i64, i64, prp, i32, i32, vp, vp]),
            "tacaw_check": (C.c_int, [vp]),
            "tacaw_selftest_wait": (C.c_int, [vp, C.c_double, vp]),
            "tacaw_set_option": (C.c_int, [vp, C.c_char_p, i64]),
            "tacaw_spectral_diffraction": (C.c_int, [vp, vp, i64, i64, i64, C.c_double, C.c_double, i32, vp, vp]),
            "tacaw_dispersion": (C.c_int, [vp, vp, i64, i64, i32, i32, C.c_double, C.c_double, vp, vp, i32, vp,
                                           vp]),
            "tacaw_accumulate": (C.c_int, [vp, vp, i64, C.c_double, vp, vp]),
            "tacaw_band_points": (C.c_int, [vp, pp, vp, C.POINTER(i64)]),
            "tacaw_spectrum_partial": (C.c_int, [vp, vp, i64, i64, i64, i64, i64, vp, vp, i64, vp, vp]),
            "tacaw_intensity": (C.c_int, [vp, vp, i64, i64, i64, vp, i64, i32, vp, vp]),
            "tacaw_spectrum_static": (C.c_int, [vp, i64, i64, i64, vp, vp]),
            "tacaw_submit": (C.c_int, [vp, C.POINTER(Request), C.POINTER(C.c_uint64)]),
            "tacaw_request_footprint": (C.c_int, [vp, C.POINTER(Request), C.POINTER(C.c_uint64)]),
            "tacaw_poll": (C.c_int, [vp, C.c_uint64, C.POINTER(Result)]),
            "tacaw_wait": (C.c_int, [vp, C.c_uint64, C.c_double, C.POINTER(Result)]),
            "tacaw_cancel": (C.c_int, [vp, C.c_uint64]),
            "tacaw_serving_hold": (C.c_int, [vp, C.c_int32]),
            "tacaw_serving_stats": (C.c_int, [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(C.c_uint64),
                                              C.POINTER(C.c_uint64)]),
            "tacaw_profile_begin": (C.c_int, [vp]),
            "tacaw_profile_select": (C.c_int, [vp, C.c_char_p]),
            "tacaw_profile_end": (C.c_int, [vp, vp, vp, vp, vp, vp, i32, C.POINTER(i32)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype, fn.argtypes = res, args
        _lib = L
    return _lib


def exported_symbols():
    return ["tacaw_version", "tacaw_axes", "tacaw_create", "tacaw_destroy", "tacaw_last_error",
            "tacaw_load_form_factors", "tacaw_bin_slices", "tacaw_build_potential", "tacaw_transmission",
            "tacaw_propagate", "tacaw_spectrum", "tacaw_run", "tacaw_check", "tacaw_profile_begin",
            "tacaw_profile_select", "tacaw_profile_end", "tacaw_spectrum_static", "tacaw_submit",
            "tacaw_request_footprint", "tacaw_poll", "tacaw_wait", "tacaw_cancel", "tacaw_serving_hold",
            "tacaw_serving_stats", "tacaw_set_option", "tacaw_spectral_diffraction", "tacaw_dispersion",
            "tacaw_accumulate", "tacaw_selftest_wait", "tacaw_band_points", "tacaw_spectrum_partial",
            "tacaw_intensity"]


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors passed to libtacaw must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("arrays passed to libtacaw must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"cannot pass {type(x)} to libtacaw")


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(ctx, rc):
    if rc != TACAW_OK:
        raise TacawError(rc, lib().tacaw_last_error(ctx).decode())
    return rc


# ------------------------------------------------------------------------------------------
# C names
# ------------------------------------------------------------------------------------------
def tacaw_version() -> str:
    return lib().tacaw_version().decode()


def tacaw_create(device=0, hbm_budget_bytes=0):
    h = C.c_void_p()
    rc = lib().tacaw_create(C.byref(h), int(device), int(hbm_budget_bytes))
    if rc != TACAW_OK:
        raise TacawError(rc, "tacaw_create failed")
    return h.value


def tacaw_destroy(ctx):
    return lib().tacaw_destroy(ctx)


def tacaw_load_form_factors(ctx, Z, coef):
    Z = np.ascontiguousarray(Z, dtype=np.int32)
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    return _check(ctx, lib().tacaw_load_form_factors(ctx, Z.ctypes.data, coef.ctypes.data, len(Z)))


def tacaw_bin_slices(ctx, params, pos, n_atoms, nf, slice_out, stream=None):
    return _check(ctx, lib().tacaw_bin_slices(ctx, C.byref(params), _ptr(pos), n_atoms, nf, _ptr(slice_out),
                                              _stream(stream)))


def tacaw_build_potential(ctx, params, pos, Z, n_atoms, nf, V_out, stream=None):
    return _check(ctx, lib().tacaw_build_potential(ctx, C.byref(params), _ptr(pos), _ptr(Z), n_atoms, nf,
                                                   _ptr(V_out), _stream(stream)))


def tacaw_transmission(ctx, params, V, nf, t_out, stream=None):
    return _check(ctx, lib().tacaw_transmission(ctx, C.byref(params), _ptr(V), nf, _ptr(t_out), _stream(stream)))


def tacaw_propagate(ctx, params, V, nf, probe: ProbeSpec, psi_k_out, stream=None):
    return _check(ctx, lib().tacaw_propagate(ctx, C.byref(params), _ptr(V), nf, C.byref(probe.c), _ptr(psi_k_out),
                                             _stream(stream)))


def tacaw_spectrum(ctx, psi_k, P, F, nq, precision, reduce, q_sel, n_sel, S_out, stream=None):
    return _check(ctx, lib().tacaw_spectrum(ctx, _ptr(psi_k), P, F, nq, precision, reduce, _ptr(q_sel), n_sel,
                                            _ptr(S_out), _stream(stream)))


def tacaw_run(ctx, params, pos, Z, n_atoms, n_frames, probe: ProbeSpec, precision, reduce, S_out, stream=None):
    return _check(ctx, lib().tacaw_run(ctx, C.byref(params), _ptr(pos), _ptr(Z), n_atoms, n_frames,
                                       C.byref(probe.c), precision, reduce, _ptr(S_out), _stream(stream)))


def tacaw_spectrum_static(psi_k, P, F, nq, S_out, stream=None):
    """Allocation-free FP32 time transform (no context); returns the TACAW_* code."""
    return lib().tacaw_spectrum_static(_ptr(psi_k), P, F, nq, _ptr(S_out), _stream(stream))


def make_request(params, pos, Z, n_atoms, n_frames, probe: ProbeSpec, precision, reduce, S_out) -> Request:
    return Request(params, probe.c, _ptr(pos), _ptr(Z), n_atoms, n_frames, precision, reduce, _ptr(S_out))


def tacaw_submit(ctx, req: Request) -> int:
    t = C.c_uint64()
    _check(ctx, lib().tacaw_submit(ctx, C.byref(req), C.byref(t)))
    return t.value


def tacaw_request_footprint(ctx, req: Request):
    """(code, bytes): the device bytes the request would reserve; code TACAW_OK or TACAW_ETOOBIG."""
    b = C.c_uint64()
    rc = lib().tacaw_request_footprint(ctx, C.byref(req), C.byref(b))
    if rc not in (TACAW_OK, TACAW_ETOOBIG):
        _check(ctx, rc)
    return rc, b.value


def tacaw_poll(ctx, ticket):
    """(code, Result): code is TACAW_PENDING, TACAW_OK or the request's error."""
    r = Result()
    rc = lib().tacaw_poll(ctx, ticket, C.byref(r))
    return rc, r


def tacaw_wait(ctx, ticket, timeout_s=-1.0):
    r = Result()
    rc = lib().tacaw_wait(ctx, ticket, float(timeout_s), C.byref(r))
    return rc, r


def tacaw_cancel(ctx, ticket):
    return lib().tacaw_cancel(ctx, ticket)


def tacaw_serving_hold(ctx, hold):
    """Hold (True) or release (False) admission of queued requests; see include/tacaw.h."""
    _check(ctx, lib().tacaw_serving_hold(ctx, 1 if hold else 0))


def tacaw_serving_stats(ctx):
    q, a, u, b = C.c_int64(), C.c_int64(), C.c_uint64(), C.c_uint64()
    _check(ctx, lib().tacaw_serving_stats(ctx, C.byref(q), C.byref(a), C.byref(u), C.byref(b)))
    return q.value, a.value, u.value, b.value


def tacaw_set_option(ctx, name, value):
    return _check(ctx, lib().tacaw_set_option(ctx, name.encode(), int(value)))


def tacaw_spectral_diffraction(ctx, S, P, F, nq, dt_fs, f_thz, fold, out, stream=None):
    return _check(ctx, lib().tacaw_spectral_diffraction(ctx, _ptr(S), P, F, nq, float(dt_fs), float(f_thz), int(fold),
                                                        _ptr(out), _stream(stream)))


def tacaw_dispersion(ctx, S, P, F, ny, nx, Lx, Ly, kx, ky, out, stream=None):
    kx = np.ascontiguousarray(kx, dtype=np.float64)
    ky = np.ascontiguousarray(ky, dtype=np.float64)
    return _check(ctx, lib().tacaw_dispersion(ctx, _ptr(S), P, F, ny, nx, float(Lx), float(Ly), kx.ctypes.data,
                                              ky.ctypes.data, kx.size, _ptr(out), _stream(stream)))


def tacaw_accumulate(ctx, S, n, weight, acc, stream=None):
    return _check(ctx, lib().tacaw_accumulate(ctx, _ptr(S), n, float(weight), _ptr(acc), _stream(stream)))


def tacaw_band_points(ctx, params):
    """The in-band q list (int32 numpy array) of a geometry, as tacaw_run transforms it."""
    n = C.c_int64()
    _check(ctx, lib().tacaw_band_points(ctx, C.byref(params), None, C.byref(n)))
    q = np.zeros(n.value, dtype=np.int32)
    _check(ctx, lib().tacaw_band_points(ctx, C.byref(params), q.ctypes.data, C.byref(n)))
    return q


def tacaw_spectrum_partial(ctx, psi_k, P, nf, f0, F, nq, psi_ref, q_sel, n_sel, psi_tilde, stream=None):
    return _check(ctx, lib().tacaw_spectrum_partial(ctx, _ptr(psi_k), P, nf, f0, F, nq, _ptr(psi_ref), _ptr(q_sel),
                                                    n_sel, _ptr(psi_tilde), _stream(stream)))


def tacaw_intensity(ctx, psi_tilde, P, F, n_sel, q_sel, nq, reduce, S_out, stream=None):
    return _check(ctx, lib().tacaw_intensity(ctx, _ptr(psi_tilde), P, F, n_sel, _ptr(q_sel), nq, reduce, _ptr(S_out),
                                             _stream(stream)))


def tacaw_check(ctx):
    return _check(ctx, lib().tacaw_check(ctx))


def tacaw_selftest_wait(ctx, timeout_ms, stream=None):
    """Run one bounded wait that nothing completes (see the header); the next check reports it."""
    return _check(ctx, lib().tacaw_selftest_wait(ctx, float(timeout_ms), _stream(stream)))


def tacaw_profile_begin(ctx):
    return _check(ctx, lib().tacaw_profile_begin(ctx))


def tacaw_profile_select(ctx, names=""):
    """Time only the named kernel classes (comma-separated) in the profiles that follow; the
    other launches are counted with 0 ms.  "" times every class."""
    return _check(ctx, lib().tacaw_profile_select(ctx, (names or "").encode()))


def tacaw_profile_end(ctx, max_n=64):
    """Per-kernel-class totals since tacaw_profile_begin: {name: (ms, launches, bytes, flops)}."""
    names = C.create_string_buffer(32 * max_n)
    ms = (C.c_double * max_n)()
    nl = (C.c_int64 * max_n)()
    by = (C.c_double * max_n)()
    fl = (C.c_double * max_n)()
    n = C.c_int32()
    _check(ctx, lib().tacaw_profile_end(ctx, names, ms, nl, by, fl, max_n, C.byref(n)))
    out = {}
    for i in range(min(n.value, max_n)):
        nm = names.raw[32 * i:32 * i + 32].split(b"\0")[0].decode()
        out[nm] = (ms[i], nl[i], by[i], fl[i])
    return out


# ------------------------------------------------------------------------------------------
# convenience wrapper over torch tensors
# ------------------------------------------------------------------------------------------
class Context:
    """A libtacaw context on one CUDA device; methods take torch tensors."""

    def __init__(self, device=0, hbm_budget_bytes=0):
        self.device = device
        self.h = tacaw_create(device, hbm_budget_bytes)

    def close(self):
        if self.h:
            tacaw_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self):
        tacaw_check(self.h)

    def spectral_diffraction(self, S, dt_fs, f_thz, fold=False, stream=None):
        """I(k, w=f) from S[P][F][...] (or the spectrum image from SI[P][F])."""
        import torch
        P, F = S.shape[0], S.shape[1]
        nq = int(math.prod(S.shape[2:])) if S.dim() > 2 else 1
        out = torch.empty((P,) + tuple(S.shape[2:]), dtype=torch.float32, device=S.device)
        tacaw_spectral_diffraction(self.h, S, P, F, nq, dt_fs, f_thz, fold, out, stream)
        return out

    def dispersion(self, S, cell, kx, ky, stream=None):
        """S[P][F][ny][nx] along the path (kx, ky) (1/A): [P][F][npts]."""
        import torch
        P, F, ny, nx = S.shape
        out = torch.empty((P, F, len(kx)), dtype=torch.float32, device=S.device)
        tacaw_dispersion(self.h, S, P, F, ny, nx, cell[0], cell[1], kx, ky, out, stream)
        return out

    def accumulate(self, S, acc, weight=1.0, stream=None):
        """acc (float64) += weight * S (float32), elementwise on the device."""
        tacaw_accumulate(self.h, S, S.numel(), weight, acc, stream)

    def set_option(self, name, value):
        tacaw_set_option(self.h, name, value)

    def load_form_factors(self, Z, coef):
        tacaw_load_form_factors(self.h, Z, coef)

    def bin_slices(self, params, pos, stream=None):
        import torch
        nf, A = pos.shape[0], pos.shape[1]
        out = torch.empty((nf, A), dtype=torch.int32, device=pos.device)
        tacaw_bin_slices(self.h, params, pos, A, nf, out, stream)
        return out

    def build_potential(self, params, pos, Z, stream=None):
        import torch
        nf, A = pos.shape[0], pos.shape[1]
        V = torch.empty((nf, params.n_slices, params.ny, params.nx), dtype=torch.float32, device=pos.device)
        tacaw_build_potential(self.h, params, pos, Z, A, nf, V, stream)
        return V

    def transmission(self, params, V, stream=None):
        import torch
        t = torch.empty(V.shape + (2,), dtype=torch.float32, device=V.device)
        tacaw_transmission(self.h, params, V, V.shape[0], t, stream)
        return torch.view_as_complex(t)

    def propagate(self, params, V, probe: ProbeSpec, stream=None):
        import torch
        nf = V.shape[0]
        out = torch.empty((probe.n_probes, nf, params.ny, params.nx, 2), dtype=torch.float32, device=V.device)
        tacaw_propagate(self.h, params, V, nf, probe, out, stream)
        return torch.view_as_complex(out)

    def spectrum(self, psi_k, precision=DFT_FP32, reduce=REDUCE_NONE, q_sel=None, stream=None):
        """psi_k: complex64 [P][F][...] tensor; returns S [P][F][...] (or [P][F])."""
        import torch
        P, F = psi_k.shape[0], psi_k.shape[1]
        nq = int(math.prod(psi_k.shape[2:]))
        shape = (P, F) + tuple(psi_k.shape[2:]) if reduce == REDUCE_NONE else (P, F)
        S = torch.empty(shape, dtype=torch.float32, device=psi_k.device)
        psi = torch.view_as_real(psi_k.contiguous())
        tacaw_spectrum(self.h, psi, P, F, nq, precision, reduce, q_sel, 0 if q_sel is None else q_sel.numel(), S,
                       stream)
        return S

    def run(self, params, pos, Z, probe: ProbeSpec, precision=DFT_FP32, reduce=REDUCE_NONE, out=None, stream=None):
        import torch
        F, A = pos.shape[0], pos.shape[1]
        P = probe.n_probes
        shape = (P, F, params.ny, params.nx) if reduce == REDUCE_NONE else (P, F)
        if out is None:
            out = torch.empty(shape, dtype=torch.float32, device=pos.device)
        tacaw_run(self.h, params, pos, Z, A, F, probe, precision, reduce, out, stream)
        return out


# ------------------------------------------------------------------------------------------
# axes (Supplement, "Sampling Considerations"), computed by tacaw_axes
# ------------------------------------------------------------------------------------------
def tacaw_axes(params, n_frames):
    """(kx [nx], ky [ny], f_thz [F], sampling [6]) of a simulation: see include/tacaw.h."""
    kx = np.zeros(params.nx)
    ky = np.zeros(params.ny)
    f = np.zeros(int(n_frames))
    smp = np.zeros(6)
    rc = lib().tacaw_axes(C.byref(params), int(n_frames), kx.ctypes.data, ky.ctypes.data, f.ctypes.data,
                          smp.ctypes.data)
    if rc != TACAW_OK:
        raise TacawError(rc, "tacaw_axes: bad sizes, lengths or dt")
    return kx, ky, f, smp


def frequency_axis_thz(n_frames, dt_fs):
    """Frequencies of the time-transform bins in FFT order (THz): f_m = m / (F dt)."""
    return tacaw_axes(make_params(1, 1, 1, (1.0, 1.0, 1.0), dt_fs=dt_fs), n_frames)[2]


def k_axis(n, L):
    """Spatial frequencies (cycles/A) of an n-point axis of length L, FFT order."""
    return tacaw_axes(make_params(int(n), 1, 1, (float(L), 1.0, 1.0)), 1)[0]


def sampling(params, n_frames):
    """(dk, k_max, df, f_max) along x of a simulation: 1/Lx, nx/(2 Lx) = 1/(2 dx), 1/(F dt),
    1/(2 dt) (1/A and THz)."""
    smp = tacaw_axes(params, n_frames)[3]
    return float(smp[0]), float(smp[2]), float(smp[4]), float(smp[5])
