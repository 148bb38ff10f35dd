"""The C-ABI library: it loads and exports every symbol include/tacaw.h declares (no compute)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2602_10064_gb300 as T
from paper_2602_10064_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    src = open(os.path.join(ROOT, "include", "tacaw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tacaw_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    return _build.build()


def test_library_builds_and_loads(libpath):
    assert os.path.exists(libpath)
    L = ctypes.CDLL(libpath)
    assert L is not None


def test_every_declared_symbol_is_exported(libpath):
    L = ctypes.CDLL(libpath)
    syms = header_symbols()
    assert "tacaw_run" in syms and "tacaw_spectrum" in syms
    for s in syms:
        assert hasattr(L, s), s


def test_binding_covers_header():
    assert set(header_symbols()) <= set(T.exported_symbols())


def test_version_string(libpath):
    assert "sm_103a" in T.tacaw_version()


def test_create_without_gpu_fails_cleanly(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(T.TacawError):
        T.tacaw_create(0)


def test_sampling_relations_minimal_example():
    # tests/golden/minimal_example_sampling.txt: the paper's worked sampling numbers
    vals = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "minimal_example_sampling.txt")):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split("=")
            vals[k.strip()] = float(v)
    # the minimal example's cell (20 x 5.431 A, the paper's 108.6 A) at 0.1 A sampling: 1086 points
    L = vals["L_A"]
    assert abs(20 * 5.431 - L) < 0.05
    p = T.make_params(1086, 1086, 54, (L, L, 27.155), dt_fs=10.0)
    dk, kmax, df, fmax = T.sampling(p, 200)
    assert abs(dk - vals["dk_inv_A"]) < 0.0005
    assert abs(kmax - vals["kmax_inv_A"]) < 1e-12
    assert abs(df - vals["df_THz"]) < 1e-12
    assert abs(fmax - vals["fmax_THz"]) < 1e-12
    f = T.frequency_axis_thz(200, 10.0)
    assert abs(f[1] - 0.5) < 1e-12 and abs(f[100] + 50.0) < 1e-12
    assert np.allclose(T.k_axis(8, 4.0), np.fft.fftfreq(8, 0.5))
    kx, ky, f2, smp = T.tacaw_axes(T.make_params(6, 4, 1, (3.0, 2.0, 1.0), dt_fs=2.0), 5)
    assert np.allclose(kx, np.fft.fftfreq(6, 0.5)) and np.allclose(ky, np.fft.fftfreq(4, 0.5))
    assert np.allclose(f2, np.fft.fftfreq(5, 2e-3))
    assert np.allclose(smp, [1 / 3.0, 1 / 2.0, 1.0, 1.0, 100.0, 250.0])
    with pytest.raises(T.TacawError):
        T.tacaw_axes(T.make_params(6, 4, 1, (3.0, 2.0, 1.0), dt_fs=0.0), 5)


def test_params_struct_layout():
    p = T.make_params(128, 64, 8, (10.0, 11.0, 12.0), dt_fs=5.0)
    assert ctypes.sizeof(p) == 4 * 4 + 8 * 3 + 8 * 3
    assert (p.nx, p.ny, p.n_slices, p.bandlimit_transmission) == (128, 64, 8, 1)
    assert list(p.cell) == [10.0, 11.0, 12.0]
