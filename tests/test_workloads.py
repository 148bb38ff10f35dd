"""The seeded input generators: determinism and the stated distributions."""
import math

import numpy as np

import workloads


def test_splitmix64_reference_values():
    # SplitMix64 seeded with 0: the first outputs of the published generator.
    g = workloads.SplitMix64(0)
    assert [g.next_u64() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_generators_are_byte_identical_per_seed():
    a = workloads.config1()
    b = workloads.config1()
    assert a.pos.tobytes() == b.pos.tobytes()
    c = workloads.diamond_si(seed=99)
    assert c.pos.tobytes() != a.pos.tobytes()


def test_config1_shape_and_amplitude():
    w = workloads.config1()
    assert w.pos.shape == (64, 64, 3) and w.pos.dtype == np.float32
    assert np.allclose(w.cell, 10.86)
    u = w.pos.astype(np.float64) - w.pos.astype(np.float64).mean(axis=0)
    assert np.abs(u).max() <= 4 * 0.05 + 1e-6  # four modes of 0.05 A
    # atomic planes sit mid-slice: static heights are (i + 1/2) dz
    dz = w.cell[2] / w.n_slices
    R, _, _ = workloads.diamond(5.43, (2, 2, 2))
    frac = ((R[:, 2] + 0.5 * dz) / dz) % 1.0
    assert np.allclose(frac, 0.5)


def test_config2_rms_exact():
    w = workloads.config2(n_frames=8)
    R, _, _ = workloads.rocksalt(4.21, (10, 10, 10))
    dz = w.cell[2] / w.n_slices
    u = w.pos.astype(np.float64) - R[None] - np.array([0, 0, 0.5 * dz])
    assert abs(math.sqrt(np.mean(u * u)) - 0.06) < 1e-6
    assert w.n_atoms == 8000 and set(np.unique(w.Z)) == {8, 12}


def test_probe_grid_periodic_no_duplicate_edge():
    xy = workloads.probe_grid(32.58, 32.58, 16)
    assert xy.shape == (256, 2)
    assert np.allclose(xy[1], [32.58 / 16, 0]) and np.allclose(xy[16], [0, 32.58 / 16])
    assert xy.max() < 32.58


def test_single_mode_frequency_on_bin():
    w = workloads.single_mode_si(n_frames=32, m0=2)
    # period of F/m0 frames
    assert np.allclose(w.pos[0], w.pos[16], atol=1e-6)
    assert not np.allclose(w.pos[0], w.pos[8], atol=1e-4)


def test_request_stream_deterministic():
    a = workloads.request_stream(20)
    b = workloads.request_stream(20)
    assert a == b
    assert all(x.arrival_s < y.arrival_s for x, y in zip(a, a[1:]))


def test_minimal_example_shape():
    w = workloads.minimal_example_si(n_frames=2)
    assert w.n_atoms == 16000 and w.n_slices == 54
    assert abs(w.cell[0] - 108.62) < 1e-9 and abs(w.cell[2] - 27.155) < 1e-9
    assert w.nx == w.ny == 1152 and w.cell[0] / w.nx <= 0.1  # 0.1 A sampling, padded
