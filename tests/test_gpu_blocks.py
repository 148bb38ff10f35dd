"""Memory-bounded runs: probe blocks, the compact exit-wave stack and the detector sum fused
into the tensor-core time transform (Methods, "Data Structure Design": the spectrum image of a
probe scan).

A run propagates and transforms its probes in blocks sized to a scratch bound; each block keeps
only the in-band points of its exit waves, and the spectrum image is summed in the epilogue of
the time transform without writing S.  Blocking only regroups independent per-probe work, so
every blocking gives the same bits; the blocked runs are also held to the oracle.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

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


def scan_workload(n_frames=12, grid=64, n_slices=5, side=3, seed=61):
    w = workloads.diamond_si(n_frames=n_frames, grid=grid, n_slices=n_slices, seed=seed)
    w.alpha_mrad, w.probes = 30.0, workloads.probe_grid(w.cell[0], w.cell[1], side)
    return w


def _reset(ctx):
    for name in ("max_probe_block", "max_run_bytes", "max_chunk_frames"):
        ctx.set_option(name, 0)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_probe_blocks_give_the_same_bits(ctx, T, prec):
    w = scan_workload()
    ctx.load_form_factors(w.form_Z, w.form_coef)
    code = {"fp32": T.DFT_FP32, "bf16x3": T.DFT_BF16X3}[prec]
    p, pr, pos, Z = T.params_of(w), T.probe_of(w), dev(w.pos), dev(w.Z)
    full = ctx.run(p, pos, Z, pr, precision=code).cpu().numpy()
    image = ctx.run(p, pos, Z, pr, precision=code, reduce=T.REDUCE_DETECTOR).cpu().numpy()
    try:
        for block, chunk in [(1, 0), (2, 0), (4, 5), (5, 3), (9, 0)]:
            ctx.set_option("max_probe_block", block)
            ctx.set_option("max_chunk_frames", chunk)
            got = ctx.run(p, pos, Z, pr, precision=code).cpu().numpy()
            assert np.array_equal(got, full), (block, chunk)
            got = ctx.run(p, pos, Z, pr, precision=code, reduce=T.REDUCE_DETECTOR).cpu().numpy()
            assert np.array_equal(got, image), (block, chunk)
    finally:
        _reset(ctx)
    ctx.check()
    ref = oracle.tacaw(w)
    assert rel(full, ref) < TOL_S
    assert rel(image, ref.sum(axis=(2, 3))) < TOL_S


def test_one_probe_per_block_without_kept_transmission(ctx, T):
    # a tiny scratch bound: one probe per block, the transmission functions rebuilt for every
    # block (compact, inverse-transformed by the row pass); held to the oracle
    w = scan_workload(n_frames=8, side=2, seed=62)
    ctx.load_form_factors(w.form_Z, w.form_coef)
    p, pr, pos, Z = T.params_of(w), T.probe_of(w), dev(w.pos), dev(w.Z)
    try:
        ctx.set_option("max_run_bytes", 1)
        S = ctx.run(p, pos, Z, pr, precision=T.DFT_BF16X3).cpu().numpy()
        SI = ctx.run(p, pos, Z, pr, precision=T.DFT_BF16X3, reduce=T.REDUCE_DETECTOR).cpu().numpy()
    finally:
        _reset(ctx)
    ctx.check()
    ref = oracle.tacaw(w)
    assert rel(S, ref) < TOL_S
    assert rel(SI, ref.sum(axis=(2, 3))) < TOL_S


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "tf32x3"])
def test_detector_sum_equals_sum_of_full_spectrum(ctx, T, prec):
    w = scan_workload(n_frames=16, grid=96, side=2, seed=63)
    ctx.load_form_factors(w.form_Z, w.form_coef)
    code = {"fp32": T.DFT_FP32, "bf16x3": T.DFT_BF16X3, "tf32x3": T.DFT_TF32X3}[prec]
    p, pr, pos, Z = T.params_of(w), T.probe_of(w), dev(w.pos), dev(w.Z)
    S = ctx.run(p, pos, Z, pr, precision=code).cpu().numpy().astype(np.float64)
    SI = ctx.run(p, pos, Z, pr, precision=code, reduce=T.REDUCE_DETECTOR).cpu().numpy()
    ctx.check()
    # the same S values summed in FP64 (out-of-band q are zero in S)
    assert rel(SI, S.sum(axis=(2, 3))) < 1e-6


def test_spectrum_detector_with_q_subset_on_tensor_cores(ctx, T):
    # tacaw_spectrum's own q_sel with the fused detector sum, across several tiles per probe
    P, F, nq = 3, 40, 1500
    psi = workloads.random_exit_waves(P, F, nq, seed=64)
    qs = np.array(sorted(np.random.default_rng(5).choice(nq, 700, replace=False)), np.int32)
    ref = oracle.spectrum(psi)[:, :, qs].sum(axis=2)
    for code in (T.DFT_BF16X3, T.DFT_TF32X3):
        SI = ctx.spectrum(dev(psi), precision=code, reduce=T.REDUCE_DETECTOR, q_sel=dev(qs)).cpu().numpy()
        ctx.check()
        assert rel(SI, ref) < 2e-5


def _request(T, w, P, reduce):
    pr = T.ProbeSpec(w.alpha_mrad, np.zeros((P, 2))) if P > 1 else T.ProbeSpec()
    return pr, T.make_request(T.params_of(w), None, None, w.n_atoms, w.n_frames, pr, T.DFT_BF16X3, reduce, None)


def test_largest_serving_scan_is_admitted(ctx, T):
    """The largest request of the serving configuration (a 16 x 16 scan, 1024 frames, 1024^2,
    40 slices, 20,000 atoms) fits the default budget: its footprint is bounded by the probe
    block, not by the 256 probes."""
    import types
    w = types.SimpleNamespace(nx=1024, ny=1024, n_slices=40, cell=(54.3, 54.3, 54.3), voltage_ev=100e3,
                              bandlimit=2.0 / 3.0, bandlimit_transmission=1, dt_fs=5.0, n_atoms=20000,
                              n_frames=1024, alpha_mrad=30.0)
    ctx.load_form_factors(*workloads.placeholder_form_factors([14]))
    _, budget = T.tacaw_serving_stats(ctx.h)[2:]
    pr, req = _request(T, w, 256, T.REDUCE_DETECTOR)
    rc, big = T.tacaw_request_footprint(ctx.h, req)
    assert rc == T.TACAW_OK and big <= budget
    pr16, req16 = _request(T, w, 16, T.REDUCE_DETECTOR)
    rc, small = T.tacaw_request_footprint(ctx.h, req16)
    assert rc == T.TACAW_OK
    assert big < 2 * small + (8 << 30)
    # a bound below one probe's stack is still honoured by one-probe blocks
    ctx.set_option("max_run_bytes", 1 << 30)
    try:
        rc, one = T.tacaw_request_footprint(ctx.h, req)
    finally:
        _reset(ctx)
    assert rc == T.TACAW_OK and one < big
