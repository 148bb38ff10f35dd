"""Serving loop (tacaw_submit / tacaw_poll): continuous batching with admission by footprint.

Each request's S must be the same when it runs alone (tacaw_run) and when it runs in a mix of
concurrently admitted requests; a request that fails must not affect the others."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2602_10064_gb300 as T
    return T


def mix():
    """A few small requests of different shapes: plane waves and probe scans."""
    out = []
    w = workloads.diamond_si(n_frames=16, grid=64, n_slices=4, seed=51)
    out.append(w)
    w = workloads.diamond_si(n_frames=8, grid=128, n_slices=8, seed=52)
    out.append(w)
    R, Z, cell = workloads.rocksalt(4.21, (2, 2, 2))
    rng = workloads.SplitMix64(53)
    modes = workloads.random_modes(rng, 4, cell, (2, 2, 2), amp=0.05)
    out.append(workloads._finish("rs", R, Z, cell, modes, 12, 5.0, 5, 64, 0.5))
    w = workloads.diamond_si(n_frames=8, grid=64, n_slices=6, seed=54)
    w.alpha_mrad, w.probes = 30.0, workloads.probe_grid(w.cell[0], w.cell[1], 2)
    out.append(w)
    w = workloads.diamond_si(n_frames=32, grid=32, n_slices=4, reps=(1, 1, 1), seed=55)
    out.append(w)
    return out


def table_for(ws):
    zs = sorted(set(int(z) for w in ws for z in w.Z))
    return workloads.placeholder_form_factors(zs)


def run_alone(T, ctx, w, precision):
    import torch
    return ctx.run(T.params_of(w), torch.from_numpy(w.pos).cuda(), torch.from_numpy(w.Z).cuda(), T.probe_of(w),
                   precision=precision).cpu().numpy()


def submit(T, ctx, w, precision, host=False, reduce=None):
    import torch
    P = w.n_probes
    reduce = T.REDUCE_NONE if reduce is None else reduce
    shape = (P, w.n_frames, w.ny, w.nx) if reduce == T.REDUCE_NONE else (P, w.n_frames)
    if host:
        pos, Z = w.pos, w.Z
        out = np.zeros(shape, np.float32)
    else:
        pos, Z = torch.from_numpy(w.pos).cuda(), torch.from_numpy(w.Z).cuda()
        out = torch.zeros(shape, dtype=torch.float32, device="cuda")
    pr = T.probe_of(w)
    req = T.make_request(T.params_of(w), pos, Z, w.n_atoms, w.n_frames, pr, precision, reduce, out)
    t = T.tacaw_submit(ctx.h, req)
    return t, out, (pos, Z, pr)


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_each_result_same_alone_and_in_mix(T, precision):
    import torch
    code = {"fp32": T.DFT_FP32, "bf16x3": T.DFT_BF16X3}[precision]
    ws = mix()
    fz, fc = table_for(ws)
    with T.Context(0) as ctx:
        ctx.load_form_factors(fz, fc)
        alone = [run_alone(T, ctx, w, code) for w in ws]
        torch.cuda.synchronize()
        subs = [submit(T, ctx, w, code, host=(i % 2 == 1)) for i, w in enumerate(ws)]
        for (t, out, keep), ref in zip(subs, alone):
            rc, r = T.tacaw_wait(ctx.h, t, 120.0)
            assert rc == T.TACAW_OK, rc
            got = out.cpu().numpy() if hasattr(out, "cpu") else out
            assert np.array_equal(got, ref)
            assert r.t_submit <= r.t_admit <= r.t_done
        assert T.tacaw_serving_stats(ctx.h)[:3] == (0, 0, 0)


def test_small_budget_serialises_admission(T):
    ws = mix()[:3]
    fz, fc = table_for(ws)
    # budget just above the largest single footprint: requests must run one at a time
    with T.Context(0) as probe_ctx:
        probe_ctx.load_form_factors(fz, fc)
        biggest = 0
        for w in ws:
            t, out, keep = submit(T, probe_ctx, w, T.DFT_FP32)
            rc, r = T.tacaw_wait(probe_ctx.h, t, 120.0)
            assert rc == T.TACAW_OK
            biggest = max(biggest, r.footprint_bytes)
    with T.Context(0, hbm_budget_bytes=int(biggest * 1.2)) as ctx:
        ctx.load_form_factors(fz, fc)
        subs = [submit(T, ctx, w, T.DFT_FP32) for w in ws]
        results = []
        for t, out, keep in subs:
            rc, r = T.tacaw_wait(ctx.h, t, 120.0)
            assert rc == T.TACAW_OK
            results.append(r)
        # no two admitted at once whose footprints exceed the budget
        for i, a in enumerate(results):
            for b in results[i + 1:]:
                overlap = a.t_admit < b.t_done and b.t_admit < a.t_done
                if overlap:
                    assert a.footprint_bytes + b.footprint_bytes <= int(biggest * 1.2)


def test_request_larger_than_budget_is_rejected(T):
    w = mix()[1]
    fz, fc = table_for([w])
    with T.Context(0, hbm_budget_bytes=1 << 20) as ctx:
        ctx.load_form_factors(fz, fc)
        with pytest.raises(T.TacawError) as ei:
            submit(T, ctx, w, T.DFT_FP32)
        assert ei.value.code == T.TACAW_ETOOBIG


def test_failed_request_does_not_poison_others(T):
    ws = mix()
    fz, fc = table_for(ws)
    with T.Context(0) as ctx:
        ctx.load_form_factors(fz, fc)
        ref = run_alone(T, ctx, ws[0], T.DFT_FP32)
        good1 = submit(T, ctx, ws[0], T.DFT_FP32)
        # a request whose species is not in the table fails at admission
        bad = workloads.diamond_si(n_frames=4, grid=32, n_slices=2, reps=(1, 1, 1))
        bad.Z = np.full_like(bad.Z, 79)
        with pytest.raises(T.TacawError):
            submit(T, ctx, bad, T.DFT_FP32)
        good2 = submit(T, ctx, ws[0], T.DFT_FP32)
        for t, out, keep in (good1, good2):
            rc, r = T.tacaw_wait(ctx.h, t, 120.0)
            assert rc == T.TACAW_OK
            assert np.array_equal(out.cpu().numpy(), ref)


def test_cancel_queued_request(T):
    ws = mix()
    fz, fc = table_for(ws)
    with T.Context(0) as ctx:
        ctx.load_form_factors(fz, fc)
        subs = [submit(T, ctx, ws[1], T.DFT_FP32) for _ in range(8)]
        last = subs[-1][0]
        assert T.tacaw_cancel(ctx.h, last) == T.TACAW_OK
        codes = [T.tacaw_wait(ctx.h, t, 120.0)[0] for t, _, _ in subs]
        assert all(c == T.TACAW_OK for c in codes[:-1])
        assert codes[-1] in (T.TACAW_ECANCELED, T.TACAW_OK)
        assert T.tacaw_poll(ctx.h, last)[0] == T.TACAW_ENOTFOUND


@pytest.mark.parametrize("scan", [False, True])
def test_same_geometry_requests_share_a_run(T, scan):
    """Requests of one geometry (different trajectories) queued together, here under a hold of
    admission, are coalesced into runs of at most max_coalesce requests whose launches cover all
    of them; each result equals the request run alone, bit for bit."""
    import torch
    ws = []
    for k in range(6):
        w = workloads.diamond_si(n_frames=16, grid=64, n_slices=4, seed=90 + k)
        if scan:
            w.alpha_mrad, w.probes = 30.0, workloads.probe_grid(w.cell[0], w.cell[1], 2)
        ws.append(w)
    fz, fc = table_for(ws)
    reduce = T.REDUCE_DETECTOR if scan else T.REDUCE_NONE
    with T.Context(0) as ctx:
        ctx.load_form_factors(fz, fc)
        alone = []
        for w in ws:
            S = ctx.run(T.params_of(w), torch.from_numpy(w.pos).cuda(), torch.from_numpy(w.Z).cuda(),
                        T.probe_of(w), precision=T.DFT_BF16X3, reduce=reduce).cpu().numpy()
            alone.append(S)
        torch.cuda.synchronize()
        T.tacaw_set_option(ctx.h, "max_coalesce", 4)
        T.tacaw_serving_hold(ctx.h, True)
        subs = [submit(T, ctx, w, T.DFT_BF16X3, host=(i % 3 == 2), reduce=reduce) for i, w in enumerate(ws)]
        queued, active = T.tacaw_serving_stats(ctx.h)[:2]
        assert (queued, active) == (6, 0)
        T.tacaw_serving_hold(ctx.h, False)
        batched = []
        for (t, out, keep), ref in zip(subs, alone):
            rc, r = T.tacaw_wait(ctx.h, t, 300.0)
            assert rc == T.TACAW_OK, rc
            got = out.cpu().numpy() if hasattr(out, "cpu") else out
            assert np.array_equal(got, ref)
            batched.append(r.batched)
        ctx.check()
    # in submission order: the first four share a run, the last two another
    assert batched == [4, 4, 4, 4, 2, 2], batched
