"""One trajectory split by frames across processes (torch.distributed, one GPU per rank).

Frames are independent until the time transform (Supplement, "Sampling Considerations"), so
each rank propagates its own contiguous range of frames and forms the partial time transform of
that range against a reference wave every rank computes without communication: the exit wave of
the trajectory's first frame.  One all-reduce (SUM) of the partial transforms gives the
transform of the whole trajectory at every bin but w = 0, where the mean-subtracted transform
vanishes (tacaw_spectrum_partial and tacaw_intensity in include/tacaw.h).  Argument marshalling
and the collective only: every step of the path runs in libtacaw.so.
"""
from __future__ import annotations

from . import (REDUCE_NONE, ProbeSpec, tacaw_band_points, tacaw_intensity, tacaw_spectrum_partial)


def frame_range(n_frames: int, rank: int, world: int) -> tuple[int, int]:
    """[f0, f1) of rank's contiguous share of n_frames (the first n_frames % world ranks get one
    more frame)."""
    if world < 1 or not 0 <= rank < world or n_frames < world:
        raise ValueError("need 0 <= rank < world <= n_frames")
    base, extra = divmod(n_frames, world)
    f0 = rank * base + min(rank, extra)
    return f0, f0 + base + (1 if rank < extra else 0)


def reduce_partials(partial, dist=None, group=None):
    """Sum the ranks' partial transforms in place (one all-reduce; no-op on one rank)."""
    if dist is not None and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(partial, op=dist.ReduceOp.SUM, group=group)
    return partial


def run_frames_sharded(ctx, params, pos_local, pos_first, Z, probe: ProbeSpec, f0: int, n_frames: int,
                       reduce=REDUCE_NONE, dist=None, group=None, stream=None):
    """S (or the spectrum image) of an n_frames trajectory of which this rank holds the frames
    [f0, f0 + len(pos_local)) (device float32 [nf][A][3]) and every rank the first frame
    (pos_first, [1][A][3]).  Every rank returns the same result."""
    import torch
    P, nf = probe.n_probes, pos_local.shape[0]
    nq = params.nx * params.ny
    q = torch.from_numpy(tacaw_band_points(ctx.h, params)).to(pos_local.device)
    nsel = q.numel()
    ref = ctx.propagate(params, ctx.build_potential(params, pos_first, Z, stream), probe, stream)[:, 0].contiguous()
    psi = ctx.propagate(params, ctx.build_potential(params, pos_local, Z, stream), probe, stream)
    part = torch.empty((P, n_frames, nsel, 2), dtype=torch.float32, device=pos_local.device)
    tacaw_spectrum_partial(ctx.h, torch.view_as_real(psi), P, nf, f0, n_frames, nq, torch.view_as_real(ref), q, nsel,
                           part, stream)
    reduce_partials(part, dist, group)
    shape = (P, n_frames, params.ny, params.nx) if reduce == REDUCE_NONE else (P, n_frames)
    S = torch.empty(shape, dtype=torch.float32, device=pos_local.device)
    tacaw_intensity(ctx.h, part, P, n_frames, nsel, q, nq, reduce, S, stream)
    return S
