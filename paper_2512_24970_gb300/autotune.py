"""Autotuners: the kept random batch lists' skin, and the launch schedule of
the mixed-precision far field.

With kept lists (``list_every = -1``) the skin trades the cost of a list build
(its candidate tests grow as (r_shell + skin)^3) against how often one is needed
(an atom must move skin/2), and the size of B against the batch's hit rate.
The best value depends on the temperature, the masses and the size of the
system, so it is measured: each candidate skin is run on a scratch context from
the same state, the steps are timed with CUDA events on the launching stream,
and the fastest is chosen.  Every candidate gives an unbiased estimator of the
same force, so the choice changes the samples, not what they estimate; runs
that must be reproducible pass the chosen skin explicitly.

The far-field schedule (``rbsog_schedule``: the structure factor's block shape
and tiles per SM, the far force's atoms per thread and k segments per block,
and how many blocks per SM the kept near field beside them may hold) changes
nothing but the order of partial sums.  Which shape is fastest depends
on N, P_F and on what the near field leaves of the SMs (the two branches of
the step run concurrently), so whole MD steps are timed for each candidate, by
coordinate search: the structure-factor shapes first, then the far-force ones.
"""
from __future__ import annotations

import dataclasses

from . import rbsog

DEFAULT_SKINS = (0.5, 0.75, 1.0, 1.25, 1.5, 2.0)


def max_skin(box, r_shell: float) -> float:
    """Largest skin the box allows (every length >= 2 (r_shell + skin))."""
    return 0.5 * float(min(box)) - r_shell - 1e-6


def tune_skin(w, params: "rbsog.MethodParams", device: int = 0, stream=None,
              skins=DEFAULT_SKINS, warmup: int = 20, steps: int = 500):
    """Time ``steps`` MD steps (after ``warmup``) of workload ``w`` for every
    candidate skin and return (best skin, [(skin, ms per step, list builds)],
    [(skin, reason)] of the candidates the system cannot run: a box shorter
    than 2 (r_shell + skin), or a list capacity the wider cells exceed).
    ``stream``: a torch CUDA stream to run on (default: the current one)."""
    import torch
    dev = torch.device("cuda", device)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    limit = max_skin(w.box, params.r_shell)
    table, rejected = [], []
    for skin in skins:
        if skin > limit:
            rejected.append((float(skin), "box too small"))
            continue
        prm = dataclasses.replace(params, list_every=-1, skin=float(skin))
        ctx = rbsog.Context(device, st.cuda_stream)
        try:
            ctx.set_workload(w, prm)
            with torch.cuda.stream(st):
                ctx.step(warmup)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(st)
                ctx.step(steps)
                b.record(st)
                b.synchronize()
            ctx.sync()
        except rbsog.RbsogError as e:           # e.g. a list capacity of the wider skin
            rejected.append((float(skin), str(e)))
            ctx.close()
            continue
        table.append((float(skin), a.elapsed_time(b) / steps, ctx.list_builds()))
        ctx.close()
    if not table:
        raise ValueError("no candidate skin runs on this system: %s" % rejected)
    best = min(table, key=lambda t: t[1])[0]
    return best, table, rejected


RHO_VARIANTS = (0, 1, 2, 3, 4, 5, 6, 7)
RHO_BLOCKS_PER_SM = (1, 2, 3, 4)
FAR_ATOMS = (1, 2, 4)
FAR_SEGMENTS = (1, 2, 4, 8)
FAR_PACKED = (1, 0)
NEAR_BLOCKS_PER_SM = (1, 2, 3, 4, 6)


def _time_steps(ctx, st, warmup, steps):
    import torch
    with torch.cuda.stream(st):
        ctx.step(warmup)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        ctx.step(steps)
        b.record(st)
        b.synchronize()
    ctx.sync()
    return a.elapsed_time(b) / steps


def tune_schedule(w, params: "rbsog.MethodParams", device: int = 0, stream=None, warmup: int = 10,
                  steps: int = 100):
    """Time ``steps`` MD steps of workload ``w`` (mixed precision) on one
    context for each far-field schedule of a coordinate search and return
    (best schedule (rho_variant, rho_blocks_per_sm, far_atoms_per_thread,
    far_segments, far_packed, near_blocks_per_sm), [(schedule, ms per step)]).
    The near field's residency cap is searched last, with kept lists only."""
    import torch
    dev = torch.device("cuda", device)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    ctx = rbsog.Context(device, st.cuda_stream)
    ctx.set_workload(w, params)
    table = []
    best = ctx.schedule()
    try:
        best_t = None
        for rv in RHO_VARIANTS:
            for bps in RHO_BLOCKS_PER_SM:
                q = (rv, bps) + tuple(best[2:])
                ctx.set_schedule(*q)
                t = _time_steps(ctx, st, warmup, steps)
                table.append((q, t))
                if best_t is None or t < best_t:
                    best, best_t = q, t
        timed = best                               # the far-force shape the first search used
        for A in FAR_ATOMS:
            for S in FAR_SEGMENTS:
                for pk in FAR_PACKED:
                    q = (timed[0], timed[1], A, S, pk) + tuple(timed[5:])
                    if q == timed:
                        continue
                    ctx.set_schedule(*q)
                    t = _time_steps(ctx, st, warmup, steps)
                    table.append((q, t))
                    if t < best_t:
                        best, best_t = q, t
        if params.list_every != 0:
            timed = best
            for nb in NEAR_BLOCKS_PER_SM:
                q = tuple(timed[:5]) + (nb,)
                if q == timed:
                    continue
                ctx.set_schedule(*q)
                t = _time_steps(ctx, st, warmup, steps)
                table.append((q, t))
                if t < best_t:
                    best, best_t = q, t
    finally:
        ctx.close()
    return best, table
