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


def timed_steps(ctx, st, warmup, steps, flush=None):
    """ms per MD step of ``steps`` steps after ``warmup``; with ``flush`` (a
    callable that evicts the L2 cache) each step is preceded by a flush and
    timed alone, as the benchmark times its steps."""
    import torch
    with torch.cuda.stream(st):
        for _ in range(warmup):
            if flush:
                flush()
            ctx.step(1)
        if flush is None:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            ctx.step(steps)
            b.record(st)
            b.synchronize()
            ctx.sync()
            return a.elapsed_time(b) / steps
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for e0, e1 in ev:
            flush()
            e0.record(st)
            ctx.step(1)
            e1.record(st)
        ev[-1][1].synchronize()
    ctx.sync()
    return sum(e0.elapsed_time(e1) for e0, e1 in ev) / steps


def tune_skin(w, params: "rbsog.MethodParams", device: int = 0, stream=None,
              skins=DEFAULT_SKINS, warmup: int = 20, steps: int = 500, flush=None):
    """Time ``steps`` MD steps (after ``warmup``) of workload ``w`` for every
    candidate skin and return (best skin, [(skin, ms per step, list builds)],
    [(skin, reason)] of the candidates the system cannot run: a box shorter
    than 2 (r_shell + skin), or a list capacity the wider cells exceed).
    ``stream``: a torch CUDA stream to run on (default: the current one);
    ``flush``: see timed_steps."""
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
            t = timed_steps(ctx, st, warmup, steps, flush)
        except rbsog.RbsogError as e:           # e.g. a list capacity of the wider skin
            rejected.append((float(skin), str(e)))
            ctx.close()
            continue
        table.append((float(skin), t, ctx.list_builds()))
        ctx.close()
    if not table:
        raise ValueError("no candidate skin runs on this system: %s" % rejected)
    best = min(table, key=lambda t: t[1])[0]
    return best, table, rejected


RHO_VARIANTS = (0, 1, 2, 3, 4, 5, 6, 7, 8, 9)
RHO_BLOCKS_PER_SM = (1, 2, 3, 4)
FAR_ATOMS = (1, 2, 4)
FAR_SEGMENTS = (1, 2, 4, 8)
FAR_PACKED = (1, 0, 2)
NEAR_BLOCKS_PER_SM = (1, 2, 3, 4, 6)


def tune_schedule(w, params: "rbsog.MethodParams", device: int = 0, stream=None, warmup: int = 10,
                  steps: int = 100, flush=None):
    """Time ``steps`` MD steps of workload ``w`` (mixed precision) on one
    context for each far-field schedule of a coordinate search and return
    (best schedule (rho_variant, rho_blocks_per_sm, far_atoms_per_thread,
    far_segments, far_packed, near_blocks_per_sm, rho_tile_atoms, near_wide,
    rho_reduce), [(schedule, ms per step)]).
    The near field's residency cap is searched last, with kept lists only."""
    import torch
    dev = torch.device("cuda", device)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    ctx = rbsog.Context(device, st.cuda_stream)
    ctx.set_workload(w, params)
    # every candidate starts from the same state: along one long trajectory
    # later candidates would run a different (e.g. warmer) system, with more
    # list rebuilds
    x0, v0, s0 = ctx.get_state()

    def run_candidate(q):
        ctx.set_schedule(*q)
        ctx.set_state(x0, v0, s0)
        return timed_steps(ctx, st, warmup, steps, flush)

    table = []
    best = ctx.schedule()
    try:
        best_t = None
        for rv in RHO_VARIANTS:
            for bps in RHO_BLOCKS_PER_SM:
                q = (rv, bps) + tuple(best[2:])
                t = run_candidate(q)
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
                    t = run_candidate(q)
                    table.append((q, t))
                    if t < best_t:
                        best, best_t = q, t
        if params.list_every != 0:
            timed = best
            for wide in (0, 1):
                for nb in (0,) + NEAR_BLOCKS_PER_SM:
                    q = tuple(timed[:5]) + (nb, timed[6], wide) + tuple(timed[8:])
                    if q == timed:
                        continue
                    t = run_candidate(q)
                    table.append((q, t))
                    if t < best_t:
                        best, best_t = q, t
        timed = best
        for red in (1, 2):                         # the tile sums' form
            q = tuple(timed[:8]) + (red,)
            if q == timed:
                continue
            t = run_candidate(q)
            table.append((q, t))
            if t < best_t:
                best, best_t = q, t
    finally:
        ctx.close()
    return best, table


ENSEMBLE_TILE_ATOMS = (128, 256, 512, 1024)
ENSEMBLE_RHO_VARIANTS = (0, 1, 2)
ENSEMBLE_FAR = ((1, 4), (2, 4), (2, 2), (1, 8), (4, 2))
ENSEMBLE_GROUPS = (1, 2, 4, 8, 16, 0)      # 0: child graphs (each replica's own step graph)


def tune_ensemble_schedule(ens, stream=None, warmup: int = 3, steps: int = 20, flush=None):
    """The launch plan of a packed ensemble, timed on whole ensemble steps by
    coordinate search: atoms per structure-factor tile (tiles in proportion to
    each replica's N; one far-field schedule for all replicas, as the packed
    launches need), replicas per packed launch (the replicas dealt into
    groups of about equal atoms, the groups as parallel graph branches; or
    child graphs), the structure factor's block shape, the far force's atoms
    per thread and k segments.  Returns ((schedule, groups), [((schedule,
    groups), ms per ensemble step)]) and leaves the best one set; groups 0
    stands for child graphs."""
    import torch
    from . import rbsog as rb
    st = stream if stream is not None else torch.cuda.current_stream()

    def apply(q, groups):
        for c in ens.replicas:
            c.set_schedule(*q)
        if groups:
            ens.set_mode(rb.ENSEMBLE_PACKED)
            ens.set_groups(groups)
        else:
            ens.set_mode(rb.ENSEMBLE_GRAPHS)

    def time_it():
        with torch.cuda.stream(st):
            for _ in range(warmup):
                if flush:
                    flush()
                ens.step(1)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            for a, b in ev:
                if flush:
                    flush()
                a.record(st)
                ens.step(1)
                b.record(st)
            ev[-1][1].synchronize()
        ens.sync()
        return sum(a.elapsed_time(b) for a, b in ev) / steps

    table = []
    best, best_t = None, None

    def trial(q, groups):
        nonlocal best, best_t
        apply(q, groups)
        t = time_it()
        table.append(((q, groups), t))
        if best_t is None or t < best_t:
            best, best_t = (q, groups), t

    for ta in ENSEMBLE_TILE_ATOMS:
        trial((0, 2, 2, 4, 1, 0, ta, 0, 0), 4)
    q0, g0 = best
    for g in ENSEMBLE_GROUPS:
        if g != g0:
            trial(q0, g)
    q0, g0 = best
    for rv in ENSEMBLE_RHO_VARIANTS:
        q = (rv,) + q0[1:]
        if q != q0:
            trial(q, g0)
    q0, g0 = best
    for A, S in ENSEMBLE_FAR:
        q = q0[:2] + (A, S) + q0[4:]
        if q != q0:
            trial(q, g0)
    q0, g0 = best
    trial(q0[:7] + (1 - q0[7],) + q0[8:], g0)     # the near field's wide gathers
    apply(*best)
    return best, table
