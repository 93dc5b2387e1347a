"""Autotuner of the kept random batch lists' skin.

With kept lists (``list_every = -1``) the skin trades the cost of a list build
(its candidate tests grow as (r_shell + skin)^3) against how often one is needed
(an atom must move skin/2), and the size of B against the batch's hit rate.
The best value depends on the temperature, the masses and the size of the
system, so it is measured: each candidate skin is run on a scratch context from
the same state, the steps are timed with CUDA events on the launching stream,
and the fastest is chosen.  Every candidate gives an unbiased estimator of the
same force, so the choice changes the samples, not what they estimate; runs
that must be reproducible pass the chosen skin explicitly.
"""
from __future__ import annotations

import dataclasses

from . import rbsog

DEFAULT_SKINS = (0.5, 0.75, 1.0, 1.25, 1.5, 2.0)


def max_skin(box, r_shell: float) -> float:
    """Largest skin the box allows (every length >= 2 (r_shell + skin))."""
    return 0.5 * float(min(box)) - r_shell - 1e-6


def tune_skin(w, params: "rbsog.MethodParams", device: int = 0, stream=None,
              skins=DEFAULT_SKINS, warmup: int = 20, steps: int = 200):
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
