"""Host logic of the autotuners, on the CPU: which candidates each search
times, the state every candidate starts from, the candidates it rejects and
the choice of the fastest.  A stand-in context records the calls and a
synthetic step time replaces the timed MD steps (no GPU, no library call)."""
import types

import pytest

from paper_2512_24970_gb300 import autotune, rbsog

INITIAL = (1, 2, 2, 4, 1, 0, 0, 0, 0)


class FakeCtx:
    """Stands in for rbsog.Context: the calls the tuners make, recorded."""
    made = []
    fail_skins = set()

    def __init__(self, device, stream=None):
        self.sched = INITIAL
        self.log = []
        self.prm = None
        self.closed = False
        FakeCtx.made.append(self)

    def set_workload(self, w, prm):
        self.prm = prm
        if prm.skin in FakeCtx.fail_skins:
            raise rbsog.RbsogError(-4, "kept list: |B| > RBSOG_MAX_KEPT")
        return self

    def get_state(self):
        return ("x0", "v0", 7)

    def set_state(self, x, v, s):
        self.log.append(("state", x, v, s))

    def set_schedule(self, *q):
        self.sched = tuple(q)
        self.log.append(("sched", tuple(q)))

    def schedule(self):
        return self.sched

    def list_builds(self):
        return int(round(60 / self.prm.skin))

    def close(self):
        self.closed = True


@pytest.fixture
def fake(monkeypatch):
    FakeCtx.made = []
    FakeCtx.fail_skins = set()
    monkeypatch.setattr(autotune.rbsog, "Context", FakeCtx)
    return FakeCtx


STREAM = types.SimpleNamespace(cuda_stream=0)


# a separable step time with one minimum: coordinate search must find it
BEST = (6, 3, 4, 2, 0, 3, 0, 1, 2)


def cost(q):
    return 1.0 + sum(0.01 * (i + 1) * abs(a - b) for i, (a, b) in enumerate(zip(q, BEST)))


def test_tune_schedule_visits_each_group_and_finds_the_optimum(fake, monkeypatch):
    timed = []

    def fake_timed(ctx, st, warmup, steps, flush=None):
        # every candidate runs from the tuner's starting state, with its own schedule
        assert ctx.log[-1] == ("state", "x0", "v0", 7)
        assert ctx.log[-2] == ("sched", ctx.sched)
        timed.append(ctx.sched)
        return cost(ctx.sched)

    monkeypatch.setattr(autotune, "timed_steps", fake_timed)
    prm = rbsog.MethodParams(list_every=-1, skin=1.5)
    best, table = autotune.tune_schedule(object(), prm, stream=STREAM)
    assert best == BEST
    assert len(timed) == len(table) == len(set(timed))        # no candidate timed twice
    n_rho = len(autotune.RHO_VARIANTS) * len(autotune.RHO_BLOCKS_PER_SM)
    n_far = len(autotune.FAR_ATOMS) * len(autotune.FAR_SEGMENTS) * len(autotune.FAR_PACKED) - 1
    n_near = 2 * (1 + len(autotune.NEAR_BLOCKS_PER_SM)) - 1
    assert len(timed) == n_rho + n_far + n_near + 2
    # the structure-factor shapes first, with the initial far-force shape
    assert all(q[2:] == INITIAL[2:] for q in timed[:n_rho])
    # then the far-force shapes on the best structure-factor shape
    assert all(q[:2] == BEST[:2] and q[5:] == INITIAL[5:] for q in timed[n_rho:n_rho + n_far])
    # then the near field's cap and gathers, then the tile sums' form
    assert all(q[:5] == BEST[:5] and q[8] == INITIAL[8] for q in timed[n_rho + n_far:-2])
    assert [q[8] for q in timed[-2:]] == [1, 2]
    assert FakeCtx.made[-1].closed


def test_tune_schedule_per_step_lists_skip_the_near_field(fake, monkeypatch):
    monkeypatch.setattr(autotune, "timed_steps", lambda ctx, st, w, s, flush=None: cost(ctx.sched))
    prm = rbsog.MethodParams(list_every=0)
    best, table = autotune.tune_schedule(object(), prm, stream=STREAM)
    n_rho = len(autotune.RHO_VARIANTS) * len(autotune.RHO_BLOCKS_PER_SM)
    n_far = len(autotune.FAR_ATOMS) * len(autotune.FAR_SEGMENTS) * len(autotune.FAR_PACKED) - 1
    assert len(table) == n_rho + n_far + 2
    assert all(q[5] == 0 and q[7] == 0 for q, _ in table)   # the near field's fields stay as they were
    assert best[:5] == BEST[:5] and best[8] == BEST[8]


def test_tune_schedule_closes_its_context_on_error(fake, monkeypatch):
    def boom(ctx, st, w, s, flush=None):
        raise rbsog.RbsogError(-5, "launch failed")

    monkeypatch.setattr(autotune, "timed_steps", boom)
    with pytest.raises(rbsog.RbsogError):
        autotune.tune_schedule(object(), rbsog.MethodParams(list_every=-1, skin=1.0), stream=STREAM)
    assert FakeCtx.made[-1].closed


def test_tune_skin_rejects_and_chooses(fake, monkeypatch):
    monkeypatch.setattr(autotune, "timed_steps",
                        lambda ctx, st, w, s, flush=None: 1.0 + abs(ctx.prm.skin - 1.25))
    FakeCtx.fail_skins = {0.75}
    w = types.SimpleNamespace(box=(27.5, 28.0, 30.0))      # 2 (r_shell + skin) <= 27.5: skin <= 1.75
    prm = rbsog.MethodParams(r_shell=12.0, list_every=0, skin=0.0)
    best, table, rejected = autotune.tune_skin(w, prm, stream=STREAM)
    assert best == 1.25
    assert [t[0] for t in table] == [0.5, 1.0, 1.25, 1.5]
    assert [t[2] for t in table] == [120, 60, 48, 40]          # list builds of each candidate's run
    assert dict(rejected)[2.0] == "box too small"
    assert "RBSOG_MAX_KEPT" in dict(rejected)[0.75]
    # every candidate ran with automatic kept lists and its own skin, on a context of its own
    ran = [c.prm for c in FakeCtx.made if c.prm is not None]
    assert [p.skin for p in ran] == [0.5, 0.75, 1.0, 1.25, 1.5]
    assert all(p.list_every == rbsog.LISTS_AUTO for p in ran)
    assert all(c.closed for c in FakeCtx.made)


def test_tune_skin_without_a_runnable_candidate(fake, monkeypatch):
    monkeypatch.setattr(autotune, "timed_steps", lambda ctx, st, w, s, flush=None: 1.0)
    w = types.SimpleNamespace(box=(24.5, 30.0, 30.0))      # no skin >= 0.5 fits
    with pytest.raises(ValueError):
        autotune.tune_skin(w, rbsog.MethodParams(r_shell=12.0), stream=STREAM)


def test_max_skin():
    assert autotune.max_skin((30.0, 26.0, 40.0), 12.0) == pytest.approx(1.0, abs=1e-5)
