"""Far-field launch schedules (rbsog_set_schedule) and their autotuner: every
structure-factor block shape and far-force split computes the same force up to
the order of its partial sums, and each stays within the mixed-precision
tolerance of the FP64 oracle; the tuner returns a schedule it timed."""
import numpy as np
import pytest

from paper_2512_24970_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-5


@pytest.fixture(scope="module")
def rb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_24970_gb300 import rbsog
    rbsog.load()
    return rbsog


def rms_rel(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


SCHEDULES = [(0, 2, 2, 4, 1, 0, 0, 0, 0), (1, 1, 1, 1, 1, 0, 0, 0, 0), (1, 4, 4, 2, 0, 0, 0, 0, 0), (2, 2, 2, 8, 1, 0, 0, 0, 0),
             (3, 1, 1, 4, 0, 0, 0, 0, 0), (3, 3, 4, 8, 1, 0, 0, 0, 0), (2, 4, 1, 2, 1, 0, 0, 0, 0), (5, 3, 2, 4, 0, 0, 0, 0, 0),
             (7, 1, 4, 1, 0, 0, 0, 0, 0), (6, 2, 2, 2, 1, 0, 0, 0, 0), (0, 2, 2, 4, 1, 0, 64, 0, 0),
             (1, 2, 2, 4, 1, 0, 1000, 0, 0), (0, 2, 2, 4, 1, 0, 0, 0, 1), (1, 4, 2, 4, 1, 0, 0, 0, 2),
             (8, 2, 2, 4, 2, 0, 0, 0, 0), (9, 3, 1, 8, 2, 0, 0, 0, 0), (9, 1, 4, 2, 2, 0, 0, 0, 0)]


@pytest.mark.parametrize("P_F", [500, 1301])       # one column of modes; three, the last ragged, odd P
def test_schedules_agree(rb, orc, P_F):
    w = W.rock_salt((7, 6, 5), seed=21, composition="LiCl-NaCl")     # N = 1680, ragged tiles
    S = orc.System(w.pos, w.species, w.charge, w.mass, w.bmh, w.box, P_R=20, P_F=P_F, seed=5, step=3)
    prm = rb.MethodParams(s=S.s, w0=float(S.w[0]), P_R=20, P_F=P_F, seed=5, precision=rb.MIXED)
    ctx = rb.Context(0)
    ctx.set_system(w.pos, w.species, w.charge, w.mass, w.bmh, w.box, prm)
    ctx.set_state(w.pos, np.zeros_like(w.pos), 3)
    o = S.forces()
    for q in SCHEDULES:
        ctx.set_schedule(*q)
        assert ctx.schedule() == q
        F = ctx.compute_forces()
        parts = ctx.debug_parts(P=P_F)
        # the same samples and arithmetic per term; the schedules differ only
        # in the order of FP32 partial sums (at most 64 atoms or one segment
        # of modes each) and FP64 tile sums: total force and rho within the
        # mixed-precision bar of the oracle for every one
        assert rms_rel(F, o["F"]) < MIXED_TOL, q
        assert rms_rel(parts["rho"], o["rho"]) < MIXED_TOL, q
    # scalar FP32 and packed FP32x2 forms of one shape: lane by lane the same operations
    ctx.set_schedule(0, 2, 2, 4, 1, 0, 0, 0, 0)
    ctx.compute_forces()
    a = ctx.debug_parts(P=P_F)
    ctx.set_schedule(4, 2, 2, 4, 0, 0, 0, 0, 0)
    ctx.compute_forces()
    b = ctx.debug_parts(P=P_F)
    np.testing.assert_array_equal(a["rho"], b["rho"])
    np.testing.assert_array_equal(a["far"], b["far"])


def test_near_residency_cap_same_forces(rb, orc):
    """Kept lists: the near field with a capped number of resident blocks
    (grid-stride over the runs of slots), and with its wide gathers, gives the
    default result bit for bit (same warps' arithmetic in the same order,
    same partials), in both precisions."""
    w = W.rock_salt((9, 8, 7), seed=23, composition="LiCl-NaCl")
    for prec in (rb.MIXED, rb.FP64):
        prm = rb.MethodParams(P_R=20, P_F=200, seed=5, precision=prec, list_every=-1, skin=1.0)
        out = []
        for nb, wide in ((0, 0), (1, 0), (3, 0), (0, 1), (2, 1)):
            ctx = rb.Context(0)
            ctx.set_system(w.pos, w.species, w.charge, w.mass, w.bmh, w.box, prm)
            ctx.set_schedule(0, 2, 2, 4, 1, nb, 0, wide, 0)
            ctx.set_velocities(W.maxwell_boltzmann(w, 1200.0))
            ctx.step(4)
            F, E = ctx.compute_forces(energy=True)
            out.append((F, E, ctx.get_state()[0]))
        for F, E, x in out[1:]:
            np.testing.assert_array_equal(F, out[0][0])
            np.testing.assert_array_equal(E, out[0][1])
            np.testing.assert_array_equal(x, out[0][2])


def test_schedule_rejects(rb):
    w = W.rock_salt((5, 5, 5), seed=1)
    ctx = rb.Context(0)
    ctx.set_system(w.pos, w.species, w.charge, w.mass, w.bmh, w.box, rb.MethodParams())
    for bad in [(10, 2, 2, 4, 1, 0, 0, 0, 0), (0, 2, 2, 4, 3, 0, 0, 0, 0), (-1, 2, 2, 4, 1, 0, 0, 0), (0, 0, 2, 4, 1, 0, 0, 0, 0), (0, 9, 2, 4, 1, 0, 0, 0, 0),
                (0, 2, 3, 4, 1, 0, 0, 0, 0), (0, 2, 2, 3, 1, 0, 0, 0, 0), (0, 2, 2, 16, 1, 0, 0, 0, 0),
                (0, 2, 2, 4, 1, -1, 0, 0, 0), (0, 2, 2, 4, 1, 17, 0, 0, 0), (0, 2, 2, 4, 1, 0, 31, 0, 0),
                (0, 2, 2, 4, 1, 0, 65537, 0, 0), (0, 2, 2, 4, 1, 0, 0, 2, 0), (0, 2, 2, 4, 1, 0, 0, 0, 3), (0, 2, 2, 4, 1, 0, 0, 0, -1)]:
        with pytest.raises(rb.RbsogError) as e:
            ctx.set_schedule(*bad)
        assert e.value.code == -1
    assert ctx.schedule() == (0, 2, 2, 4, 1, 0, 0, 0, 0)


def test_tune_schedule(rb):
    from paper_2512_24970_gb300 import autotune
    w = W.rock_salt((8, 8, 8), seed=7)
    w.vel = W.maxwell_boltzmann(w, 1200.0)
    prm = rb.MethodParams(P_R=20, P_F=300, precision=rb.MIXED, list_every=-1, skin=1.0)
    best, table = autotune.tune_schedule(w, prm, warmup=3, steps=10)
    assert best in [q for q, _ in table]
    assert all(t > 0 for _, t in table)
    assert len(table) == 10 * 4 + 3 * 4 * 3 - 1 + 2 * 6 - 1 + 2
    assert min(t for _, t in table) == dict(table)[best]
