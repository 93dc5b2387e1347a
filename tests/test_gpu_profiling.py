"""Stage events of a force evaluation (rbsog_set_profiling, rbsog_get_stage_times,
rbsog_get_stage_marks): the marks follow the order of each stream and of the join, and
every stage duration is the difference of its two marks."""
import numpy as np
import pytest

from paper_2512_24970_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_24970_gb300 import rbsog
    rbsog.load()
    return rbsog


@pytest.mark.parametrize("list_every", [0, -1])
def test_stage_marks(rb, list_every):
    w = W.rock_salt((8, 8, 8), seed=3)
    w.vel = W.maxwell_boltzmann(w, 1200.0)
    prm = rb.MethodParams(P_R=20, P_F=200, precision=rb.MIXED, T=1200.0, list_every=list_every,
                          skin=1.0 if list_every else 0.0)
    ctx = rb.Context(0)
    ctx.set_workload(w, prm)
    ctx.set_profiling(True)
    for _ in range(3):
        ctx.step(1)
        st = dict(zip(rb.STAGES, ctx.stage_times()))
        mk = dict(zip(rb.MARKS, ctx.stage_marks()))
        eps = 1e-3                                   # ms: event resolution
        assert mk["start"] == 0.0
        main = ["start", "prepared", "binned", "near_done", "corr_done", "joined", "end"]
        side = ["side_start", "rho_start", "rho_done", "reduce_done", "far_done"]
        for seq in (main, side):
            t = [mk[k] for k in seq]
            assert all(b >= a - eps for a, b in zip(t, t[1:])), (seq, t)
        assert mk["rho_start"] >= mk["prepared"] - eps           # the structure factor needs the coordinates
        assert mk["joined"] >= mk["far_done"] - eps
        for stage, (a, b) in {"prepare": ("start", "prepared"), "bin": ("prepared", "binned"),
                              "near": ("binned", "near_done"), "far": ("side_start", "far_done"),
                              "finish": ("joined", "end"), "total": ("start", "end"),
                              "rho": ("rho_start", "rho_done"), "farforce": ("reduce_done", "far_done")}.items():
            assert st[stage] == pytest.approx(mk[b] - mk[a], abs=eps), stage
    ctx.set_profiling(False)
    ctx.close()
