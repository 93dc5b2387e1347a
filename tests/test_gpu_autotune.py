"""The skin autotuner of the kept random batch lists (autotune.tune_skin)."""
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


def test_tune_skin(rb):
    from paper_2512_24970_gb300 import autotune
    w = W.rock_salt((8, 8, 8), seed=7, composition="LiCl")
    w.vel = W.maxwell_boltzmann(w, 1300.0)
    prm = rb.MethodParams(P_R=20, P_F=200, precision=rb.MIXED, T=1300.0)
    best, table, rejected = autotune.tune_skin(w, prm, skins=(0.25, 1.0, 1.75, 20.0), warmup=5, steps=40)
    skins = [t[0] for t in table]
    assert skins == [0.25, 1.0, 1.75]
    assert [r[0] for r in rejected] == [20.0]             # 20 A does not fit the box
    assert best in skins
    assert all(t[1] > 0 for t in table)
    builds = [t[2] for t in table]
    assert builds[0] > builds[1] >= builds[2] >= 1        # a wider skin is rebuilt less often
    assert autotune.max_skin(w.box, 12.0) == pytest.approx(0.5 * 50.4 - 12.0, abs=1e-5)
