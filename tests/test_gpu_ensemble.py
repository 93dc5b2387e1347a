"""The ensemble of independent replicas (rbsog_ensemble_*): replicas of
uneven size, composition and integrator stepped together on one GPU end in
exactly the states they reach when each is stepped alone."""
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


def replicas(rb):
    reps = []
    for k, (cells, comp, prec, integ) in enumerate([((4, 4, 4), "NaCl", "MIXED", "LANGEVIN_BAOAB"),
                                                    ((6, 6, 6), "LiCl", "FP64", "NVE_VV"),
                                                    ((8, 8, 8), "LiCl-NaCl", "MIXED", "LANGEVIN_BAOAB"),
                                                    ((5, 6, 7), "NaCl", "MIXED", "NVE_VV")]):
        w = W.rock_salt(cells, seed=20 + k, composition=comp)
        w.vel = W.maxwell_boltzmann(w, 1100.0 + 50 * k)
        prm = rb.MethodParams(P_R=20, P_F=200 + 50 * k, seed=100 + k, precision=getattr(rb, prec),
                              integrator=getattr(rb, integ), T=1100.0 + 50 * k)
        reps.append((w, prm))
    return reps


def test_ensemble_matches_replicas_alone(rb):
    reps = replicas(rb)
    ens = rb.Ensemble(0, max_replicas=len(reps))
    views = []
    for w, prm in reps:
        c = ens.add_workload(w, prm)
        c.set_velocities(w.vel)
        views.append(c)
    ens.step(7)
    ens.sync()
    for (w, prm), c in zip(reps, views):
        alone = rb.Context(0)
        alone.set_workload(w, prm)
        alone.step(7)
        pa, va, sa = alone.get_state()
        pe, ve, se = c.get_state()
        assert sa == se == 7
        np.testing.assert_array_equal(pe, pa)
        np.testing.assert_array_equal(ve, va)
        alone.close()
    ens.close()


def test_ensemble_capacity_and_errors(rb):
    w = W.rock_salt((4, 4, 4), seed=1)
    ens = rb.Ensemble(0, max_replicas=1)
    ens.add_workload(w, rb.MethodParams())
    with pytest.raises(rb.RbsogError) as e:
        ens.add_workload(w, rb.MethodParams())
    assert e.value.code == -1
    with pytest.raises(rb.RbsogError) as e:
        ens.add(w.pos, w.species, w.charge, w.mass, w.bmh, w.box * 0.7, rb.MethodParams())
    assert e.value.code in (-1, -3)
    ens.close()
