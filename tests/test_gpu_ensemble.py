"""The ensemble of independent replicas (rbsog_ensemble_*): replicas of
uneven size, composition and integrator stepped together on one GPU end in
exactly the states they reach when each is stepped alone, in the packed mode
(one launch per stage over all replicas) and in the child-graph mode, and a
mix the packing cannot take falls back to the child graphs."""
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


def packable_replicas(rb, list_every, integ):
    """Mixed precision, one integrator and list mode; sizes from 512 atoms
    (short box: minimum-image walk) to 4096, three compositions."""
    reps = []
    for k, (cells, comp) in enumerate([((4, 4, 4), "NaCl"), ((8, 8, 8), "LiCl-NaCl"), ((5, 6, 7), "LiCl"),
                                       ((4, 5, 4), "NaCl"), ((7, 7, 7), "NaCl")]):
        w = W.rock_salt(cells, seed=40 + k, composition=comp)
        w.vel = W.maxwell_boltzmann(w, 1100.0 + 40 * k)
        skin = min(1.0, 0.5 * float(w.box.min()) - 12.0 - 0.01) if list_every else 0.0
        prm = rb.MethodParams(P_R=20, P_F=150 + 70 * k, seed=300 + k, precision=rb.MIXED,
                              integrator=integ, T=1100.0 + 40 * k, list_every=list_every, skin=skin)
        reps.append((w, prm))
    return reps


@pytest.mark.parametrize("list_every,integ,groups", [(0, "LANGEVIN_BAOAB", 1), (-1, "LANGEVIN_BAOAB", 1),
                                                     (-1, "NVE_VV", 1), (-1, "LANGEVIN_BAOAB", 2), (0, "NVE_VV", 9)])
def test_packed_ensemble_bit_identical(rb, list_every, integ, groups):
    reps = packable_replicas(rb, list_every, getattr(rb, integ))
    ens = rb.Ensemble(0, max_replicas=len(reps))
    ens.set_groups(groups)
    views = []
    for w, prm in reps:
        c = ens.add_workload(w, prm)
        c.set_velocities(w.vel)
        views.append(c)
    ens.step(5)
    assert ens.used_mode() == rb.ENSEMBLE_PACKED
    ens.step(4)                                  # the same graph again
    ens.sync()
    for (w, prm), c in zip(reps, views):
        alone = rb.Context(0)
        alone.set_workload(w, prm)
        alone.step(9)
        pa, va, sa = alone.get_state()
        pe, ve, se = c.get_state()
        assert sa == se == 9
        np.testing.assert_array_equal(pe, pa)
        np.testing.assert_array_equal(ve, va)
        if list_every:
            assert c.list_builds() == alone.list_builds()
        alone.close()
    # and a direct step of one replica in between, then the packed steps again
    views[1].step(2)
    ens.step(3)
    ens.sync()
    assert views[1].get_state()[2] == 14 and views[0].get_state()[2] == 12
    ens.close()


def test_packed_ensemble_falls_back(rb):
    """An FP64 replica among mixed ones: the step runs as child graphs."""
    reps = replicas(rb)
    ens = rb.Ensemble(0, max_replicas=len(reps))
    for w, prm in reps:
        ens.add_workload(w, prm).set_velocities(w.vel)
    ens.step(2)
    assert ens.used_mode() == rb.ENSEMBLE_GRAPHS
    ens.sync()
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


def _alone(rb, w, prm, nsteps):
    alone = rb.Context(0)
    alone.set_workload(w, prm)
    alone.step(nsteps)
    out = alone.get_state()
    alone.close()
    return out


def test_ensemble_graph_rebuilt_after_direct_steps(rb):
    """One graph per ensemble step; a replica stepped on its own in between
    (and re-captured after a profiling switch) keeps every state exact."""
    import dataclasses
    reps = replicas(rb)
    reps[1] = (reps[1][0], dataclasses.replace(reps[1][1], list_every=-1, skin=1.0))   # kept lists, automatic
    reps[2] = (reps[2][0], dataclasses.replace(reps[2][1], integrator=rb.NOSE_HOOVER, tdamp=0.05))
    ens = rb.Ensemble(0, max_replicas=len(reps))
    views = []
    for w, prm in reps:
        c = ens.add_workload(w, prm)
        c.set_velocities(w.vel)
        views.append(c)
    ens.step(3)
    views[0].step(2)
    views[3].set_profiling(True)                 # forces a new step graph
    ens.step(2)
    ens.sync()
    for k, ((w, prm), c) in enumerate(zip(reps, views)):
        n = 7 if k == 0 else 5
        pa, va, sa = _alone(rb, w, prm, n)
        pe, ve, se = c.get_state()
        assert sa == se == n
        np.testing.assert_array_equal(pe, pa)
        np.testing.assert_array_equal(ve, va)
    ens.close()


def test_ensemble_fixed_schedule_replicas(rb):
    """Kept lists on a fixed rebuild schedule: each replica launches its own
    graphs (the host picks the variant per step); states exact."""
    import dataclasses
    reps = [(w, dataclasses.replace(prm, list_every=3, skin=1.0)) for w, prm in replicas(rb)[1:3]]
    ens = rb.Ensemble(0, max_replicas=2)
    views = []
    for w, prm in reps:
        c = ens.add_workload(w, prm)
        c.set_velocities(w.vel)
        views.append(c)
    ens.step(7)
    ens.sync()
    for (w, prm), c in zip(reps, views):
        pa, va, sa = _alone(rb, w, prm, 7)
        pe, ve, se = c.get_state()
        np.testing.assert_array_equal(pe, pa)
        np.testing.assert_array_equal(ve, va)
    ens.close()
