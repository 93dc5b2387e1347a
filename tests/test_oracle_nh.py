"""Pins of the oracle's Nose-Hoover chain integrator (the NVT thermostat of the
paper's production runs, Sec. 3; the chain and its splitting are a reading:
Martyna, Tuckerman, Klein 1996).

  - with the deterministic force (whole shell, fixed enumerated modes) the
    extended energy K + U + sum_j Q_j v_j^2 / 2 + g kT eta_0 + kT sum_{j>0}
    eta_j is conserved to O(dt^2), and halving dt cuts its drift about 4x;
  - an infinitely slow thermostat (tdamp -> infinity) is velocity Verlet;
  - a cold start heats towards the target temperature.
"""
import numpy as np

from paper_2512_24970_gb300 import workloads as W


def make(orc, w, **kw):
    return orc.System(w.pos, w.species, w.charge, w.mass, w.bmh, w.box, **kw)


def extended_energy(orc, S, v, km):
    U = S.forces(energy=True, kmodes=km, all_shell=True)["energy"][3]
    return 0.5 * S.kinetic2(v) + U + S.chain.energy()


def test_nh_conserves_extended_energy(orc):
    w = W.rock_salt((4, 4, 4), seed=31)
    v0 = W.maxwell_boltzmann(w, 900.0)
    drifts = []
    for dt, n in ((0.002, 20), (0.001, 40)):
        S = make(orc, w)
        km = S.enumerated_modes(8)
        S.chain = orc.NHChain(3, 1200.0, 0.02, 3 * w.n - 3)
        H0 = extended_energy(orc, S, v0, km)
        v, _ = S.run(v0, n, dt, integrator=orc.INTEGRATOR_NOSE_HOOVER, T=1200.0, kmodes=km, all_shell=True)
        H1 = extended_energy(orc, S, v, km)
        drifts.append(abs(H1 - H0))
        # the thermostat did work: the chain is far from rest
        assert abs(S.chain.energy()) > 10 * drifts[-1]
    K = 0.5 * w.n * 3 * orc.KB * 900.0
    assert drifts[0] < 2e-3 * K, drifts
    assert 2.5 < drifts[0] / drifts[1] < 6.0, drifts


def test_slow_thermostat_is_velocity_verlet(orc):
    w = W.rock_salt((4, 4, 4), seed=32)
    v0 = W.maxwell_boltzmann(w, 1200.0)
    kw = dict(P_R=4000, P_F=60, seed=3)
    A = make(orc, w, **kw)
    B = make(orc, w, **kw)
    vA, _ = A.run(v0, 6, 0.001, integrator=orc.INTEGRATOR_NOSE_HOOVER, T=1200.0, tdamp=1e7)
    vB, _ = B.run(v0, 6, 0.001, integrator=orc.INTEGRATOR_NVE_VV)
    np.testing.assert_allclose(A.pos, B.pos, rtol=0, atol=1e-12)
    np.testing.assert_allclose(vA, vB, rtol=1e-10, atol=1e-10)


def test_nh_heats_cold_start(orc):
    w = W.rock_salt((4, 4, 4), seed=33)
    v0 = W.maxwell_boltzmann(w, 300.0)
    S = make(orc, w, P_R=20, P_F=60, seed=4)
    T0 = S.kinetic2(v0) / (3 * w.n * orc.KB)
    v, _ = S.run(v0, 60, 0.001, integrator=orc.INTEGRATOR_NOSE_HOOVER, T=1500.0, tdamp=0.01)
    T1 = S.kinetic2(v) / (3 * w.n * orc.KB)
    assert T1 > T0 + 200.0, (T0, T1)
