"""Pin of the oracle's BAOAB Langevin integrator (the SDE of Sec. 2.3 with the
B-A-O-A-B splitting of Leimkuhler and Matthews).

With every force zero the O-step is the exact Ornstein-Uhlenbeck update of the
velocities, v <- c1 v + sqrt((1 - c1^2) kT/m) xi with c1 = e^{-gamma dt}, so
from rest the velocity variance of each species after n steps is
(1 - e^{-2 gamma dt n}) kT/m and tends to equipartition, kT/m per component,
independently of the integrator's own arithmetic.  A wrong friction factor, a
wrong noise amplitude, a missing unit factor or a mass taken from the wrong
species fails it; the masses of Li+ and Cl- differ fivefold.  The A half
steps around the O step move a free atom by dt/2 (v_n + v_{n+1})."""
import numpy as np

from paper_2512_24970_gb300 import workloads as W

T, GAMMA, DT = 1200.0, 20.0, 0.002     # K, 1/ps, ps


def free_system(orc):
    w = W.rock_salt((4, 4, 4), seed=2, composition="LiCl")
    bmh = w.bmh.copy()
    bmh[..., 0] = 0.0      # A
    bmh[..., 3] = 0.0      # C
    bmh[..., 4] = 0.0      # D
    S = orc.System(w.pos, w.species, np.zeros_like(w.charge), w.mass, bmh, w.box, P_F=10, P_R=10, seed=4)
    return w, S


def temperature_ratio(orc, w, v):
    """Per species: mean of m v^2 per component over kT."""
    m = w.mass[w.species]
    out = {}
    for sp in np.unique(w.species):
        sel = w.species == sp
        out[int(sp)] = float((m[sel, None] * v[sel] ** 2).mean() / orc.FCONV / (orc.KB * T))
    return out


def test_baoab_free_particles_relax_to_equipartition(orc):
    w, S = free_system(orc)
    assert len(np.unique(w.species)) == 2
    v, F = S.run(np.zeros_like(w.pos), 10, DT, T=T, gamma=GAMMA)
    assert np.abs(F).max() == 0.0
    expect = 1.0 - np.exp(-2.0 * GAMMA * DT * 10)             # 0.551
    for sp, r in temperature_ratio(orc, w, v).items():
        nsamp = 3 * int((w.species == sp).sum())
        # chi-square with nsamp degrees of freedom: relative sd sqrt(2 / nsamp) (6 %)
        assert abs(r / expect - 1.0) < 5.0 * np.sqrt(2.0 / nsamp), (sp, r, expect)
    # long after the relaxation time 1/(2 gamma) = 12.5 steps: equipartition,
    # averaged over steps one relaxation time apart
    v, F = S.run(v, 90, DT, T=T, gamma=GAMMA, F=F)
    acc = {}
    for _ in range(16):
        v, F = S.run(v, 25, DT, T=T, gamma=GAMMA, F=F)
        for sp, r in temperature_ratio(orc, w, v).items():
            acc.setdefault(sp, []).append(r)
    for sp, rs in acc.items():
        nsamp = 3 * int((w.species == sp).sum()) * len(rs)
        assert abs(np.mean(rs) - 1.0) < 5.0 * np.sqrt(2.0 / nsamp), (sp, np.mean(rs))
    # the two A half steps: with no force a step moves every atom by
    # dt/2 (v_n + v_{n+1}), the velocities before and after its O step
    for _ in range(3):
        x0 = S.pos.copy()
        v1, F = S.run(v, 1, DT, T=T, gamma=GAMMA, F=F)
        # (to a few ulps of positions of up to ~30 A)
        np.testing.assert_allclose(S.pos - x0, 0.5 * DT * (v + v1), rtol=1e-12, atol=2e-14)
        v = v1
