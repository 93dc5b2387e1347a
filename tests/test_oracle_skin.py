"""Pins of the oracle's kept (Verlet-skin) random batch lists.

Lists built at positions r_b with outer radius r_shell + skin: A = pairs
inside r_core at r_b (summed exactly), B = the rest inside r_shell + skin
(Floyd's P_R of |B| with weight |B|/P_R); every term carries the indicator
r < r_shell at the current positions (reading of Sec. 2.2 with the paper's
neighbour lists of Sec. 3 and the per-step cost of Sec. 2.4).  What fixes
it independently of its own code:
  - skin 0 at the build positions is the per-step RBL list, sample and force
    bit for bit (Sec. 2.2);
  - taking all of B after the atoms have moved by less than skin/2 gives the
    r_shell-cutoff force at the new positions (the per-step whole-shell
    identity, itself pinned against the full cutoff sum);
  - the sampled estimator is unbiased for that force (z-test, 1/sqrt(n));
  - list membership agrees with FP64 minimum-image distances up to FP32
    rounding of the thresholds; the order is canonical on the coarser grid;
  - an MD run that takes all of B follows the per-step whole-shell run (the
    rebuild schedule and the indicator under real motion).
"""
import numpy as np

from paper_2512_24970_gb300 import workloads as W


def make(orc, w, **kw):
    return orc.System(w.pos, w.species, w.charge, w.mass, w.bmh, w.box, **kw)


def displaced(w, amp, seed):
    """Positions moved by random vectors of length < amp."""
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(w.n, 3))
    d *= (amp * rng.uniform(0.0, 1.0, size=(w.n, 1)) ** (1 / 3)) / np.linalg.norm(d, axis=1, keepdims=True)
    return w.pos + d


def test_skin_zero_is_per_step_list(orc):
    """skin = 0 at the build positions: A = core list, B = shell list, the same
    Floyd batch and the same near force, bit for bit."""
    w = W.rock_salt((5, 5, 5), seed=11)
    S0 = make(orc, w, P_R=20, seed=7, step=3)
    S1 = make(orc, w, P_R=20, seed=7, step=3, skin=0.0, list_every=1)
    sel = np.arange(0, w.n, 9)
    L0 = S0.lists(sel, cap_core=256, cap_shell=2048)
    L1 = S1.lists_skin(sel, cap_a=256, cap_b=2048)
    np.testing.assert_array_equal(L1["nA"], L0["ncore"])
    np.testing.assert_array_equal(L1["nB"], L0["nshell"])
    np.testing.assert_array_equal(L1["A"], L0["core"])
    np.testing.assert_array_equal(L1["B"], L0["shell"])
    np.testing.assert_array_equal(L1["batch"], L0["batch"])
    np.testing.assert_array_equal(L1["weight"], L0["weight"])
    F0, E0 = S0.near(energy=True)
    F1, E1 = S1.near(energy=True)
    np.testing.assert_array_equal(F1, F0)
    np.testing.assert_array_equal(E1, E0)


def test_skin_whole_batch_is_cutoff_force_after_motion(orc):
    """Atoms moved by < skin/2 since the build: A and the whole of B with the
    indicator give the r_shell-cutoff force at the new positions."""
    w = W.rock_salt((5, 5, 5), seed=12)
    skin = 1.0
    S = make(orc, w, skin=skin, list_every=10)
    S.near()                                   # builds the lists at w.pos
    S.pos = displaced(w, 0.49 * skin, 3)
    Fk = S.near(all_shell=True)
    R = make(orc, w)
    R.pos = S.pos.copy()
    Fr = R.near(all_shell=True)
    scale = np.abs(Fr).max()
    assert np.abs(Fk - Fr).max() < 1e-12 * scale
    # the kept lists really are stale: some pairs crossed r_shell since the build
    R0 = make(orc, w)
    n0 = R0.lists(np.arange(0, w.n, 5), cap_shell=2048)["nshell"]
    n1 = R.lists(np.arange(0, w.n, 5), cap_shell=2048)["nshell"]
    assert np.any(n0 != n1)


def _zstats(samples, ref):
    mean = samples.mean(0)
    sd = samples.std(0, ddof=1) / np.sqrt(samples.shape[0])
    return (mean - ref) / np.maximum(sd, 1e-300)


def test_skin_estimator_unbiased(orc):
    """E over the shell batch of the kept-list estimator = r_shell-cutoff force
    at the current positions; the error of the n-sample mean decays as 1/sqrt(n)."""
    w = W.rock_salt((5, 5, 5), seed=13)
    skin = 1.5
    S = make(orc, w, P_R=10, skin=skin, list_every=1000)
    S.near()
    S.pos = displaced(w, 0.45 * skin, 4)
    sel = np.arange(0, w.n, 20)
    R = make(orc, w)
    R.pos = S.pos.copy()
    ref = R.near(sel, all_shell=True)
    draws = []
    for step in range(400):
        S.step = step
        draws.append(S.near(sel))
    X = np.array(draws)
    z = _zstats(X, ref)
    assert np.abs(z).max() < 5.0, np.abs(z).max()
    e1 = np.sqrt(((X[:25].mean(0) - ref) ** 2).mean())
    e2 = np.sqrt(((X.mean(0) - ref) ** 2).mean())
    assert 1.5 < e1 / e2 < 7.0, (e1, e2)


def test_skin_lists_against_float64_distances(orc):
    """A / B membership against FP64 minimum-image distances at the build
    positions (radii r_core and r_shell + skin) up to FP32 rounding of the
    thresholds; B in canonical order (cell of the r_list/2 grid, u_x, j)."""
    w = W.rock_salt((5, 5, 5), seed=14)
    S = make(orc, w, skin=1.0, list_every=5)
    sel = np.arange(0, w.n, 11)
    L = S.lists_skin(sel)
    u = S.fixed_point()
    nc = S.cell_grid_skin()
    assert np.all(nc == np.floor(w.box / (0.5 * 13.0 * (1 + 2.0 ** -12))))
    cell = (u.astype(np.uint64) * nc.astype(np.uint64)) >> np.uint64(32)
    lin = cell[:, 0] + nc[0] * (cell[:, 1] + nc[1] * cell[:, 2])
    tol = 1e-4
    for q, i in enumerate(sel):
        d = w.pos - w.pos[i]
        d -= w.box * np.round(d / w.box)
        r = np.sqrt((d**2).sum(1))
        r[i] = np.inf
        A = set(L["A"][q, :L["nA"][q]].tolist())
        B = set(L["B"][q, :L["nB"][q]].tolist())
        assert not (A & B)
        assert set(np.where(r < 6.0 - tol)[0]) <= A <= set(np.where(r < 6.0 + tol)[0])
        assert set(np.where((r > 6.0 + tol) & (r < 13.0 - tol))[0]) <= B
        assert B <= set(np.where((r > 6.0 - tol) & (r < 13.0 + tol))[0])
        b_list = L["B"][q, :L["nB"][q]]
        key = np.lexsort((b_list, u[b_list, 0], lin[b_list]))
        np.testing.assert_array_equal(key, np.arange(len(b_list)))
        bt = L["batch"][q, :L["nbatch"][q]]
        assert set(bt.tolist()) <= B and len(set(bt.tolist())) == len(bt)
        assert L["weight"][q] == L["nB"][q] / S.P_R


def test_skin_run_follows_per_step_whole_shell_run(orc):
    """NVE run with kept lists (rebuilt every 3 steps) and the whole of B in
    every batch = the per-step whole-shell run; the lists are rebuilt exactly
    at the multiples of 3."""
    w = W.rock_salt((5, 5, 5), seed=15)
    v0 = W.maxwell_boltzmann(w, 1200.0)
    kw = dict(P_R=4000, P_F=50, seed=2)
    S = make(orc, w, skin=1.0, list_every=3, **kw)
    R = make(orc, w, **kw)
    vS, FS = S.run(v0, 7, 0.001, integrator=0)
    vR, FR = R.run(v0, 7, 0.001, integrator=0)
    assert S.step == 7
    np.testing.assert_allclose(S.pos, R.pos, rtol=0, atol=1e-11)
    np.testing.assert_allclose(vS, vR, rtol=0, atol=1e-9)
    assert np.abs(FS - FR).max() < 1e-11 * np.abs(FR).max()
    # lists of the last build (step 6) are those of the step-6 positions
    T = make(orc, w, skin=1.0, list_every=3, **kw)
    T.run(v0, 6, 0.001, integrator=0)
    np.testing.assert_array_equal(S.build_pos, T.pos)


def test_auto_rebuild_keeps_every_cutoff_pair(orc):
    """list_every = -1: lists rebuilt whenever an atom has moved by more than
    skin/2; with the whole of B taken, a run follows the per-step whole-shell
    run through several automatic rebuilds."""
    w = W.rock_salt((5, 5, 5), seed=16)
    v0 = W.maxwell_boltzmann(w, 3000.0)
    kw = dict(P_R=4000, P_F=50, seed=2)
    S = make(orc, w, skin=0.12, list_every=-1, **kw)
    R = make(orc, w, **kw)
    vS, FS = S.run(v0, 12, 0.001, integrator=0)
    vR, FR = R.run(v0, 12, 0.001, integrator=0)
    assert S.builds >= 2, S.builds
    np.testing.assert_allclose(S.pos, R.pos, rtol=0, atol=1e-11)
    assert np.abs(FS - FR).max() < 1e-11 * np.abs(FR).max()
    # and the displacement since the last build is within the limit
    d2 = ((S.pos - S.build_pos) ** 2).sum(1)
    assert d2.max() <= S.displacement_limit2()
