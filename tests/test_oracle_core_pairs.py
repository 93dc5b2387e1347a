"""Pins of species-dependent core radii (the adaptive, species-dependent
cutoff named in Sec. 1; reading: a symmetric table r_core(a, b) <= r_core, the
core/shell split of the pair (i, j) at r_core(s_i, s_j), r_shell unchanged).

  - a table equal to r_core everywhere is the default split, bit for bit;
  - membership agrees with FP64 minimum-image distances and each pair's radius;
  - the whole shell gives the r_shell-cutoff force whatever the split;
  - the sampled estimator stays unbiased for it (only its variance depends on
    the split)."""
import numpy as np

from paper_2512_24970_gb300 import workloads as W


def make(orc, w, **kw):
    return orc.System(w.pos, w.species, w.charge, w.mass, w.bmh, w.box, **kw)


def test_uniform_table_is_default(orc):
    w = W.rock_salt((5, 5, 5), seed=41, composition="LiCl-NaCl")
    ns = w.charge.size
    A = make(orc, w, P_R=20, seed=3, step=2)
    B = make(orc, w, P_R=20, seed=3, step=2, r_core_pair=np.full((ns, ns), 6.0))
    sel = np.arange(0, w.n, 7)
    La, Lb = A.lists(sel), B.lists(sel)
    for k in ("core", "ncore", "shell", "nshell", "batch", "weight"):
        np.testing.assert_array_equal(La[k], Lb[k])
    np.testing.assert_array_equal(A.near(), B.near())


def test_pair_radii_membership(orc):
    w = W.rock_salt((5, 5, 5), seed=42, composition="LiCl-NaCl")
    rc = W.core_radii_from_sigma(w.bmh, 6.0)
    assert rc.max() == 6.0 and rc.min() < 5.0
    S = make(orc, w, r_core_pair=rc)
    sel = np.arange(0, w.n, 13)
    L = S.lists(sel)
    tol = 1e-4
    for q, i in enumerate(sel):
        d = w.pos - w.pos[i]
        d -= w.box * np.round(d / w.box)
        r = np.sqrt((d ** 2).sum(1))
        r[i] = np.inf
        rcp = rc[w.species[i], w.species]
        core = set(L["core"][q, :L["ncore"][q]].tolist())
        shell = set(L["shell"][q, :L["nshell"][q]].tolist())
        assert set(np.where(r < rcp - tol)[0]) <= core <= set(np.where(r < rcp + tol)[0])
        assert set(np.where((r > rcp + tol) & (r < 12.0 - tol))[0]) <= shell
        assert shell <= set(np.where((r > rcp - tol) & (r < 12.0 + tol))[0])


def test_whole_shell_independent_of_split(orc):
    w = W.rock_salt((5, 5, 5), seed=43, composition="LiCl-NaCl")
    A = make(orc, w)
    B = make(orc, w, r_core_pair=W.core_radii_from_sigma(w.bmh, 6.0))
    Fa, Fb = A.near(all_shell=True), B.near(all_shell=True)
    assert np.abs(Fa - Fb).max() < 1e-12 * np.abs(Fa).max()


def test_pair_split_unbiased(orc):
    w = W.rock_salt((4, 4, 4), seed=44, composition="LiCl-NaCl")
    S = make(orc, w, P_R=10, r_core_pair=W.core_radii_from_sigma(w.bmh, 6.0))
    sel = np.arange(0, w.n, 16)
    ref = S.near(sel, all_shell=True)
    X = []
    for step in range(300):
        S.step = step
        X.append(S.near(sel))
    X = np.array(X)
    z = (X.mean(0) - ref) / np.maximum(X.std(0, ddof=1) / np.sqrt(len(X)), 1e-300)
    assert np.abs(z).max() < 5.0, np.abs(z).max()
