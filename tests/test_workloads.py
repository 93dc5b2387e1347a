"""The seeded input generators against the recipe they state: sizes, density,
neutrality, composition, jitter, velocities and the replica mix of the
ensemble; the same seed gives the same input (CPU, no GPU)."""
import numpy as np
import pytest

from paper_2512_24970_gb300 import workloads as W


def test_rock_salt_shape_density_neutrality():
    w = W.rock_salt((5, 6, 7), seed=3)
    assert w.n == 8 * 5 * 6 * 7
    np.testing.assert_allclose(w.box, [5 * 6.3, 6 * 6.3, 7 * 6.3])
    assert w.n / np.prod(w.box) == pytest.approx(8 / 6.3 ** 3)          # 0.0320 ions / A^3
    assert w.n / np.prod(w.box) == pytest.approx(0.0320, abs=5e-5)
    q = w.charge[w.species]
    assert q.sum() == 0.0 and set(np.unique(q)) == {-1.0, 1.0}
    # every ion within a few jitter widths of its lattice site: the unjittered lattice
    # is the same generator with jitter 0
    w0 = W.rock_salt((5, 6, 7), seed=3, jitter=0.0)
    d = w.pos - w0.pos
    assert abs(d.std() - 0.25) < 0.01 and abs(d.mean()) < 0.01
    assert np.abs(d).max() < 8 * 0.25
    # nearest cation-anion distance of the perfect lattice: a / 2
    cat, an = w0.pos[w0.species == 0], w0.pos[w0.species == 1]
    dd = np.linalg.norm(cat[:50, None, :] - an[None, :, :], axis=-1).min()
    assert dd == pytest.approx(3.15)


def test_same_seed_same_input():
    a, b, c = W.rock_salt((4, 4, 4), seed=7), W.rock_salt((4, 4, 4), seed=7), W.rock_salt((4, 4, 4), seed=8)
    np.testing.assert_array_equal(a.pos, b.pos)
    assert not np.array_equal(a.pos, c.pos)
    np.testing.assert_array_equal(W.maxwell_boltzmann(a, 1200.0), W.maxwell_boltzmann(b, 1200.0))


def test_mixture_composition():
    w = W.rock_salt((6, 6, 6), seed=2, composition="LiCl-NaCl")
    assert w.names == ["Li", "Na", "Cl"]
    ncat = w.n // 2
    assert np.sum(w.species == 0) == round(0.59 * ncat)
    assert np.sum(w.species == 1) == ncat - round(0.59 * ncat)
    assert np.sum(w.species == 2) == ncat
    # the cations are shuffled over the sites: both kinds in each half of the lattice
    first = w.species[: ncat // 2]
    assert 0 < np.sum(first == 0) < ncat // 2
    w2 = W.rock_salt((4, 4, 4), seed=2, composition="LiCl")
    assert set(np.unique(w2.species)) == {0, 2}
    with pytest.raises(ValueError):
        W.rock_salt((2, 2, 2), composition="KCl")


def test_bmh_tables_symmetric():
    for names, bmh in (W.nacl_params(), W.licl_nacl_params()):
        t = np.asarray(bmh)
        assert t.shape == (len(names), len(names), 5)
        np.testing.assert_array_equal(t, t.transpose(1, 0, 2))
        assert np.all(t[..., 0] > 0) and np.all(t[..., 1] > 0) and np.all(t[..., 4] > 0)


def test_maxwell_boltzmann_temperature_and_momentum():
    w = W.rock_salt((8, 8, 8), seed=1)
    T = 1200.0
    v = W.maxwell_boltzmann(w, T)
    m = w.mass[w.species]
    np.testing.assert_allclose((m[:, None] * v).sum(0), 0.0, atol=1e-9)
    ekin = 0.5 * (m[:, None] * v * v).sum() / W.FCONV                    # eV
    T_meas = 2.0 * ekin / (3 * w.n * W.KB)
    assert abs(T_meas / T - 1.0) < 4.0 * np.sqrt(2.0 / (3 * w.n))        # equipartition, within 4 sigma


def test_configs():
    sizes = {"nacl_1k": 1000, "nacl_64k": 64000, "liclnacl_216k": 216000, "nacl_1m": 1024000}
    for key, n in sizes.items():
        c = W.CONFIGS[key]
        assert 8 * int(np.prod(c.cells)) == n
    w, c = W.make("nacl_1k")
    assert w.n == 1000 and c.integrator == "nve" and c.P_F == 200 and w.vel.shape == (1000, 3)
    w, c = W.make("nacl_1k", P_F=50)
    assert c.P_F == 50


def test_ensemble_recipe():
    reps = W.ensemble(n_rep=64, seed=5)
    assert len(reps) == 64
    ns = np.array([w.n for w, _ in reps])
    assert ns.min() >= 512 and ns.max() <= 32768
    for w, T in reps:
        k = round((w.n / 8) ** (1 / 3))
        assert 8 * k ** 3 == w.n and 4 <= k <= 16
        assert 1100.0 <= T <= 1300.0
        assert w.charge[w.species].sum() == 0.0
    comps = {w.name.split()[0] for w, _ in reps}
    assert comps == {"NaCl", "LiCl", "LiCl-NaCl"}
    assert len(set(ns)) > 8                                             # uneven sizes
    np.testing.assert_array_equal(reps[3][0].pos, W.ensemble(n_rep=64, seed=5)[3][0].pos)


def test_core_radii_rule():
    names, bmh = W.licl_nacl_params()
    rc = W.core_radii_from_sigma(bmh, 6.0)
    np.testing.assert_array_equal(rc, rc.T)
    assert rc.max() == 6.0 and np.all(rc > 0) and np.all(rc <= 6.0)
    i = names.index("Cl")
    assert rc[i, i] == 6.0                                               # the largest sigma
