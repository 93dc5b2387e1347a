"""Pins of the oracle's virial W = W_N + W_F* (xx, yy, zz, xy, xz, yz).

W is minus the derivative of the energy under a homogeneous strain of
positions and box (the pair part is the familiar sum of r_ij (x) f_ij).
What fixes it independently of its own code:
  - a central difference of the deterministic energy (whole shell, every k
    with |m_d| <= m_max weighted Fhat) under a stretch of one axis gives the
    diagonal, near and far parts together (Coulomb only: the SOG residual is
    C^1 at r_shell, so pairs crossing the cutoff under the strain add nothing);
  - two atoms: W = d (x) F_1 with the pinned pair force (off-diagonals, the 1/2);
  - permuting the axes permutes W (the far part's k_a k_b indices);
  - the sampled estimator (shell batch, k-batch) is unbiased for it.
"""
import numpy as np

from paper_2512_24970_gb300 import workloads as W

COMP = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))


def make(orc, w, bmh=None, charge=None, **kw):
    return orc.System(w.pos, w.species, w.charge if charge is None else charge, w.mass,
                      w.bmh if bmh is None else bmh, w.box, **kw)


def coulomb_only(w):
    b = w.bmh.copy()
    b[..., 0] = 0.0
    b[..., 3] = 0.0
    b[..., 4] = 0.0
    return b


def det_energy(S, m_max):
    out = S.forces(energy=True, kmodes=S.enumerated_modes(m_max), all_shell=True)
    return out["energy"][3], out


def test_virial_is_strain_derivative_of_energy(orc):
    w = W.rock_salt((5, 5, 5), seed=21)
    S = make(orc, w, bmh=coulomb_only(w))
    U0, out = det_energy(S, 10)
    Wv = out["virial"]
    h = 1e-4
    scale = np.abs(Wv[:3]).max()
    for a in range(3):
        Us = []
        for sgn in (+1, -1):
            T = make(orc, w, bmh=coulomb_only(w))
            f = 1.0 + sgn * h
            T.pos = w.pos.copy()
            T.pos[:, a] *= f
            T.box = w.box.copy()
            T.box[a] *= f
            Us.append(det_energy(T, 10)[0])
        dUde = (Us[0] - Us[1]) / (2 * h)
        assert abs(-dUde - Wv[a]) < 2e-6 * scale, (a, -dUde, Wv[a])


def test_two_atom_pair_virial(orc):
    """BMH only, two neutral atoms in a large box: W = d (x) F_1 = d (x) f_12."""
    w = W.rock_salt((5, 5, 5), seed=1)
    pos = np.array([[10.0, 11.0, 12.0], [12.1, 13.3, 9.8]])
    sp = np.array([0, 1], dtype=np.int32)
    S = orc.System(pos, sp, np.zeros(2), w.mass, w.bmh, w.box, P_R=20)
    F, E, Wn = S.near(energy=True, virial=True)
    d = pos[0] - pos[1]
    ref = np.array([d[a] * F[0, b] for a, b in COMP])
    np.testing.assert_allclose(Wn.sum(0), ref, rtol=1e-9, atol=1e-12)
    assert abs(ref[3]) > 1e-3 and abs(ref[5]) > 1e-3      # off-diagonals are exercised


def test_virial_permutes_with_axes(orc):
    w = W.rock_salt((5, 5, 5), seed=22)
    S = make(orc, w, P_F=300, P_R=20, seed=4)
    Wv = S.forces(energy=True)["virial"]
    perm = [1, 2, 0]                        # new axis a is old axis perm[a]
    T = make(orc, w, P_F=300, P_R=20, seed=4)
    T.pos = w.pos[:, perm].copy()
    T.box = w.box[perm].copy()
    # the k-batch is drawn in box units, the same for a cubic box; the shell
    # batch order follows the cells, which the permutation relabels, so compare
    # the deterministic forms instead
    m, c = S.enumerated_modes(8)
    A = S.forces(energy=True, kmodes=(m, c), all_shell=True)["virial"]
    B = T.forces(energy=True, kmodes=(m, c), all_shell=True)["virial"]
    full = lambda v: np.array([[v[0], v[3], v[4]], [v[3], v[1], v[5]], [v[4], v[5], v[2]]])
    np.testing.assert_allclose(full(B), full(A)[np.ix_(perm, perm)], rtol=1e-10, atol=1e-9)
    assert np.isfinite(Wv).all()


def test_sampled_virial_unbiased(orc):
    w = W.rock_salt((4, 4, 4), seed=23)
    S = make(orc, w, P_R=10, P_F=100, seed=5)
    m, c = S.enumerated_modes(12)
    ref = S.forces(energy=True, kmodes=(m, c), all_shell=True)["virial"]
    X = []
    for step in range(300):
        S.step = step
        X.append(S.forces(energy=True)["virial"])
    X = np.array(X)
    z = (X.mean(0) - ref) / (X.std(0, ddof=1) / np.sqrt(len(X)))
    assert np.abs(z).max() < 5.0, z


def test_kinetic_tensor(orc):
    """K = sum_i m_i v_i (x) v_i: its trace is twice the kinetic energy
    (kinetic2, which the Nose-Hoover conserved quantity pins), permuting the
    axes of the velocities permutes K, and for Maxwell-Boltzmann velocities
    K / N tends to kT times the identity (equipartition, per component)."""
    w = W.rock_salt((5, 5, 5), seed=2, composition="LiCl")
    S = make(orc, w)
    v = W.maxwell_boltzmann(w, 1300.0, seed=3)
    K = S.kinetic_tensor(v)
    assert abs(K[:3].sum() - S.kinetic2(v)) < 1e-12 * S.kinetic2(v)
    perm = [2, 0, 1]
    Kp = S.kinetic_tensor(v[:, perm])
    full = lambda k: np.array([[k[0], k[3], k[4]], [k[3], k[1], k[5]], [k[4], k[5], k[2]]])
    np.testing.assert_allclose(full(Kp), full(K)[np.ix_(perm, perm)], rtol=1e-13)
    kT = orc.KB * 1300.0
    n = w.n
    assert np.all(np.abs(K[:3] / (n * kT) - 1.0) < 5.0 * np.sqrt(2.0 / n))        # chi-square, n dof
    assert np.all(np.abs(K[3:]) / (n * kT) < 5.0 / np.sqrt(n))                     # mean-zero products
