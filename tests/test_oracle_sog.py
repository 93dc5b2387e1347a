"""Pins of the oracle's SOG split (Sec. 2.1) and of its k-space sampler
(Eq. (Pk)): C^1 conditions, positivity of the near part below r_c, accuracy
of 1/r = N + F against the exact kernel, the Fourier transform of Eq.
(Fouriertransform) against a numerical radial Fourier integral, S against a
brute-force lattice sum, and sampled k-vectors against P(k) by chi-square."""
import numpy as np
import pytest
from scipy import integrate, stats

B, M, RC = 1.3, 64, 12.0


@pytest.fixture(scope="module")
def sog(orc):
    return orc.sog_solve(B, M, RC)


def test_c1_conditions(orc, sog):
    s, w = sog
    F, dF = orc.sog_eval(B, M, s, w, np.array([RC]))
    assert abs(1.0 / RC - F[0]) < 1e-15                     # N(r_c) = 0
    assert abs(-1.0 / RC**2 - dF[0]) * RC**2 < 1e-12         # N'(r_c) = 0
    w0nom = np.sqrt(2.0) * np.log(B) / (np.sqrt(np.pi) * s)
    assert 0.9 < w[0] / w0nom < 1.1
    # nominal weights for m >= 1 (Eq. (far))
    m = np.arange(1, M + 1)
    np.testing.assert_allclose(w[1:], np.sqrt(2) * np.log(B) / (np.sqrt(np.pi) * B**m * s), rtol=1e-14)


def test_near_part_positive_below_rc(orc, sog):
    """r_c is the smallest root of r F(r) = 1: N(r) = 1/r - F(r) > 0 on (0, r_c)."""
    s, w = sog
    r = np.linspace(0.05, RC * (1 - 1e-3), 20000)
    F, _ = orc.sog_eval(B, M, s, w, r)
    assert np.all(1.0 / r - F > 0.0)
    # r_c is a double root (N = N' = 0): N ~ (r - r_c)^2 just below it
    r = np.linspace(RC * (1 - 1e-3), RC, 2000)
    F, _ = orc.sog_eval(B, M, s, w, r)
    assert np.all(1.0 / r - F > -1e-16)


def test_split_accuracy_past_cutoff(orc, sog):
    """Beyond r_c the far part alone must reproduce the Coulomb kernel: the
    relative potential and force errors stay at the 1e-6 level (BSA bound of
    Eq. (asymperror) at b = 1.3 is 1.9e-8; the w_0 change dominates)."""
    s, w = sog
    bound = 2 * np.sqrt(2) * np.exp(-np.pi**2 / (2 * np.log(B)))
    assert bound < 2e-8
    r = np.linspace(RC, 4 * RC, 5000)
    F, dF = orc.sog_eval(B, M, s, w, r)
    assert np.max(np.abs(1.0 - r * F)) < 1e-6
    assert np.max(np.abs(1.0 + r * r * dF)) < 3e-6


def test_bilateral_series_bound():
    """Eq. (asymperror) for the untruncated BSA of Eq. (1-r), checked with an
    independent evaluation of the bilateral series."""
    s = 2.0
    r = np.linspace(0.5, 40.0, 300)
    m = np.arange(-60, 400)[:, None]
    bsa = 2 * np.log(B) / np.sqrt(2 * np.pi * s**2) * np.sum(B ** (-m) * np.exp(-r**2 / (2 * B ** (2 * m) * s**2)), 0)
    err = np.abs(1 - r * bsa)
    assert err.max() <= 2 * np.sqrt(2) * np.exp(-np.pi**2 / (2 * np.log(B))) * 1.05


def _sys(orc, sog, box=(31.5, 31.5, 31.5), P_F=200):
    from paper_2512_24970_gb300 import workloads as W
    w = W.rock_salt((2, 2, 2), seed=1)
    s, wt = sog
    return orc.System(w.pos, w.species, w.charge, w.mass, w.bmh, np.array(box), s=s, w=wt, P_F=P_F)


def test_fourier_transform(orc, sog):
    """Fhat(k) = 4 pi int_0^inf F(r) r^2 sin(kr)/(kr) dr for the radial F."""
    s, w = sog
    S = _sys(orc, sog)
    # truncate the sum to Gaussians resolvable by the quadrature (b^m s < 400)
    mm = int(np.floor(np.log(400.0 / s) / np.log(B)))
    wt = w.copy()
    wt[mm + 1:] = 0.0
    S.w = wt
    for k in (0.05, 0.2, 0.5, 1.0, 2.0):
        def f(r):
            F, _ = orc.sog_eval(B, M, s, wt, np.array([r]))
            return 4 * np.pi * F[0] * r * np.sin(k * r) / k
        # integrate each Gaussian scale separately for accuracy
        edges = [0.0] + [min(40 * (B**m) * s, 3e4) for m in range(0, mm + 1, 4)] + [3e4]
        edges = sorted(set(edges))
        val = sum(integrate.quad(f, a, b, limit=400, epsabs=0, epsrel=1e-11)[0] for a, b in zip(edges[:-1], edges[1:]))
        ref = S.fhat(np.array([k * k]))[0]
        assert abs(val - ref) <= max(1e-7 * abs(ref), 1e-11), (k, val, ref)


@pytest.mark.parametrize("box", [(31.5, 31.5, 31.5), (25.2, 30.0, 50.4)])
def test_S_closed_form_vs_lattice_sum(orc, sog, box):
    """S of Eq. (Pk) from the separable mixture equals sum_{k != 0} k^2 Fhat(k)
    summed directly over the lattice with Eq. (Fouriertransform)."""
    S = _sys(orc, sog, box)
    mmax = [int(np.ceil(3.9 * b / (2 * np.pi))) for b in box]   # e^{-s^2 k^2/2} < 1e-26
    r = [np.arange(-m, m + 1) for m in mmax]
    mm = np.stack(np.meshgrid(*r, indexing="ij"), -1).reshape(-1, 3)
    mm = mm[np.any(mm != 0, 1)]
    k2 = ((2 * np.pi * mm / np.array(box)) ** 2).sum(1)
    direct = np.sum(k2 * S.fhat(k2))
    assert abs(S.sampler_S() - direct) <= 1e-13 * direct


def test_kbatch_distribution(orc, sog):
    """Sampled m follow P(k) = k^2 Fhat(k)/S (chi-square over the most likely
    modes plus one tail bin); c_p = S/(P_F |k_p|^2); m != 0 always."""
    S = _sys(orc, sog, (25.2, 25.2, 25.2), P_F=5000)
    ms = []
    for step in range(8):
        S.step = step
        m, c, Sv = S.kbatch()
        k2 = ((2 * np.pi * m / S.box) ** 2).sum(1)
        np.testing.assert_allclose(c, Sv / (S.P_F * k2), rtol=1e-14)
        assert np.all(np.any(m != 0, 1))
        ms.append(m)
    m = np.concatenate(ms)
    r = np.arange(-14, 15)
    lat = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    lat = lat[np.any(lat != 0, 1)]
    k2 = ((2 * np.pi * lat / S.box) ** 2).sum(1)
    p = k2 * S.fhat(k2) / S.sampler_S()
    assert abs(p.sum() - 1) < 1e-10
    order = np.argsort(-p)[:300]
    index = {tuple(x): i for i, x in enumerate(lat[order])}
    counts = np.zeros(len(order) + 1)
    for x in map(tuple, m):
        counts[index.get(x, len(order))] += 1
    exp = np.append(p[order], 1 - p[order].sum()) * m.shape[0]
    chi2, pval = stats.chisquare(counts, exp)
    assert pval > 1e-4, (chi2, pval)
