"""Pins of the oracle's random streams: Philox4x32-10 against cuRAND's host
generator, Floyd's sampling without replacement against the uniform law on
subsets, and the Langevin noise against N(0, 1)."""
import ctypes
import ctypes.util
import itertools
import os

import numpy as np
import pytest
from scipy import stats


def _curand():
    for cand in ("/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")):
        if cand and os.path.exists(cand) or (cand and not cand.startswith("/")):
            try:
                return ctypes.CDLL(cand)
            except OSError:
                continue
    return None


CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161
CURAND_ORDERING_PSEUDO_LEGACY = 103


@pytest.mark.parametrize("seed", [0, 1, 0x0123456789ABCDEF, 2**64 - 1])
def test_philox_matches_curand_host(orc, seed):
    """cuRAND's host Philox4x32-10 generator (legacy ordering) emits block t as
    philox(counter=(0, 0, t, 0), key=(seed_lo, seed_hi)); the oracle's
    implementation of the published round function must reproduce it."""
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOrdering(gen, CURAND_ORDERING_PSEUDO_LEGACY) == 0
        nblk = 4096
        out = np.zeros(4 * nblk, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(out.size)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    ctr = np.zeros((nblk, 4), dtype=np.uint32)
    ctr[:, 2] = np.arange(nblk, dtype=np.uint32)
    mine = orc.philox(ctr, (seed & 0xFFFFFFFF, seed >> 32))
    np.testing.assert_array_equal(mine.reshape(-1), out)


def test_draw_counter_layout(orc):
    """draw() = philox((index, step_lo, step_hi, stream<<24|block), seed)."""
    seed, step = 0xDEADBEEF12345678, (7 << 32) + 5
    idx = np.arange(10, dtype=np.uint32)
    got = orc.draw(seed, step, idx, 2, 3)
    ctr = np.stack([idx, np.full(10, step & 0xFFFFFFFF), np.full(10, step >> 32),
                    np.full(10, (2 << 24) | 3)], 1).astype(np.uint32)
    np.testing.assert_array_equal(got, orc.philox(ctr, (seed & 0xFFFFFFFF, seed >> 32)))


def test_floyd_uniform_subsets(orc):
    """Floyd's algorithm picks every P_R-subset of the N_shell positions with
    equal probability (sampling without replacement, Sec. 2.2 proof)."""
    L = orc.lib()
    n, p = 9, 3
    subsets = {s: i for i, s in enumerate(itertools.combinations(range(n), p))}
    counts = np.zeros(len(subsets))
    t = np.zeros(p, dtype=np.int32)
    draws = 42000
    for k in range(draws):
        got = L.orc_floyd(11, k // 1000, k % 1000, n, p, t.ctypes.data)
        assert got == p
        assert len(set(t.tolist())) == p and t.min() >= 0 and t.max() < n
        assert np.all(np.diff(t) > 0)
        counts[subsets[tuple(t.tolist())]] += 1
    chi2, pval = stats.chisquare(counts)
    assert pval > 1e-4, (chi2, pval)


def test_floyd_takes_all_when_shell_small(orc):
    L = orc.lib()
    t = np.zeros(20, dtype=np.int32)
    assert L.orc_floyd(1, 0, 0, 7, 20, t.ctypes.data) == 7
    np.testing.assert_array_equal(t[:7], np.arange(7))
    assert L.orc_floyd(1, 0, 0, 20, 20, t.ctypes.data) == 20
    np.testing.assert_array_equal(t, np.arange(20))


def test_langevin_noise_is_standard_normal(orc):
    from paper_2512_24970_gb300 import workloads as W
    w = W.rock_salt((6, 6, 6), seed=3)
    S = orc.System(w.pos, w.species, w.charge, w.mass, w.bmh, w.box, seed=9)
    xi = np.concatenate([S.gaussian_noise(s).reshape(-1) for s in range(1, 6)])
    assert abs(xi.mean()) < 5.0 / np.sqrt(xi.size)
    assert abs(xi.var() - 1.0) < 0.02
    assert stats.kstest(xi, "norm").pvalue > 1e-4
