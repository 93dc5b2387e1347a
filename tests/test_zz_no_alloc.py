"""The allocation-free structure factor (rbsog_structure_factor_static, whose
scratch is a static device array) against the context's own structure factor
(a fixed k-batch through rbsog_compute_forces, read back with
rbsog_debug_get_parts) and against the oracle's, on two calls in a row with
different mode counts, and on calls from two contexts of different size (so a
different tile count) with nothing cleared in between, so that partials left
in the static scratch by one call would show in the next.  Collected last (file
name) so that it also runs after the rest of the GPU suite; it passes alone as
well."""
import ctypes

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


def modes(P, seed, mmax=9):
    g = np.random.default_rng(seed)
    m = g.integers(-mmax, mmax + 1, size=(P, 3)).astype(np.int32)
    m[np.all(m == 0, axis=1)] = (1, 0, 0)
    return m


def context_rho(ctx, m):
    """rho(k) of the same modes by the context's own path (FP64 k_rho)."""
    ctx.debug_set_kbatch(m, np.ones(m.shape[0]))
    ctx.compute_forces()
    return ctx.debug_parts(P=m.shape[0])["rho"]


def test_static_structure_factor_two_calls(rb):
    import torch
    w = W.rock_salt((10, 10, 10), seed=11, composition="LiCl-NaCl")     # N = 8000: 32 tiles
    prm = rb.MethodParams(P_F=64, seed=4, precision=rb.FP64)
    ctx = rb.Context(0)
    ctx.set_system(w.pos, w.species, w.charge, w.mass, w.bmh, w.box, prm)
    m1, m2 = modes(1000, 1), modes(300, 2)
    d1 = torch.from_numpy(m1).cuda()
    d2 = torch.from_numpy(m2).cuda()
    r1 = ctx.structure_factor_static(d1).cpu().numpy()                  # two calls in a row,
    r2 = ctx.structure_factor_static(d2).cpu().numpy()                  # the second smaller
    tol = 1e-12 * w.n
    np.testing.assert_allclose(r1, context_rho(ctx, m1), rtol=0, atol=tol)
    np.testing.assert_allclose(r2, context_rho(ctx, m2), rtol=0, atol=tol)
    # |rho| is O(sqrt(N)) for a random-phase sum: the comparison is not vacuous
    assert np.abs(r1).max() > 1.0
    # after the state moves, both paths follow it
    ctx.set_velocities(W.maxwell_boltzmann(w, 1200.0))
    ctx.step(3)
    r3 = ctx.structure_factor_static(d2).cpu().numpy()
    np.testing.assert_allclose(r3, context_rho(ctx, m2), rtol=0, atol=tol)
    assert np.abs(r3 - r2).max() > 1e-6


def test_static_structure_factor_tile_counts(rb, orc):
    """Two contexts of different N (32 and 4 tiles) called back to back, each
    against the oracle's rho(k) of the same positions."""
    import torch
    ws = [W.rock_salt((10, 10, 10), seed=12), W.rock_salt((5, 5, 5), seed=13, composition="LiCl")]
    ctxs = []
    for w in ws:
        c = rb.Context(0)
        c.set_system(w.pos, w.species, w.charge, w.mass, w.bmh, w.box, rb.MethodParams(P_F=64, precision=rb.FP64))
        ctxs.append(c)
    m = modes(700, 3)
    d = torch.from_numpy(m).cuda()
    for rep in range(2):
        for w, c in zip(ws, ctxs):
            got = c.structure_factor_static(d).cpu().numpy()
            S = orc.System(w.pos, w.species, w.charge, w.mass, w.bmh, w.box, P_F=64)
            np.testing.assert_allclose(got, S.rho(m), rtol=0, atol=1e-12 * w.n)


def test_static_structure_factor_rejects(rb):
    import torch
    w = W.rock_salt((5, 5, 5), seed=1)
    ctx = rb.Context(0)
    ctx.set_system(w.pos, w.species, w.charge, w.mass, w.bmh, w.box, rb.MethodParams(precision=rb.FP64))
    big = torch.zeros((rb.SF_STATIC_PMAX + 1, 3), dtype=torch.int32, device="cuda")
    with pytest.raises(rb.RbsogError) as e:
        ctx.structure_factor_static(big)
    assert e.value.code == -1
    m = np.ones((4, 3), dtype=np.int32)           # host memory: rejected before any launch
    rho = torch.empty((4, 2), dtype=torch.float64, device="cuda")
    rc = ctx._L.rbsog_structure_factor_static(ctx.h, 4, ctypes.c_void_p(m.ctypes.data),
                                              ctypes.c_void_p(rho.data_ptr()))
    assert rc == -1
    empty = torch.zeros((0, 3), dtype=torch.int32, device="cuda")
    assert ctx.structure_factor_static(empty).shape == (0, 2)
