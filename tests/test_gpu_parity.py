"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Bars: lists, shell batches and k-batches bit-exact; FP64 forces and energies
within 1e-12 (RMS relative); mixed precision within 1e-5 RMS relative force
error (the tolerance of the metric), all on identical state and samples.
"""
import numpy as np
import pytest

from paper_2512_24970_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_TOL = 1e-5


@pytest.fixture(scope="module")
def rb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_24970_gb300 import rbsog
    rbsog.load()
    return rbsog


def rms_rel(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (b**2).sum()))


def setup_pair(rb, orc, w, *, P_R=20, P_F=200, precision=None, seed=3, step=0, r_core=6.0,
               integrator=None, T=1200.0):
    """GPU context and oracle system on the same workload and SOG parameters."""
    S = orc.System(w.pos, w.species, w.charge, w.mass, w.bmh, w.box, P_R=P_R, P_F=P_F, seed=seed,
                   step=step, r_core=r_core)
    prm = rb.MethodParams(s=S.s, w0=float(S.w[0]), P_R=P_R, P_F=P_F, seed=seed, r_core=r_core,
                          precision=rb.FP64 if precision is None else precision,
                          integrator=rb.LANGEVIN_BAOAB if integrator is None else integrator, T=T)
    ctx = rb.Context(0)
    ctx.set_system(w.pos, w.species, w.charge, w.mass, w.bmh, w.box, prm)
    if step:
        ctx.set_state(w.pos, np.zeros_like(w.pos), step)
    return ctx, S


CASES = {
    "nacl_1k": lambda: W.rock_salt((5, 5, 5), seed=1),                     # n_c = 5: fast stencil
    "small_box": lambda: W.rock_salt((4, 4, 4), seed=2),                   # n_c = 4: small-box path
    "ragged": lambda: W.rock_salt((6, 5, 7), seed=3, composition="LiCl-NaCl"),  # 3 species, orthorhombic
    "six_cells": lambda: W.rock_salt((6, 6, 6), seed=4, composition="LiCl"),      # whole rows of 6 cells
}


@pytest.mark.parametrize("case", list(CASES))
def test_lists_and_batches_bitexact(rb, orc, case):
    w = CASES[case]()
    ctx, S = setup_pair(rb, orc, w, step=5)
    sel = np.arange(w.n)
    g = ctx.debug_lists(sel, cap_core=128, cap_shell=512)
    o = S.lists(sel, cap_core=128, cap_shell=512)
    np.testing.assert_array_equal(g["ncore"], o["ncore"])
    np.testing.assert_array_equal(g["nshell"], o["nshell"])
    np.testing.assert_array_equal(g["core"], o["core"])
    np.testing.assert_array_equal(g["shell"], o["shell"])
    np.testing.assert_array_equal(g["nbatch"], o["nbatch"])
    np.testing.assert_array_equal(g["batch"], o["batch"])
    np.testing.assert_array_equal(g["weight"], o["weight"])


@pytest.mark.parametrize("step", [0, 7, 2**33 + 1])
def test_kbatch_bitexact(rb, orc, step):
    w = W.rock_salt((5, 5, 5), seed=1)
    ctx, S = setup_pair(rb, orc, w, P_F=1000, step=step)
    ctx.compute_forces()
    mg, cg = ctx.debug_kbatch()
    mo, co, So = S.kbatch()
    np.testing.assert_array_equal(mg, mo)
    np.testing.assert_allclose(cg, co, rtol=1e-13)
    s, wt, Sg = ctx.sog()
    assert abs(Sg - So) <= 1e-13 * So


@pytest.mark.parametrize("case", list(CASES))
def test_fp64_forces_and_energy(rb, orc, case):
    w = CASES[case]()
    ctx, S = setup_pair(rb, orc, w, P_F=300, step=2)
    Fg, Eg = ctx.compute_forces(energy=True)
    o = S.forces(energy=True)
    assert rms_rel(Fg, o["F"]) < FP64_TOL
    parts = ctx.debug_parts()
    assert rms_rel(parts["near"], o["near"]) < FP64_TOL
    assert rms_rel(parts["far"], o["far"]) < FP64_TOL
    np.testing.assert_allclose(parts["Fcorr"], o["Fcorr"], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(Eg, o["energy"], rtol=FP64_TOL)


@pytest.mark.parametrize("case", list(CASES))
def test_fp64_force_only_fcorr(rb, orc, case):
    """Force-only evaluations (every MD step) take F^corr from the near
    field's 64-bit integer totals in units of 2^-40, energy evaluations from
    k_corr's FP64 sum of the warp partials: both against the oracle, and
    against each other to the fixed point's rounding (at most one 2^-41 per
    warp partial, divided by N)."""
    w = CASES[case]()
    ctx, S = setup_pair(rb, orc, w, P_F=300, step=2)
    F = ctx.compute_forces()
    fc = ctx.debug_parts()["Fcorr"]
    Fe, _ = ctx.compute_forces(energy=True)
    fce = ctx.debug_parts()["Fcorr"]
    o = S.forces()
    assert rms_rel(F, o["F"]) < FP64_TOL
    np.testing.assert_allclose(fc, o["Fcorr"], rtol=1e-9, atol=1e-12)
    # at most N/4 warp partials (runs of 8 padded slots), one rounding of 2^-41 each
    assert np.abs(fc - fce).max() < (w.n / 4) * 2.0 ** -41 / w.n + 1e-14
    assert rms_rel(F, Fe) < 1e-13


@pytest.mark.parametrize("case", list(CASES))
def test_mixed_forces(rb, orc, case):
    w = CASES[case]()
    ctx, S = setup_pair(rb, orc, w, P_F=300, precision=rb.MIXED, step=4)
    Fg, Eg = ctx.compute_forces(energy=True)
    o = S.forces(energy=True)
    eps = rms_rel(Fg, o["F"])
    assert eps < MIXED_TOL, eps
    np.testing.assert_allclose(Eg[3], o["energy"][3], rtol=1e-5)


def test_deterministic_limits(rb, orc):
    """Whole shell + all k with weight Fhat: the deterministic SOG force of
    Eq. (Fshort) + Eq. (Long), FP64 and mixed."""
    w = W.rock_salt((4, 4, 4), seed=7)
    for prec, tol in ((rb.FP64, FP64_TOL), (rb.MIXED, MIXED_TOL)):
        ctx, S = setup_pair(rb, orc, w, precision=prec)
        m, c = S.enumerated_modes(12)
        ctx.debug_whole_shell(True)
        ctx.debug_set_kbatch(m, c)
        Fg, Eg = ctx.compute_forces(energy=True)
        o = S.forces(kmodes=(m, c), all_shell=True, energy=True)
        assert rms_rel(Fg, o["F"]) < tol
        np.testing.assert_allclose(Eg[3], o["energy"][3], rtol=max(tol, 1e-12))


@pytest.mark.parametrize("integ", ["nve", "langevin"])
def test_fp64_trajectory(rb, orc, integ):
    w = W.rock_salt((5, 5, 5), seed=1)
    v0 = W.maxwell_boltzmann(w, 1200.0)
    ig = rb.NVE_VV if integ == "nve" else rb.LANGEVIN_BAOAB
    ctx, S = setup_pair(rb, orc, w, P_F=100, integrator=ig)
    ctx.set_velocities(v0)
    ctx.step(10)
    pos, vel, step = ctx.get_state()
    vo, _ = S.run(v0, 10, 0.001, integrator=0 if integ == "nve" else 1, T=1200.0, gamma=1.0)
    assert step == 10 and S.step == 10
    assert np.sqrt(((pos - S.pos) ** 2).mean()) < 1e-10
    assert rms_rel(vel, vo) < 1e-10


def test_c1_nve_100_steps(rb, orc):
    """Molten NaCl N = 1000 (5^3 cells, seed 1), P_R = 20, P_F = 200, FP64: one
    force evaluation (forces and energies within 1e-12), then 100 velocity
    Verlet steps at dt = 1 fs from Maxwell-Boltzmann velocities at 1200 K,
    following the oracle's run with the same samples at every step."""
    w = W.rock_salt((5, 5, 5), seed=1)
    v0 = W.maxwell_boltzmann(w, 1200.0)
    ctx, S = setup_pair(rb, orc, w, P_F=200, integrator=rb.NVE_VV)
    Fg, Eg = ctx.compute_forces(energy=True)
    o = S.forces(energy=True)
    assert rms_rel(Fg, o["F"]) < FP64_TOL
    np.testing.assert_allclose(Eg, o["energy"], rtol=1e-12, atol=1e-9)
    ctx.set_velocities(v0)
    ctx.step(100)
    pos, vel, step = ctx.get_state()
    vo, _ = S.run(v0, 100, 0.001, integrator=0)
    assert step == 100 and S.step == 100
    dpos = float(np.sqrt(((pos - S.pos) ** 2).mean()))
    assert dpos < 1e-9, dpos
    assert rms_rel(vel, vo) < 1e-8, rms_rel(vel, vo)
    assert float(np.sqrt(((pos - w.pos) ** 2).mean())) > 0.05       # the atoms did move


def test_resume_bit_identical(rb, orc):
    w = W.rock_salt((5, 5, 5), seed=1)
    v0 = W.maxwell_boltzmann(w, 1200.0)
    runs = []
    for split in (False, True):
        ctx, _ = setup_pair(rb, orc, w, precision=rb.MIXED)
        ctx.set_velocities(v0)
        if split:
            ctx.step(6)
            p, v, s = ctx.get_state()
            ctx2, _ = setup_pair(rb, orc, w, precision=rb.MIXED)
            ctx2.set_state(p, v, s)
            ctx2.step(6)
            runs.append(ctx2.get_state())
        else:
            ctx.step(12)
            runs.append(ctx.get_state())
    np.testing.assert_array_equal(runs[0][0], runs[1][0])
    np.testing.assert_array_equal(runs[0][1], runs[1][1])
    assert runs[0][2] == runs[1][2] == 12


@pytest.mark.parametrize("key", ["nacl_64k", "liclnacl_216k", "nacl_1m"])
def test_full_size_sampled(rb, orc, key):
    """The full-size workloads (molten NaCl N = 64,000, the benchmark; the
    LiCl-NaCl mixture N = 216,000; NaCl N = 1,024,000): lists and batches of
    sampled atoms bit-exact, k-batch bit-exact, mixed forces of the sample
    within 1e-5 RMS of the oracle's FP64 near + far field."""
    w, cfg = W.make(key)
    ctx, S = setup_pair(rb, orc, w, P_R=cfg.P_R, P_F=cfg.P_F, precision=rb.MIXED, seed=cfg.seed, step=3)
    Fg = ctx.compute_forces()
    parts = ctx.debug_parts()
    sel = np.linspace(0, w.n - 1, 96).astype(np.int64)
    g = ctx.debug_lists(sel, cap_core=128, cap_shell=512)
    o = S.lists(sel, cap_core=128, cap_shell=512)
    for k in ("ncore", "nshell", "core", "shell", "nbatch", "batch", "weight"):
        np.testing.assert_array_equal(g[k], o[k])
    m, c, _ = S.kbatch()
    mg, cg = ctx.debug_kbatch()
    np.testing.assert_array_equal(mg, m)
    near = S.near(sel)
    far, _ = S.far(m, c, sel=sel)
    ref = near + far                                  # uncorrected total
    got = Fg[sel] + parts["Fcorr"]
    assert rms_rel(got, ref) < MIXED_TOL
    # F^corr is the mean near field: the corrected near field sums to zero
    assert np.abs((parts["near"] - parts["Fcorr"]).sum(0)).max() < 1e-6 * w.n
    assert np.abs(parts["far"].sum(0)).max() < 1e-5 * np.sqrt(w.n)


def test_error_codes(rb, orc):
    w = W.rock_salt((5, 5, 5), seed=1)
    ctx = rb.Context(0)
    prm = rb.MethodParams()
    q = w.charge.copy()
    q[0] = 2.0
    with pytest.raises(rb.RbsogError) as e:
        ctx.set_system(w.pos, w.species, q, w.mass, w.bmh, w.box, prm)
    assert e.value.code == -2
    with pytest.raises(rb.RbsogError) as e:
        ctx.set_system(w.pos, w.species, w.charge, w.mass, w.bmh, w.box * 0.7, prm)
    assert e.value.code == -3
    with pytest.raises(rb.RbsogError) as e:
        ctx.set_system(w.pos, w.species, w.charge, w.mass, w.bmh, w.box, rb.MethodParams(P_R=0))
    assert e.value.code == -1
    with pytest.raises(rb.RbsogError) as e:
        ctx.compute_forces()
    assert e.value.code == -8
    # the library's own SOG solve agrees with the oracle's: the root of
    # N'(r_c; s) = 0 is determined only to the rounding noise of N' divided by
    # its slope (~1e-11 relative), so two independent bisections agree to that
    ctx.set_system(w.pos, w.species, w.charge, w.mass, w.bmh, w.box, prm)
    s, wt, Sg = ctx.sog()
    so, wo = orc.sog_solve(prm.b, prm.M, prm.r_shell)
    assert abs(s - so) < 1e-10 * so
    np.testing.assert_allclose(wt, wo, rtol=1e-9)


def test_device_phase_factors(rb):
    """The FP32 phase factors of the mixed far field.  The half turn is taken
    off exactly and the remainder phi in [-pi/2, pi/2) carries at most
    2^6 / 2^32 of a turn (9.4e-8 rad) from its rounding to 24 bits, 4.4e-8 from
    the binary32 value of 2 pi / 2^32 and 6e-8 from the product's rounding; the
    minimax polynomials add 5e-9 and the result's rounding 6e-8, so the error
    stays below 2.5e-7.  Over the whole circle it has no bias: an error smooth
    in the angle would add up coherently in rho(k) over atoms sharing a phase."""
    ctx = rb.Context(0)
    th = (np.arange(1 << 20, dtype=np.uint64) << np.uint64(12)).astype(np.uint32)
    th = np.concatenate([th, np.random.default_rng(0).integers(0, 2**32, 1 << 20, dtype=np.uint64).astype(np.uint32)])
    s, c = ctx.debug_sincos(th)
    ang = 2 * np.pi * th.astype(np.float64) / 2**32
    es, ec = s - np.sin(ang), c - np.cos(ang)
    assert np.abs(es).max() < 2.5e-7 and np.abs(ec).max() < 2.5e-7
    assert abs(es.mean()) < 1e-9 and abs(ec.mean()) < 1e-9


def virial_err(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("case", list(CASES))
def test_fp64_virial(rb, orc, case):
    """Virial W_N + W_F* (xx, yy, zz, xy, xz, yz) of the same samples as the
    oracle's: FP64 within 1e-11 of its largest component."""
    w = CASES[case]()
    ctx, S = setup_pair(rb, orc, w, P_F=300, step=2)
    Fg, Eg, Wg = ctx.compute_forces(energy=True, virial=True)
    o = S.forces(energy=True)
    assert virial_err(Wg, o["virial"]) < 1e-11, (Wg, o["virial"])
    assert rms_rel(Fg, o["F"]) < FP64_TOL


def test_virial_mixed_and_deterministic(rb, orc):
    """Mixed precision within 1e-5; the deterministic limit (whole shell, all k
    weighted Fhat) in both precisions."""
    w = W.rock_salt((6, 5, 7), seed=3, composition="LiCl-NaCl")
    ctx, S = setup_pair(rb, orc, w, P_F=300, precision=rb.MIXED, step=4)
    _, Wg = ctx.compute_forces(virial=True)
    assert virial_err(Wg, S.forces(energy=True)["virial"]) < MIXED_TOL
    m, c = S.enumerated_modes(10)
    ref = S.forces(kmodes=(m, c), all_shell=True, energy=True)["virial"]
    for prec, tol in ((rb.FP64, 1e-11), (rb.MIXED, MIXED_TOL)):
        ctx, _ = setup_pair(rb, orc, w, precision=prec, step=4)
        ctx.debug_whole_shell(True)
        ctx.debug_set_kbatch(m, c)
        _, Wd = ctx.compute_forces(virial=True)
        assert virial_err(Wd, ref) < tol, (prec, Wd, ref)


def setup_nh(rb, orc, w, precision, tdamp=0.05, chain=3, T=1500.0):
    S = orc.System(w.pos, w.species, w.charge, w.mass, w.bmh, w.box, P_R=20, P_F=100, seed=3)
    prm = rb.MethodParams(s=S.s, w0=float(S.w[0]), P_R=20, P_F=100, seed=3, precision=precision,
                          integrator=rb.NOSE_HOOVER, T=T, tdamp=tdamp, nh_chain=chain)
    ctx = rb.Context(0)
    ctx.set_system(w.pos, w.species, w.charge, w.mass, w.bmh, w.box, prm)
    return ctx, S


def test_nose_hoover_fp64_trajectory(rb, orc):
    """Nose-Hoover chain (length 3, tdamp 0.05 ps, target 1500 K from 1200 K):
    10 FP64 steps follow the oracle, chain state included."""
    w = W.rock_salt((5, 5, 5), seed=1)
    v0 = W.maxwell_boltzmann(w, 1200.0)
    ctx, S = setup_nh(rb, orc, w, rb.FP64)
    ctx.set_velocities(v0)
    ctx.step(10)
    pos, vel, step = ctx.get_state()
    eta, ve = ctx.thermostat()
    vo, _ = S.run(v0, 10, 0.001, integrator=orc.INTEGRATOR_NOSE_HOOVER, T=1500.0, tdamp=0.05, nh_chain=3)
    assert step == 10
    assert np.sqrt(((pos - S.pos) ** 2).mean()) < 1e-10
    assert rms_rel(vel, vo) < 1e-10
    np.testing.assert_allclose(eta, S.chain.eta, rtol=1e-9, atol=1e-13)
    np.testing.assert_allclose(ve, S.chain.v, rtol=1e-9, atol=1e-11)
    assert np.abs(ve).max() > 1e-3                 # the chain moved


def test_nose_hoover_resume_bit_identical(rb, orc):
    w = W.rock_salt((5, 5, 5), seed=2)
    v0 = W.maxwell_boltzmann(w, 1200.0)
    ctx, _ = setup_nh(rb, orc, w, rb.MIXED)
    ctx.set_velocities(v0)
    ctx.step(12)
    ref = ctx.get_state()
    ctx1, _ = setup_nh(rb, orc, w, rb.MIXED)
    ctx1.set_velocities(v0)
    ctx1.step(6)
    p, v, s = ctx1.get_state()
    eta, ve = ctx1.thermostat()
    ctx2, _ = setup_nh(rb, orc, w, rb.MIXED)
    ctx2.set_state(p, v, s)
    ctx2.set_thermostat(eta, ve)
    ctx2.step(6)
    got = ctx2.get_state()
    np.testing.assert_array_equal(got[0], ref[0])
    np.testing.assert_array_equal(got[1], ref[1])
    assert got[2] == ref[2] == 12
