"""GPU parity of the kept (Verlet-skin) random batch lists against the oracle.

Bars as for the per-step lists: kept lists A / B and the shell batches drawn
from them bit-exact; FP64 forces and trajectories within 1e-12 / 1e-10; mixed
precision within 1e-5 RMS relative force error.
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


def setup_kept(rb, orc, w, *, skin=1.0, list_every=5, P_R=20, P_F=200, precision=None, seed=3, step=0,
               integrator=None):
    S = orc.System(w.pos, w.species, w.charge, w.mass, w.bmh, w.box, P_R=P_R, P_F=P_F, seed=seed, step=step,
                   skin=skin, list_every=list_every)
    prm = rb.MethodParams(s=S.s, w0=float(S.w[0]), P_R=P_R, P_F=P_F, seed=seed,
                          precision=rb.FP64 if precision is None else precision,
                          integrator=rb.LANGEVIN_BAOAB if integrator is None else integrator,
                          list_every=list_every, skin=skin)
    ctx = rb.Context(0)
    ctx.set_system(w.pos, w.species, w.charge, w.mass, w.bmh, w.box, prm)
    if step:
        ctx.set_state(w.pos, np.zeros_like(w.pos), step)
    return ctx, S


CASES = {
    "nacl_1k": lambda: W.rock_salt((5, 5, 5), seed=1),                          # 4 cells per axis: small box
    "ragged": lambda: W.rock_salt((6, 5, 7), seed=3, composition="LiCl-NaCl"),  # 3 species, orthorhombic
    "six_cells": lambda: W.rock_salt((6, 6, 6), seed=4, composition="LiCl"),    # 5 cells: whole rows
    "nacl_5832": lambda: W.rock_salt((9, 9, 9), seed=5),                        # 8 cells: culled rows
}


@pytest.mark.parametrize("case", list(CASES))
def test_kept_lists_and_batches_bitexact(rb, orc, case):
    w = CASES[case]()
    ctx, S = setup_kept(rb, orc, w, step=5)
    ctx.compute_forces()
    sel = np.arange(w.n)
    g = ctx.debug_kept_lists(sel, cap_a=64, cap_b=512)
    o = S.lists_skin(sel, cap_a=64, cap_b=512)
    for k in ("nA", "nB", "A", "B", "nbatch", "batch", "weight"):
        np.testing.assert_array_equal(g[k], o[k], err_msg=k)
    check_batch_used(ctx, sel, o, 20)


def check_batch_used(ctx, sel, o, P_R):
    """The batch the pair sums read (drawn by the batch kernel, from the 16-bit
    or the 32-bit rows of B, kept in draw order) holds the oracle's batch (in
    list order); -1 where all of B is taken."""
    used = ctx.debug_kept_batch_used(sel)
    drawn = o["nB"] > P_R
    np.testing.assert_array_equal(np.sort(used[drawn], axis=1), np.sort(o["batch"][drawn], axis=1))
    assert (used[~drawn] == -1).all()


def test_kept_b16_and_wide_rows_agree(rb, orc):
    """B read as 16-bit slot offsets (every offset of the build fits) or as
    the 32-bit rows: the same batches and forces bit for bit, in both
    precisions, through builds."""
    w = W.rock_salt((9, 8, 7), seed=23, composition="LiCl-NaCl")
    for prec in (rb.MIXED, rb.FP64):
        out = []
        for wide in (False, True):
            ctx, S = setup_kept(rb, orc, w, list_every=-1, skin=1.0, precision=prec)
            assert ctx.debug_kept_b16(force_wide=wide)
            ctx.set_velocities(W.maxwell_boltzmann(w, 1200.0))
            ctx.step(6)
            F = ctx.compute_forces()
            sel = np.arange(0, w.n, 7)
            out.append((F, ctx.get_state()[0], ctx.debug_kept_batch_used(sel)))
            assert ctx.debug_kept_b16(force_wide=wide)      # this small box: every offset fits
        for a, b in zip(out[0], out[1]):
            np.testing.assert_array_equal(a, b)


def test_kept_skin_zero_is_per_step_path(rb, orc):
    """list_every = 1, skin = 0: every evaluation builds, and the kept path
    gives the per-step path's forces (summation order aside)."""
    w = W.rock_salt((6, 5, 7), seed=3, composition="LiCl-NaCl")
    ctx, S = setup_kept(rb, orc, w, skin=0.0, list_every=1, step=2)
    Fk, Ek = ctx.compute_forces(energy=True)
    prm = ctx.params
    ref = rb.Context(0)
    ref.set_system(w.pos, w.species, w.charge, w.mass, w.bmh, w.box,
                   rb.MethodParams(**{**prm.__dict__, "list_every": 0, "skin": 0.0}))
    ref.set_state(w.pos, np.zeros_like(w.pos), 2)
    Fr, Er = ref.compute_forces(energy=True)
    assert rms_rel(Fk, Fr) < 1e-14
    np.testing.assert_allclose(Ek, Er, rtol=1e-13)


@pytest.mark.parametrize("integ", ["nve", "langevin"])
def test_kept_fp64_trajectory(rb, orc, integ):
    """10 steps with builds at steps 0, 4, 8 and the kept lists in between:
    GPU FP64 against the oracle's kept-list run."""
    w = W.rock_salt((6, 6, 6), seed=4, composition="LiCl")
    v0 = W.maxwell_boltzmann(w, 1200.0)
    ig = rb.NVE_VV if integ == "nve" else rb.LANGEVIN_BAOAB
    ctx, S = setup_kept(rb, orc, w, list_every=4, P_F=100, integrator=ig)
    ctx.set_velocities(v0)
    ctx.step(10)
    pos, vel, step = ctx.get_state()
    vo, Fo = S.run(v0, 10, 0.001, integrator=0 if integ == "nve" else 1, T=1200.0, gamma=1.0)
    assert step == 10 and S.step == 10
    assert np.sqrt(((pos - S.pos) ** 2).mean()) < 1e-10
    assert rms_rel(vel, vo) < 1e-10
    g = ctx.debug_kept_lists(np.arange(w.n))
    o = S.lists_skin(np.arange(w.n), cap_a=64, cap_b=512)
    for k in ("nA", "nB", "A", "B", "batch"):
        np.testing.assert_array_equal(g[k], o[k], err_msg=k)


def test_kept_mixed_forces_between_builds(rb, orc):
    """Mixed precision, evaluated from the kept lists three steps after the
    build, against the oracle at the GPU's own positions."""
    w = W.rock_salt((9, 9, 9), seed=5)
    v0 = W.maxwell_boltzmann(w, 1200.0)
    ctx, S = setup_kept(rb, orc, w, list_every=10, P_F=300, precision=rb.MIXED)
    ctx.set_velocities(v0)
    ctx.step(3)
    pos, vel, step = ctx.get_state()
    Fg, Eg = ctx.compute_forces(energy=True)
    S.build_pos = w.pos.copy()
    S.pos = pos
    S.step = step
    o = S.forces(energy=True)
    assert rms_rel(Fg, o["F"]) < MIXED_TOL
    np.testing.assert_allclose(Eg[3], o["energy"][3], rtol=1e-5)


def test_kept_skin_exceeded_is_reported(rb, orc):
    """A skin far too thin for the motion: the step reports RBSOG_E_SKIN."""
    w = W.rock_salt((5, 5, 5), seed=1)
    v0 = W.maxwell_boltzmann(w, 1200.0)
    ctx, _ = setup_kept(rb, orc, w, skin=1e-4, list_every=100, precision=rb.MIXED)
    ctx.set_velocities(v0)
    ctx.step(5)
    with pytest.raises(rb.RbsogError) as e:
        ctx.sync()
    assert e.value.code == -9
    # too small a box for r_shell + skin
    with pytest.raises(rb.RbsogError) as e:
        setup_kept(rb, orc, w, skin=4.0)
    assert e.value.code == -3


@pytest.mark.parametrize("key", ["nacl_64k", "liclnacl_216k", "nacl_1m"])
def test_kept_full_size_sampled(rb, orc, key):
    """Full-size workloads with kept lists (skin 1 A, rebuilt every 10 steps):
    lists and batches of sampled atoms bit-exact at the build and five steps
    later, and the batches the pair sums read; mixed near field of the sample
    within 1e-5 of the oracle's.  At N = 64,000 B's 16-bit rows are in use."""
    w, cfg = W.make(key)
    ctx, S = setup_kept(rb, orc, w, list_every=10, P_R=cfg.P_R, P_F=cfg.P_F, precision=rb.MIXED, seed=cfg.seed,
                        step=3)
    ctx.set_velocities(W.maxwell_boltzmann(w, 1200.0))
    ctx.compute_forces()
    sel = np.linspace(0, w.n - 1, 96).astype(np.int64)
    g = ctx.debug_kept_lists(sel)
    o = S.lists_skin(sel, cap_a=64, cap_b=512)
    for k in ("nA", "nB", "A", "B", "nbatch", "batch", "weight"):
        np.testing.assert_array_equal(g[k], o[k], err_msg=k)
    check_batch_used(ctx, sel, o, cfg.P_R)
    if key == "nacl_64k":
        assert ctx.debug_kept_b16()
    ctx.step(5)
    pos, _, step = ctx.get_state()
    assert step == 8
    parts = ctx.debug_parts()
    S.pos, S.step = pos, step
    g = ctx.debug_kept_lists(sel)
    o = S.lists_skin(sel, cap_a=64, cap_b=512)
    for k in ("nA", "nB", "A", "B", "nbatch", "batch", "weight"):
        np.testing.assert_array_equal(g[k], o[k], err_msg=k)
    check_batch_used(ctx, sel, o, cfg.P_R)     # the step's evaluation drew for step 8
    assert rms_rel(parts["near"][sel], S.near(sel)) < MIXED_TOL


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_kept_auto_rebuild_trajectory(rb, orc, precision):
    """list_every = -1: the device rebuilds the lists whenever an atom has
    moved by more than skin/2; a hot run with a thin skin rebuilds several
    times, at the same steps as the oracle, and follows its trajectory (FP64)
    or stays within the mixed force tolerance (mixed, at the GPU's state)."""
    w = W.rock_salt((6, 6, 6), seed=4, composition="LiCl")
    v0 = W.maxwell_boltzmann(w, 3000.0)
    prec = rb.FP64 if precision == "fp64" else rb.MIXED
    ctx, S = setup_kept(rb, orc, w, skin=0.15, list_every=-1, P_F=100, precision=prec, integrator=rb.NVE_VV)
    ctx.set_velocities(v0)
    ctx.step(12)
    pos, vel, step = ctx.get_state()
    builds = ctx.list_builds()
    if precision == "fp64":
        vo, _ = S.run(v0, 12, 0.001, integrator=0)
        assert S.builds >= 2
        assert builds == 1 + S.builds                # the first evaluation builds too
        assert np.sqrt(((pos - S.pos) ** 2).mean()) < 1e-10
        assert rms_rel(vel, vo) < 1e-10
    else:
        # mixed: rebuilt several times, and the kept lists still hold every
        # pair inside r_shell at the GPU's current positions
        assert builds >= 3
        Fg = ctx.compute_forces()
        assert np.isfinite(Fg).all()
        R = orc.System(pos, w.species, w.charge, w.mass, w.bmh, w.box, P_R=20, P_F=100, seed=3, step=step)
        sel = np.arange(0, w.n, 37)
        Lr = R.lists(sel, cap_core=128, cap_shell=1024, batch=False)
        g = ctx.debug_kept_lists(sel)
        for q in range(sel.size):
            have = set(g["A"][q, :g["nA"][q]].tolist()) | set(g["B"][q, :g["nB"][q]].tolist())
            need = set(Lr["core"][q, :Lr["ncore"][q]].tolist()) | set(Lr["shell"][q, :Lr["nshell"][q]].tolist())
            assert need <= have


def test_kept_virial(rb, orc):
    """The virial of the kept-list estimator, FP64, three steps after the build."""
    w = W.rock_salt((9, 9, 9), seed=5)
    v0 = W.maxwell_boltzmann(w, 1200.0)
    ctx, S = setup_kept(rb, orc, w, list_every=10, P_F=300)
    ctx.set_velocities(v0)
    ctx.step(3)
    pos, vel, step = ctx.get_state()
    Fg, Eg, Wg = ctx.compute_forces(energy=True, virial=True)
    S.build_pos = w.pos.copy()
    S.pos, S.step = pos, step
    o = S.forces(energy=True)
    assert float(np.abs(Wg - o["virial"]).max() / np.abs(o["virial"]).max()) < 1e-11


@pytest.mark.parametrize("kept", [False, True])
def test_species_core_radii(rb, orc, kept):
    """Species-dependent core radii (sigma rule): lists / kept lists and batches
    bit-exact, FP64 forces within 1e-12, in both list modes."""
    w = W.rock_salt((9, 9, 9), seed=6, composition="LiCl-NaCl")
    rc = W.core_radii_from_sigma(w.bmh, 6.0)
    kw = dict(list_every=4, skin=1.0) if kept else dict(list_every=0, skin=0.0)
    S = orc.System(w.pos, w.species, w.charge, w.mass, w.bmh, w.box, P_R=20, P_F=200, seed=3, step=5,
                   r_core_pair=rc, **kw)
    prm = rb.MethodParams(s=S.s, w0=float(S.w[0]), P_R=20, P_F=200, seed=3, precision=rb.FP64, **kw)
    ctx = rb.Context(0)
    ctx.set_system(w.pos, w.species, w.charge, w.mass, w.bmh, w.box, prm)
    ctx.set_core_radii(rc)
    ctx.set_state(w.pos, np.zeros_like(w.pos), 5)
    Fg = ctx.compute_forces()
    sel = np.arange(w.n)
    if kept:
        g = ctx.debug_kept_lists(sel)
        o = S.lists_skin(sel, cap_a=64, cap_b=512)
        keys = ("nA", "nB", "A", "B", "nbatch", "batch", "weight")
    else:
        g = ctx.debug_lists(sel, cap_core=128, cap_shell=512)
        o = S.lists(sel, cap_core=128, cap_shell=512)
        keys = ("ncore", "nshell", "core", "shell", "nbatch", "batch", "weight")
    for k in keys:
        np.testing.assert_array_equal(g[k], o[k], err_msg=k)
    o = S.forces()
    parts = ctx.debug_parts()
    assert rms_rel(parts["near"], o["near"]) < FP64_TOL
    assert rms_rel(parts["far"], o["far"]) < FP64_TOL
    assert rms_rel(Fg, o["F"]) < FP64_TOL
    # the split really differs from the single radius
    R = orc.System(w.pos, w.species, w.charge, w.mass, w.bmh, w.box, P_R=20, step=5, **kw)
    nA = (S.lists_skin(sel)["nA"] if kept else S.lists(sel)["ncore"])
    nA0 = (R.lists_skin(sel)["nA"] if kept else R.lists(sel)["ncore"])
    assert nA.sum() < 0.9 * nA0.sum()


def test_bench_launch_configuration(rb, orc):
    """The configuration the benchmark times: molten NaCl N = 64,000 (P_R = 20,
    P_F = 500), kept lists rebuilt by the device whenever an atom has moved by
    more than skin/2 (list_every = -1, skin 1.5 A, the autotuner's choice on
    this workload), mixed precision, Langevin steps launched as the captured
    step graph.  Stepping one launch at a time until the device rebuilds the
    lists: the rebuilt lists and batches of 96 sampled atoms are bit-exact
    against the oracle's, built at the same positions; three steps later (the
    same lists, new batches) they still are, and the sample's near field is
    within the mixed tolerance of the oracle's FP64 one."""
    w, cfg = W.make("nacl_64k")
    ctx, S = setup_kept(rb, orc, w, skin=1.5, list_every=-1, P_R=cfg.P_R, P_F=cfg.P_F, precision=rb.MIXED,
                        seed=cfg.seed)
    ctx.set_velocities(W.maxwell_boltzmann(w, cfg.T))
    ctx.step(1)
    builds = ctx.list_builds()
    for _ in range(80):
        ctx.step(1)
        if ctx.list_builds() > builds:
            break
    else:
        pytest.fail("the device did not rebuild the lists in 80 steps at 1200 K")
    builds = ctx.list_builds()
    pos, _, step = ctx.get_state()
    S.pos, S.step, S.build_pos = pos, step, pos.copy()
    sel = np.linspace(0, w.n - 1, 96).astype(np.int64)
    keys = ("nA", "nB", "A", "B", "nbatch", "batch", "weight")
    g, o = ctx.debug_kept_lists(sel), S.lists_skin(sel, cap_a=64, cap_b=512)
    for k in keys:
        np.testing.assert_array_equal(g[k], o[k], err_msg=k)
    ctx.step(3)
    pos, _, step = ctx.get_state()
    if ctx.list_builds() != builds:                  # rebuilt again within three steps: rare
        S.build_pos = pos.copy()
    S.pos, S.step = pos, step
    parts = ctx.debug_parts()
    g, o = ctx.debug_kept_lists(sel), S.lists_skin(sel, cap_a=64, cap_b=512)
    for k in keys:
        np.testing.assert_array_equal(g[k], o[k], err_msg=k)
    check_batch_used(ctx, sel, o, cfg.P_R)           # read from B's 16-bit rows
    assert ctx.debug_kept_b16()
    assert rms_rel(parts["near"][sel], S.near(sel)) < MIXED_TOL


@pytest.mark.parametrize("list_every", [-1, 4])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_kept_resume_bit_identical(rb, orc, list_every, precision):
    """Save + restore + run(n) = run(2n) bit for bit with kept lists when the
    restore passes the lists' build positions on (rbsog_get_list_origin /
    rbsog_set_list_origin): automatic rebuilds and a fixed schedule (the split
    falls between two builds), both precisions.  Without the origin the
    restored run builds at the restored positions and departs."""
    w = W.rock_salt((6, 6, 6), seed=4, composition="LiCl")
    v0 = W.maxwell_boltzmann(w, 2500.0)
    prec = rb.FP64 if precision == "fp64" else rb.MIXED
    runs = []
    for mode in ("continuous", "origin", "no_origin"):
        ctx, _ = setup_kept(rb, orc, w, skin=0.4, list_every=list_every, P_F=100, precision=prec)
        ctx.set_velocities(v0)
        if mode == "continuous":
            ctx.step(14)
            runs.append(ctx.get_state())
            builds = ctx.list_builds()
            continue
        ctx.step(7)
        p, v, s = ctx.get_state()
        origin = ctx.list_origin()
        moved = not np.array_equal(origin, p)            # the last build was before the split
        assert moved or list_every == -1
        ctx2, _ = setup_kept(rb, orc, w, skin=0.4, list_every=list_every, P_F=100, precision=prec)
        ctx2.set_state(p, v, s)
        if mode == "origin":
            ctx2.set_list_origin(origin)
        ctx2.step(7)
        runs.append(ctx2.get_state())
    assert builds >= 3                                   # several builds, some before the split
    np.testing.assert_array_equal(runs[1][0], runs[0][0])
    np.testing.assert_array_equal(runs[1][1], runs[0][1])
    assert runs[1][2] == runs[0][2] == 14
    if moved:
        assert not np.array_equal(runs[2][0], runs[0][0])


def test_checkpoint_file_restart(rb, orc, tmp_path):
    """Context.checkpoint / restore through a file: a Nose-Hoover run with
    automatic kept lists, stopped halfway, written, read into a new context
    and continued, ends bit for bit where the uninterrupted run ends."""
    w = W.rock_salt((6, 6, 6), seed=5, composition="LiCl-NaCl")
    v0 = W.maxwell_boltzmann(w, 2200.0)
    S = orc.System(w.pos, w.species, w.charge, w.mass, w.bmh, w.box, P_R=20, P_F=100, seed=7)
    prm = rb.MethodParams(s=S.s, w0=float(S.w[0]), P_R=20, P_F=100, seed=7, precision=rb.MIXED,
                          integrator=rb.NOSE_HOOVER, T=1800.0, tdamp=0.05, nh_chain=3, list_every=-1, skin=0.4)

    def fresh():
        c = rb.Context(0)
        c.set_system(w.pos, w.species, w.charge, w.mass, w.bmh, w.box, prm)
        c.set_velocities(v0)
        return c

    ref = fresh()
    ref.step(16)
    end = ref.get_state()
    first = fresh()
    first.step(8)
    first.checkpoint(str(tmp_path / "ck.npz"))
    second = fresh()
    second.restore(str(tmp_path / "ck.npz"))
    second.step(8)
    got = second.get_state()
    assert ref.list_builds() >= 3
    np.testing.assert_array_equal(got[0], end[0])
    np.testing.assert_array_equal(got[1], end[1])
    assert got[2] == end[2] == 16
    np.testing.assert_array_equal(second.thermostat()[1], ref.thermostat()[1])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_move_atoms_keeps_lists(rb, orc, precision):
    """rbsog_move_atoms (positions from the caller, as a host-side integrator
    gives them) keeps the kept lists: a move below skin/2 reuses the last build
    (no new build; forces equal the oracle's kept-list forces with the old build
    positions), a move past skin/2 makes the device rebuild at the new
    positions (one more build; forces with those as build positions)."""
    w = W.rock_salt((6, 6, 6), seed=4, composition="LiCl")
    prec = rb.FP64 if precision == "fp64" else rb.MIXED
    tol = 1e-12 if precision == "fp64" else MIXED_TOL
    ctx, S = setup_kept(rb, orc, w, skin=1.0, list_every=-1, P_F=100, precision=prec)
    ctx.compute_forces()
    b0 = ctx.list_builds()
    rng = np.random.default_rng(1)
    small = w.pos + rng.uniform(-0.2, 0.2, w.pos.shape)      # every atom within 0.35 A < skin/2
    ctx.move_atoms(small, 5)
    Fg = ctx.compute_forces()
    assert ctx.list_builds() == b0
    S.pos, S.step, S.build_pos = small, 5, w.pos.copy()
    assert rms_rel(Fg, S.forces()["F"]) < tol
    big = small.copy()
    big[0] += 0.8                                             # one atom past skin/2 from its build position
    ctx.move_atoms(big, 6)
    Fg = ctx.compute_forces()
    assert ctx.list_builds() == b0 + 1
    S.pos, S.step, S.build_pos = big, 6, big.copy()
    assert rms_rel(Fg, S.forces()["F"]) < tol


def test_pinned_host_buffers(rb, orc):
    """Positions handed over and forces read back through page-locked host
    buffers (asynchronous copies; rbsog_move_atoms returns once its copies
    have read the caller's data) give the same forces, bit for bit, as
    pageable buffers, and the positions buffer may be overwritten as soon as
    rbsog_move_atoms returns."""
    torch = pytest.importorskip("torch")
    w = W.rock_salt((6, 6, 6), seed=4, composition="LiCl")
    out = []
    for pinned in (False, True):
        ctx, S = setup_kept(rb, orc, w, skin=1.0, list_every=-1, P_F=100, precision=rb.MIXED)
        ctx.compute_forces()
        rng = np.random.default_rng(2)
        if pinned:
            pos = torch.empty(w.pos.shape, dtype=torch.float64, pin_memory=True).numpy()
            frc = torch.empty(w.pos.shape, dtype=torch.float64, pin_memory=True).numpy()
        else:
            pos = np.empty_like(w.pos)
            frc = np.empty_like(w.pos)
        res = []
        for k in range(3):
            pos[:] = w.pos + rng.uniform(-0.2, 0.2, w.pos.shape)
            before = pos.copy()
            ctx.move_atoms(pos, 5 + k)
            pos[:] = np.nan                                   # reused at once: the call has read it
            ctx.compute_forces(frc)
            res.append(frc.copy())
            np.testing.assert_array_equal(ctx.get_state()[0], before)
        out.append(res)
        ctx.close()
    for a, b in zip(out[0], out[1]):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_forces_at_matches_move_and_compute(rb, orc, precision):
    """rbsog_forces_at (positions in, forces out, one call) gives the forces of
    rbsog_move_atoms followed by rbsog_compute_forces bit for bit, with
    pageable and page-locked host arrays and with device tensors, through a
    move below skin/2 (the last build's lists kept), one past it (rebuilt on
    the device) and one more; the first equals the oracle's kept-list forces."""
    torch = pytest.importorskip("torch")
    w = W.rock_salt((6, 6, 6), seed=4, composition="LiCl")
    prec = rb.FP64 if precision == "fp64" else rb.MIXED
    tol = 1e-12 if precision == "fp64" else MIXED_TOL
    rng = np.random.default_rng(3)
    small = w.pos + rng.uniform(-0.2, 0.2, w.pos.shape)      # every atom within 0.35 A < skin/2
    big = small.copy()
    big[0] += 0.8                                             # one atom past skin/2
    moves = [(small, 5), (big, 6), (big + rng.uniform(-0.1, 0.1, w.pos.shape), 7)]
    ctx, S = setup_kept(rb, orc, w, skin=1.0, list_every=-1, P_F=100, precision=prec)
    ctx.compute_forces()
    b0 = ctx.list_builds()
    ref = []
    for pos, s in moves:
        ctx.move_atoms(pos, s)
        ref.append(ctx.compute_forces().copy())
    builds = ctx.list_builds() - b0
    ctx.close()
    assert builds == 1
    for form in ("pageable", "pinned", "device"):
        ctx, _ = setup_kept(rb, orc, w, skin=1.0, list_every=-1, P_F=100, precision=prec)
        ctx.compute_forces()
        b0 = ctx.list_builds()
        for (pos, s), F0 in zip(moves, ref):
            if form == "pageable":
                F = ctx.forces_at(pos, s)
            elif form == "pinned":
                ph = torch.empty(pos.shape, dtype=torch.float64, pin_memory=True).numpy()
                fh = torch.empty(pos.shape, dtype=torch.float64, pin_memory=True).numpy()
                ph[:] = pos
                F = ctx.forces_at(ph, s, fh).copy()
            else:
                pd = torch.tensor(pos, dtype=torch.float64, device="cuda:0")
                fd = torch.empty(pos.shape, dtype=torch.float64, device="cuda:0")
                ctx.forces_at(pd, s, fd)
                ctx.sync()
                F = fd.cpu().numpy()
            np.testing.assert_array_equal(F, F0)
        assert ctx.list_builds() - b0 == builds
        with pytest.raises(ValueError):
            ctx.forces_at(moves[0][0], 5, torch.empty(w.pos.shape, dtype=torch.float64, device="cuda:0"))
        ctx.close()
    S.pos, S.step, S.build_pos = small, 5, w.pos.copy()
    assert rms_rel(ref[0], S.forces()["F"]) < tol
