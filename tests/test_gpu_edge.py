"""Degenerate and ragged inputs through the C ABI against the oracle: the
smallest neutral system (two ions, almost every cell empty), a dilute random
gas (ragged and empty rows, random cell occupancy), batches of size one
(P_R = 1, P_F = 1), in both precisions and both list modes."""
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


def rms_rel(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


def gas(n, L, seed):
    """n ions (Na+/Cl- alternating) placed uniformly at random, no two closer than 2.2 A."""
    rng = np.random.default_rng(seed)
    base = W.rock_salt((5, 5, 5), seed=1)
    pos = []
    while len(pos) < n:
        p = rng.uniform(0.0, L, 3)
        if all(np.linalg.norm((p - q) - L * np.round((p - q) / L)) > 2.2 for q in pos):
            pos.append(p)
    species = np.array([k % 2 for k in range(n)], dtype=np.int32)
    return np.array(pos), species, base.charge, base.mass, base.bmh, np.array([L, L, L])


CASES = {
    "two_ions": (lambda: (np.array([[3.0, 4.0, 5.0], [6.1, 4.9, 3.3]]), np.array([0, 1], dtype=np.int32)) +
                 gas(2, 26.0, 0)[2:5] + (np.array([26.0, 26.5, 27.0]),), 20, 50),
    "dilute_gas": (lambda: gas(40, 30.0, 5), 20, 100),
    "batches_of_one": (lambda: gas(60, 28.0, 6), 1, 1),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("mode", ["per_step", "kept"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_edge_cases(rb, orc, case, mode, precision):
    make, P_R, P_F = CASES[case]
    pos, sp, q, m, bmh, box = make()
    kw = dict(list_every=-1, skin=0.5) if mode == "kept" else dict(list_every=0, skin=0.0)
    S = orc.System(pos, sp, q, m, bmh, box, P_R=P_R, P_F=P_F, seed=9, step=3, **kw)
    prm = rb.MethodParams(s=S.s, w0=float(S.w[0]), P_R=P_R, P_F=P_F, seed=9,
                          precision=rb.FP64 if precision == "fp64" else rb.MIXED, **kw)
    ctx = rb.Context(0)
    ctx.set_system(pos, sp, q, m, bmh, box, prm)
    ctx.set_state(pos, np.zeros_like(pos), 3)
    Fg, Eg = ctx.compute_forces(energy=True)
    o = S.forces(energy=True)
    tol = 1e-12 if precision == "fp64" else 1e-5
    assert rms_rel(Fg, o["F"]) < tol
    np.testing.assert_allclose(Eg[3], o["energy"][3], rtol=max(tol, 1e-12))
    sel = np.arange(pos.shape[0])
    if mode == "kept":
        g = ctx.debug_kept_lists(sel)
        ol = S.lists_skin(sel, cap_a=64, cap_b=512)
        keys = ("nA", "nB", "A", "B", "nbatch", "batch", "weight")
    else:
        g = ctx.debug_lists(sel, cap_core=128, cap_shell=512)
        ol = S.lists(sel, cap_core=128, cap_shell=512)
        keys = ("ncore", "nshell", "core", "shell", "nbatch", "batch", "weight")
    for k in keys:
        np.testing.assert_array_equal(g[k], ol[k], err_msg=k)
    # a few MD steps run and stay finite
    ctx.set_velocities(np.zeros_like(pos))
    ctx.step(3)
    ctx.sync()
    p1, v1, s1 = ctx.get_state()
    assert s1 == 6 and np.isfinite(p1).all() and np.isfinite(v1).all()


def test_empty_and_single_ion_rejected(rb):
    """No system of fewer than two ions (a neutral system needs two): n = 0 and
    n = 1 fail with RBSOG_E_INVAL and leave the context without a system."""
    w = W.rock_salt((5, 5, 5), seed=1)
    prm = rb.MethodParams()
    ctx = rb.Context(0)
    for n in (0, 1):
        with pytest.raises(rb.RbsogError) as e:
            ctx.set_system(w.pos[:n], w.species[:n], w.charge, w.mass, w.bmh, w.box, prm)
        assert e.value.code == -1
    with pytest.raises(rb.RbsogError) as e:
        ctx.compute_forces()
    assert e.value.code == -8                         # RBSOG_E_NO_SYSTEM
    ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_largest_batches(rb, orc, precision):
    """P_R at its cap (RBSOG_MAX_PR = 64) and P_F = 2000 (four columns of the
    structure factor, four chunks of the far-field force, the last ragged):
    lists, batches and k-batch bit-exact, forces within the precision's bound."""
    w = W.rock_salt((6, 6, 6), seed=8, composition="LiCl-NaCl")
    P_R, P_F = 64, 2000
    S = orc.System(w.pos, w.species, w.charge, w.mass, w.bmh, w.box, P_R=P_R, P_F=P_F, seed=11, step=2)
    prm = rb.MethodParams(s=S.s, w0=float(S.w[0]), P_R=P_R, P_F=P_F, seed=11,
                          precision=rb.FP64 if precision == "fp64" else rb.MIXED)
    ctx = rb.Context(0)
    ctx.set_system(w.pos, w.species, w.charge, w.mass, w.bmh, w.box, prm)
    ctx.set_state(w.pos, np.zeros_like(w.pos), 2)
    Fg = ctx.compute_forces()
    sel = np.arange(0, w.n, 29)
    g = ctx.debug_lists(sel, cap_core=128, cap_shell=512)
    o = S.lists(sel, cap_core=128, cap_shell=512)
    for k in ("ncore", "nshell", "core", "shell", "nbatch", "batch", "weight"):
        np.testing.assert_array_equal(g[k], o[k], err_msg=k)
    m, c, _ = S.kbatch()
    mg, cg = ctx.debug_kbatch()
    np.testing.assert_array_equal(mg, m)
    ref = S.forces()["F"]
    assert rms_rel(Fg, ref) < (1e-12 if precision == "fp64" else 1e-5)
    ctx.close()
