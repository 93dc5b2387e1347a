"""The kinetic tensor K = sum_i m_i v_i (x) v_i of the current velocities
(rbsog_get_kinetic_tensor), the velocity half of the stress S = K + W, through
the C ABI against the oracle's definition, for host and device outputs, in both
precision modes, after MD steps (velocities the device integrated)."""
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


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_kinetic_tensor(rb, orc, precision):
    import torch
    w = W.rock_salt((7, 7, 7), seed=4, composition="LiCl-NaCl")
    w.vel = W.maxwell_boltzmann(w, 1250.0)
    prm = rb.MethodParams(P_R=20, P_F=200, precision=rb.FP64 if precision == "fp64" else rb.MIXED, T=1250.0)
    ctx = rb.Context(0)
    ctx.set_workload(w, prm)
    S = orc.System(w.pos, w.species, w.charge, w.mass, w.bmh, w.box)
    for nsteps in (0, 7):
        ctx.step(nsteps)
        ctx.sync()
        _, vel, _ = ctx.get_state()
        ref = S.kinetic_tensor(vel)
        K = ctx.kinetic_tensor()
        np.testing.assert_allclose(K, ref, rtol=1e-12, atol=1e-12 * np.abs(ref[:3]).max())
        out = torch.zeros(6, dtype=torch.float64, device="cuda")
        ctx.kinetic_tensor(out=out)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), K)      # same kernels, same order
    # with the virial: the stress S = K + W is finite and symmetric in the
    # order (xx, yy, zz, xy, xz, yz); tr K = 2 E_kin
    _, Wv = ctx.compute_forces(virial=True)
    assert np.isfinite(K + Wv).all()
    assert abs(K[:3].sum() - S.kinetic2(vel)) < 1e-12 * S.kinetic2(vel)
    ctx.close()
