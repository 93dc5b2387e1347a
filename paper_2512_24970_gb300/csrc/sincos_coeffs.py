"""Coefficients of the FP32 sine and cosine polynomials of the mixed-precision
far field (``sincos_turn`` / ``sincos_turn2`` in rbsog_internal.cuh).

The phase is reduced to the half turn phi in [-pi/2, pi/2]; there
    sin(phi) ~ phi (1 + z (s3 + z (s5 + z (s7 + z s9)))),      z = phi^2
    cos(phi) ~ 1 + z (c2 + z (c4 + z (c6 + z (c8 + z c10)))).
Each polynomial minimises the largest absolute error over the interval
(minimax), found by linear programming on a dense grid (minimise t subject
to |p(phi_i) - f(phi_i)| <= t at every grid point), then rounded to FP32.
Run as a script to print the coefficients and the error of their FP32
Horner evaluation (each step rounded to binary32, fused multiply-add).
"""
import numpy as np
from scipy.optimize import linprog

HALF_PI = np.pi / 2


def minimax(basis, target, x, scale=1e6):
    """min_c max_i |sum_k c_k basis_k(x_i) - target(x_i)| as a linear program
    (rows scaled so that the errors sit well above the solver's tolerances)."""
    B = scale * np.stack([b(x) for b in basis], axis=1)
    f = scale * target(x)
    n = B.shape[1]
    cost = np.zeros(n + 1)
    cost[-1] = 1.0
    A = np.block([[B, -np.ones((x.size, 1))], [-B, -np.ones((x.size, 1))]])
    rhs = np.concatenate([f, -f])
    res = linprog(cost, A_ub=A, b_ub=rhs, bounds=[(None, None)] * n + [(0, None)], method="highs")
    return res.x[:n] * 1.0, res.x[-1] / scale


def minimax_f32(basis, target, x):
    """Minimax coefficients that are binary32 numbers: round the lowest-order
    coefficient, refit the others with it fixed, and so on."""
    fixed = []
    err = None
    for k in range(len(basis)):
        known = lambda x: sum(np.float64(v) * basis[j](x) for j, v in enumerate(fixed)) if fixed else 0.0
        c, err = minimax(basis[k:], lambda x: target(x) - known(x), x)
        fixed.append(np.float32(c[0]))
    return np.array(fixed, dtype=np.float32), err


def fit():
    x = np.linspace(0.0, HALF_PI, 4001)
    # sin(phi) - phi = phi^3 (s3 + s5 z + s7 z^2 + s9 z^3)
    sb = [lambda x, k=k: x ** (2 * k + 3) for k in range(4)]
    s, es = minimax_f32(sb, lambda x: np.sin(x) - x, x)
    # cos(phi) - 1 = z (c2 + c4 z + ... + c10 z^4)
    cb = [lambda x, k=k: x ** (2 * k + 2) for k in range(5)]
    c, ec = minimax_f32(cb, lambda x: np.cos(x) - 1.0, x)
    return s, c, es, ec


def f32(v):
    return np.float32(v)


def fma32(a, b, c):
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def eval32(phi, s, c):
    phi = phi.astype(np.float32)
    z = (phi * phi).astype(np.float32)
    ps = fma32(fma32(fma32(s[3], z, s[2]), z, s[1]), z, s[0])
    sn = fma32((ps * z).astype(np.float32), phi, phi)
    pc = fma32(fma32(fma32(fma32(c[4], z, c[3]), z, c[2]), z, c[1]), z, c[0])
    cs = fma32(pc, z, np.float32(1.0))
    return sn, cs


if __name__ == "__main__":
    s, c, es, ec = fit()
    print("sin s3..s9:", ", ".join("%.9ef" % v for v in s), " minimax error %.2e" % es)
    print("cos c2..c10:", ", ".join("%.9ef" % v for v in c), " minimax error %.2e" % ec)
    phi = np.linspace(-HALF_PI, HALF_PI, 2000001)
    z = phi * phi
    ps64 = phi + phi * z * (s[0] + z * (s[1] + z * (s[2] + z * np.float64(s[3]))))
    pc64 = 1.0 + z * (c[0] + z * (c[1] + z * (c[2] + z * (c[3] + z * np.float64(c[4])))))
    print("FP32-rounded coefficients in FP64: max |sin err| %.2e, max |cos err| %.2e" %
          (np.abs(ps64 - np.sin(phi)).max(), np.abs(pc64 - np.cos(phi)).max()))
    sn, cs = eval32(phi, s, c)
    p32 = phi.astype(np.float32).astype(np.float64)
    print("FP32 evaluation: max |sin err| %.2e, max |cos err| %.2e" %
          (np.abs(sn - np.sin(p32)).max(), np.abs(cs - np.cos(p32)).max()))
