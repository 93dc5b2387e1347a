"""Sensitivity of the oracle's pins.

Each case plants one plausible mistake (a dropped term, a wrong sign or
factor, a transposed operand, an off-by-one range, a wrong index) in a copy of
the C oracle, compiles the copy into a temporary directory, swaps it in for the
oracle's library and checks that the pin aimed at that part of the method
fails.  The unchanged oracle passes the same pins in their own modules; the
committed oracle source is never changed.  Together the cases show that a
mistake in the pair terms (Eq. (Fshort)), the far field (Eqs. (Long),
(long-rangeforce)), the phases, the list predicate, the shell batch (Sec. 2.2),
the k-space sampler (Eq. (Pk)), the self term, the virial, the kept lists'
indicator and weight, or the random streams does not pass the pins unnoticed."""
import ctypes
import importlib.util
import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _load(name):
    spec = importlib.util.spec_from_file_location("pins_" + name, os.path.join(HERE, "test_oracle_%s.py" % name))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


# (case, pin module, pin function, pin arguments beyond orc, [(text, replacement, occurrences)])
CASES = [
    ("sog_residual_without_m0", "physics", "test_sog_matches_ewald", {},
     [("  double g = 0.0, f = 0.0;\n  for (int m = 0; m <= S->M; m++) {",
       "  double g = 0.0, f = 0.0;\n  for (int m = 1; m <= S->M; m++) {", 1)]),
    ("far_force_sign", "physics", "test_force_is_minus_energy_gradient", {},
     [("F[3 * q + e] = -ORC_KE * qi / V * f[e];", "F[3 * q + e] = ORC_KE * qi / V * f[e];", 1)]),
    ("k_without_two_pi", "physics", "test_force_is_minus_energy_gradient", {},
     [("kv[3 * p + e] = 2.0 * M_PI * m[3 * p + e] / S->L[e];", "kv[3 * p + e] = M_PI * m[3 * p + e] / S->L[e];", 1)]),
    ("dispersion_force_power", "physics", "test_force_is_minus_energy_gradient", {},
     [("- 6.0 * C / r8 -", "- 6.0 * C / (r6 * r) -", 1)]),
    ("phase_operands_transposed", "physics", "test_sog_matches_ewald", {},
     [("(uint32_t)m[1] * u[1] + (uint32_t)m[2] * u[2];", "(uint32_t)m[1] * u[2] + (uint32_t)m[2] * u[1];", 1)]),
    ("far_phase_sign", "physics", "test_sog_matches_ewald", {},
     [("cs * rho[2 * p + 1] - sn * rho[2 * p];", "cs * rho[2 * p + 1] + sn * rho[2 * p];", 1)]),
    ("no_minimum_image_in_pairs", "physics", "test_sog_matches_ewald", {},
     [("(double)(int32_t)(ui[a] - uj[a]) * sc[a]", "((double)ui[a] - (double)uj[a]) * sc[a]", 4)]),
    ("self_term_without_m0", "physics", "test_madelung_rock_salt", {},
     [("for (int m = 0; m <= S->M; m++) f0 += S->w[m];", "for (int m = 1; m <= S->M; m++) f0 += S->w[m];", 1)]),
    ("predicate_without_z", "physics", "test_lists_against_float64_distances", {},
     [("  r2 = fmaf(d[2], d[2], r2);\n", "", 1)]),
    ("shell_batch_unweighted", "physics", "test_rbl_estimator_unbiased", {},
     [("wgt = (double)ns / (double)S->P_R;", "wgt = 1.0;", 1)]),
    ("floyd_range_off_by_one", "rng", "test_floyd_uniform_subsets", {},
     [("((uint64_t)J + 1u)", "((uint64_t)J)", 1)]),
    ("philox_multiplier", "rng", "test_philox_matches_curand_host", {"seed": 1},
     [("0xCD9E8D57u * (uint64_t)x2", "0xCD9E8D55u * (uint64_t)x2", 1)]),
    ("sampler_without_k2_weight", "sog", "test_S_closed_form_vs_lattice_sum", {"box": (31.5, 31.5, 31.5)},
     [("e2[q] = k * k * e0[q];", "e2[q] = e0[q];", 1)]),
    ("virial_xz_index", "virial", "test_two_atom_pair_virial", {},
     [("w[4] += d[0] * phi * d[2];", "w[4] += d[1] * phi * d[2];", 1)]),
    ("kept_lists_without_indicator", "skin", "test_skin_whole_batch_is_cutoff_force_after_motion", {},
     [("if (!(pred_r2(ui, uj, Gn.h) < Gn.rs2)) continue;", "(void)0;", 2)]),
    ("kept_batch_unweighted", "skin", "test_skin_estimator_unbiased", {},
     [("wgt = (double)n_b / (double)S->P_R;", "wgt = 1.0;", 1)]),
]


@pytest.fixture(scope="module")
def pins():
    return {m: _load(m) for m in ("physics", "rng", "sog", "virial", "skin")}


def _build(orc, tmp_path, name, edits):
    """The oracle source with `edits` applied, compiled like the oracle."""
    with open(orc._SRC) as f:
        src = f.read()
    for text, repl, count in edits:
        assert src.count(text) == count, (name, text)       # the mistake lands where intended
        src = src.replace(text, repl)
    c_path, so_path = str(tmp_path / ("%s.c" % name)), str(tmp_path / ("lib%s.so" % name))
    with open(c_path, "w") as f:
        f.write(src)
    orc.compile_c(c_path, so_path)
    return so_path


def _run_pin(orc, pins, so_path, mod, fn, kw):
    """Run the pin with the library at so_path in place of the oracle's."""
    args = dict(kw)
    if mod == "sog":
        args["sog"] = orc.sog_solve(pins["sog"].B, pins["sog"].M, pins["sog"].RC)
    saved = orc.lib()
    swapped = ctypes.CDLL(so_path)
    orc._declare(swapped)
    orc._lib = swapped
    try:
        getattr(pins[mod], fn)(orc, **args)
    finally:
        orc._lib = saved


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_pin_catches_planted_mistake(orc, pins, tmp_path, case):
    name, mod, fn, kw, edits = case
    so_path = _build(orc, tmp_path, name, edits)
    with pytest.raises(AssertionError):
        _run_pin(orc, pins, so_path, mod, fn, kw)


PINS = sorted({(c[1], c[2], tuple(sorted(c[3].items()))) for c in CASES})


@pytest.mark.parametrize("pin", PINS, ids=["%s.%s" % (p[0], p[1]) for p in PINS])
def test_control_unchanged_source_passes(orc, pins, tmp_path, pin):
    """The same harness with no mistake planted: every pin above passes, so a
    failure in a mutant case comes from its mistake."""
    mod, fn, kw = pin
    _run_pin(orc, pins, _build(orc, tmp_path, "control", []), mod, fn, dict(kw))


# The oracle's Python parts (integrators, kinetic tensor): the same, with the
# mistake planted in a copy of oracle/__init__.py loaded as a separate module
# that uses the oracle's C library.
PY_CASES = [
    ("baoab_noise_amplitude", "langevin", "test_baoab_free_particles_relax_to_equipartition", {},
     [("sig = np.sqrt((1.0 - c1 * c1) * KB", "sig = np.sqrt((1.0 - c1) * KB", 1)]),
    ("baoab_friction_half", "langevin", "test_baoab_free_particles_relax_to_equipartition", {},
     [("c1 = np.exp(-gamma * dt)", "c1 = np.exp(-0.5 * gamma * dt)", 1)]),
    ("nose_hoover_G0_sign", "nh", "test_nh_conserves_extended_energy", {},
     [("return (k2 - self.g * self.kT) / self.Q[0]", "return (k2 + self.g * self.kT) / self.Q[0]", 1)]),
    ("nose_hoover_scale_direction", "nh", "test_nh_conserves_extended_energy", {},
     [("s = float(np.exp(-d * self.v[0]))", "s = float(np.exp(d * self.v[0]))", 1)]),
    ("kinetic_tensor_components", "virial", "test_kinetic_tensor", {},
     [("for c, (a, b) in enumerate(((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))):\n            out[c]",
       "for c, (a, b) in enumerate(((0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (0, 2))):\n            out[c]", 1)]),
]


@pytest.fixture(scope="module")
def py_pins():
    return {m: _load(m) for m in ("langevin", "nh", "virial")}


def _py_oracle(orc, tmp_path, name, edits):
    """A copy of the oracle's Python module with `edits` applied, on the oracle's C library."""
    src_path = os.path.join(os.path.dirname(orc._SRC), "__init__.py")
    with open(src_path) as f:
        src = f.read()
    for text, repl, count in edits:
        assert src.count(text) == count, (name, text)
        src = src.replace(text, repl)
    path = str(tmp_path / ("oracle_%s.py" % name))
    with open(path, "w") as f:
        f.write(src)
    spec = importlib.util.spec_from_file_location("oracle_" + name, path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    orc.lib()                                       # the oracle's library, built
    mod._SRC, mod._LIB, mod._lib = orc._SRC, orc._LIB, None   # the copy opens it with its own declarations
    return mod


@pytest.mark.parametrize("case", PY_CASES, ids=[c[0] for c in PY_CASES])
def test_python_pin_catches_planted_mistake(orc, py_pins, tmp_path, case):
    name, mod, fn, kw, edits = case
    bad = _py_oracle(orc, tmp_path, name, edits)
    with pytest.raises(AssertionError):
        getattr(py_pins[mod], fn)(bad, **kw)


PY_PINS = sorted({(c[1], c[2]) for c in PY_CASES})


@pytest.mark.parametrize("pin", PY_PINS, ids=["%s.%s" % p for p in PY_PINS])
def test_python_control_unchanged_source_passes(orc, py_pins, tmp_path, pin):
    mod, fn = pin
    getattr(py_pins[mod], fn)(_py_oracle(orc, tmp_path, "control", []))

