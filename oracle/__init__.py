"""FP64 CPU oracle of the RBSOG + RBL force evaluation (arXiv 2512.24970).

TEST INFRASTRUCTURE ONLY: the plain, slow reference the CUDA library is
checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import it.  It shares no
code with the CUDA path; the C part (``rbsog_oracle.c``) is compiled with gcc
by :func:`build`.

Sections of the paper followed here (Sec. 2.1 split and spectral form,
Sec. 2.2 RBL and RBSOG estimators, Sec. 2.3 Langevin dynamics) are cited on
each function.  Parity of the sampled MD trajectory statistics is unpinned
(the paper's observables need PPPM runs); everything else is pinned by the
tests listed in the repository's design notes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rbsog_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

KE = 14.3996454784          # eV * Angstrom / e^2
KB = 8.617333262e-5         # eV / K
FCONV = 9648.53321          # (eV / Angstrom) / amu -> Angstrom / ps^2

INTEGRATOR_NVE_VV = 0
INTEGRATOR_LANGEVIN_BAOAB = 1
INTEGRATOR_NOSE_HOOVER = 2


class NHChain:
    """Nose-Hoover chain thermostat of length M (Martyna, Tuckerman, Klein,
    Mol. Phys. 87 (1996) 1117), the NVT thermostat of the paper's production
    runs (Sec. 3).  Masses Q_0 = g kT tau^2, Q_j = kT tau^2; forces on the
    chain G_0 = (2K - g kT)/Q_0, G_j = (Q_{j-1} v_{j-1}^2 - kT)/Q_j.  One half
    step of length d = dt/2 (one Trotter stage, no Suzuki-Yoshida weights):
    the chain from its end to v_0 (each v_j damped by e^{-d v_{j+1}/4} before
    and after its kick d G_j / 2), the velocity scale s = e^{-d v_0}, the
    positions eta_j += d v_j, then the chain back from v_0 to its end.
    K in eV, v_j in 1/ps."""

    def __init__(self, M, T, tdamp, ndof):
        self.M, self.g = int(M), float(ndof)
        self.kT = KB * float(T)
        self.Q = np.array([self.g * self.kT * tdamp ** 2] + [self.kT * tdamp ** 2] * (self.M - 1))
        self.eta = np.zeros(self.M)
        self.v = np.zeros(self.M)

    def _G(self, j, k2):
        if j == 0:
            return (k2 - self.g * self.kT) / self.Q[0]
        return (self.Q[j - 1] * self.v[j - 1] ** 2 - self.kT) / self.Q[j]

    def _kick(self, j, k2, d):
        if j + 1 < self.M:
            x = np.exp(-0.25 * d * self.v[j + 1])
            self.v[j] = (self.v[j] * x + 0.5 * d * self._G(j, k2)) * x
        else:
            self.v[j] += 0.5 * d * self._G(j, k2)

    def half_step(self, k2, dt):
        """k2 = sum_i m_i v_i^2 in eV (twice the kinetic energy); returns the
        factor that scales every velocity."""
        d = 0.5 * dt
        for j in range(self.M - 1, -1, -1):
            self._kick(j, k2, d)
        s = float(np.exp(-d * self.v[0]))
        k2 *= s * s
        self.eta += d * self.v
        for j in range(self.M):
            self._kick(j, k2, d)
        return s

    def energy(self):
        """Thermostat part of the conserved quantity."""
        return float(0.5 * (self.Q * self.v ** 2).sum() + self.g * self.kT * self.eta[0]
                     + self.kT * self.eta[1:].sum())


def compile_c(src: str, out: str) -> None:
    """gcc -O2, no FP contraction, OpenMP: the one way the C oracle is built."""
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-shared", "-fPIC", src, "-o", out, "-lm"]
    subprocess.check_call(cmd)


def build(force: bool = False) -> str:
    """Compile the C oracle (compile_c) into oracle/_build."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        compile_c(_SRC, tmp)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _declare(_lib)
    return _lib


class _Sys(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64), ("n_species", ctypes.c_int32), ("M", ctypes.c_int32),
        ("pos", ctypes.c_void_p), ("species", ctypes.c_void_p), ("charge", ctypes.c_void_p),
        ("bmh", ctypes.c_void_p), ("w", ctypes.c_void_p),
        ("L", ctypes.c_double * 3), ("b", ctypes.c_double), ("s", ctypes.c_double),
        ("r_core", ctypes.c_double), ("r_shell", ctypes.c_double),
        ("P_R", ctypes.c_int32), ("P_F", ctypes.c_int32),
        ("seed", ctypes.c_uint64), ("step", ctypes.c_int64), ("skin", ctypes.c_double),
        ("r_core_pair", ctypes.c_void_p),
    ]


_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_U32 = ctypes.c_uint32
_U64 = ctypes.c_uint64
_D = ctypes.c_double


def _declare(L):
    sp = ctypes.POINTER(_Sys)
    L.orc_philox.argtypes = [_I64, _P, _P, _P]
    L.orc_draw.argtypes = [_U64, _I64, _I64, _P, _U32, _U32, _P]
    L.orc_sog_solve.argtypes = [_D, _I32, _D, _P, _P]
    L.orc_sog_solve.restype = ctypes.c_int
    L.orc_sog_eval.argtypes = [_I32, _D, _D, _P, _I64, _P, _P, _P]
    L.orc_sog_fhat.argtypes = [sp, _I64, _P, _P]
    L.orc_sog_fhat_dk2.argtypes = [sp, _I64, _P, _P]
    L.orc_pair_terms.argtypes = [sp, _I32, _I32, _I64, _P, _P, _P]
    L.orc_fixed_point.argtypes = [sp, _P]
    L.orc_cell_grid.argtypes = [sp, _P]
    L.orc_cell_grid_skin.argtypes = [sp, _P]
    L.orc_lists_skin.argtypes = [sp, _P, _P, _I64, _I32, _I32, _P, _P, _P, _P, _P, _P, _P]
    L.orc_lists_skin.restype = ctypes.c_int
    L.orc_near_skin.argtypes = [sp, _P, _P, _I64, _I32, _P, _P, _P]
    L.orc_near_skin.restype = ctypes.c_int
    L.orc_floyd.argtypes = [_U64, _I64, _U32, _I32, _I32, _P]
    L.orc_floyd.restype = _I32
    L.orc_lists.argtypes = [sp, _P, _I64, _I32, _I32, _P, _P, _P, _P, _P, _P, _P]
    L.orc_lists.restype = ctypes.c_int
    L.orc_near.argtypes = [sp, _P, _I64, _I32, _P, _P, _P]
    L.orc_near.restype = ctypes.c_int
    L.orc_sampler_S.argtypes = [sp]
    L.orc_sampler_S.restype = _D
    L.orc_sampler_Z.argtypes = [sp, _P]
    L.orc_kbatch.argtypes = [sp, _P, _P]
    L.orc_kbatch.restype = _D
    L.orc_rho.argtypes = [sp, _I32, _P, _P]
    L.orc_far.argtypes = [sp, _I32, _P, _P, _P, _P, _I64, _P, _P]
    L.orc_self_energy.argtypes = [sp]
    L.orc_self_energy.restype = _D
    L.orc_num_threads.restype = _I32
    L.orc_set_num_threads.argtypes = [_I32]


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's later OpenMP regions."""
    lib().orc_set_num_threads(int(n))


# --------------------------------------------------------------------------
# Philox4x32-10 (Salmon et al. 2011)

def philox(ctr: np.ndarray, key) -> np.ndarray:
    """Raw Philox4x32-10 blocks: ctr [n,4] uint32, key (k0, k1) -> [n,4] uint32."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.empty_like(ctr)
    lib().orc_philox(ctr.shape[0], _ptr(ctr), _ptr(k), _ptr(out))
    return out


def draw(seed: int, step: int, index: np.ndarray, stream: int, block: int) -> np.ndarray:
    """Method draws: ctr = (index, step_lo, step_hi, stream<<24 | block), key = seed."""
    idx = np.ascontiguousarray(index, dtype=np.uint32).reshape(-1)
    out = np.empty((idx.size, 4), dtype=np.uint32)
    lib().orc_draw(seed, step, idx.size, _ptr(idx), stream, block, _ptr(out))
    return out


# --------------------------------------------------------------------------
# SOG split (Sec. 2.1)

def sog_solve(b: float = 1.3, M: int = 64, rc: float = 12.0):
    """(s, w[0..M]) with w_0 set for N(r_c) = 0 and s for N'(r_c) = 0."""
    s = np.zeros(1)
    w = np.zeros(M + 1)
    st = lib().orc_sog_solve(b, M, rc, _ptr(s), _ptr(w))
    if st != 0:
        raise RuntimeError("oracle SOG solve failed: %d" % st)
    return float(s[0]), w


def sog_eval(b, M, s, w, r):
    r = np.ascontiguousarray(r, dtype=np.float64)
    F = np.empty_like(r)
    dF = np.empty_like(r)
    lib().orc_sog_eval(M, b, s, _ptr(np.ascontiguousarray(w, dtype=np.float64)), r.size,
                       _ptr(r), _ptr(F), _ptr(dF))
    return F, dF


# --------------------------------------------------------------------------

class System:
    """A BMH system with its RBSOG/RBL parameters, held as numpy arrays.

    ``list_every = 0`` (default): the random batch list is rebuilt from the
    current positions at every evaluation (Sec. 2.2).  ``list_every = n >= 1``:
    kept lists with outer radius r_shell + ``skin``, built at the first
    evaluation, at every step that is a multiple of n, and after
    :meth:`invalidate_lists` (see ``orc_near_skin``).  ``list_every = -1``:
    kept lists rebuilt at every step where some atom has moved by more than
    skin/2 since the last build (the displacement limit under which the kept
    lists still hold every pair inside r_shell).
    """

    def __init__(self, pos, species, charge, mass, bmh, box, *, b=1.3, M=64, s=None, w=None,
                 r_core=6.0, r_shell=12.0, P_R=20, P_F=200, seed=1, step=0, skin=0.0,
                 list_every=0, r_core_pair=None):
        self.pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
        self.species = np.ascontiguousarray(species, dtype=np.int32).reshape(-1)
        self.charge = np.ascontiguousarray(charge, dtype=np.float64)
        self.mass = np.ascontiguousarray(mass, dtype=np.float64)
        ns = self.charge.size
        self.bmh = np.ascontiguousarray(bmh, dtype=np.float64).reshape(ns, ns, 5)
        self.box = np.asarray(box, dtype=np.float64).reshape(3)
        self.b, self.M = float(b), int(M)
        if s is None or w is None:
            s, w = sog_solve(self.b, self.M, float(r_shell))
        self.s = float(s)
        self.w = np.ascontiguousarray(w, dtype=np.float64)
        self.r_core, self.r_shell = float(r_core), float(r_shell)
        self.P_R, self.P_F = int(P_R), int(P_F)
        self.seed, self.step = int(seed), int(step)
        self.skin, self.list_every = float(skin), int(list_every)
        # species-dependent core radii [ns][ns] (symmetric, none above r_core) or None
        self.r_core_pair = None if r_core_pair is None else np.ascontiguousarray(r_core_pair, dtype=np.float64)
        self.build_pos = None   # positions the kept lists were built from
        self.builds = 0         # automatic rebuilds (list_every = -1) during run()

    @property
    def kept_lists(self):
        return self.list_every != 0

    def displacement_limit2(self):
        """(skin/2)^2, shaded by 2^-10 so that the FP32 list predicate's
        rounding stays inside the margin."""
        return 0.25 * self.skin * self.skin * (1.0 - 1.0 / 1024.0)

    def invalidate_lists(self):
        """The next evaluation builds the kept lists from the positions it sees."""
        self.build_pos = None

    def _ensure_lists(self):
        if self.build_pos is None:
            self.build_pos = self.pos.copy()

    @property
    def n(self):
        return self.pos.shape[0]

    @property
    def volume(self):
        return float(np.prod(self.box))

    def q(self):
        return self.charge[self.species]

    def _c(self):
        st = _Sys()
        st.n = self.n
        st.n_species = self.charge.size
        st.M = self.M
        st.pos = self.pos.ctypes.data
        st.species = self.species.ctypes.data
        st.charge = self.charge.ctypes.data
        st.bmh = self.bmh.ctypes.data
        st.w = self.w.ctypes.data
        for a in range(3):
            st.L[a] = self.box[a]
        st.b, st.s = self.b, self.s
        st.r_core, st.r_shell = self.r_core, self.r_shell
        st.P_R, st.P_F = self.P_R, self.P_F
        st.seed, st.step = self.seed, self.step
        st.skin = self.skin
        st.r_core_pair = self.r_core_pair.ctypes.data if self.r_core_pair is not None else None
        return st

    # ---- geometry -------------------------------------------------------
    def fixed_point(self):
        u = np.empty((self.n, 3), dtype=np.uint32)
        st = self._c()
        lib().orc_fixed_point(ctypes.byref(st), _ptr(u))
        return u

    def cell_grid(self):
        nc = np.zeros(3, dtype=np.int32)
        st = self._c()
        lib().orc_cell_grid(ctypes.byref(st), _ptr(nc))
        return nc

    def lists(self, sel=None, cap_core=256, cap_shell=1024, batch=True):
        """Core and shell lists (canonical order) and the shell batch of ``sel``."""
        sel = np.arange(self.n, dtype=np.int64) if sel is None else np.ascontiguousarray(sel, dtype=np.int64)
        k = sel.size
        core = np.full((k, cap_core), -1, dtype=np.int32)
        ncore = np.zeros(k, dtype=np.int32)
        shell = np.full((k, cap_shell), -1, dtype=np.int32)
        nshell = np.zeros(k, dtype=np.int32)
        PR = max(self.P_R, 1)
        bt = np.full((k, PR), -1, dtype=np.int32) if batch else None
        nb = np.zeros(k, dtype=np.int32) if batch else None
        wt = np.zeros(k, dtype=np.float64) if batch else None
        st = self._c()
        rc = lib().orc_lists(ctypes.byref(st), _ptr(sel), k, cap_core, cap_shell, _ptr(core),
                             _ptr(ncore), _ptr(shell), _ptr(nshell), _ptr(bt), _ptr(nb), _ptr(wt))
        if rc != 0:
            raise RuntimeError("oracle list capacity exceeded")
        out = dict(core=core, ncore=ncore, shell=shell, nshell=nshell)
        if batch:
            out.update(batch=bt, nbatch=nb, weight=wt)
        return out

    def cell_grid_skin(self):
        nc = np.zeros(3, dtype=np.int32)
        st = self._c()
        lib().orc_cell_grid_skin(ctypes.byref(st), _ptr(nc))
        return nc

    def lists_skin(self, sel=None, cap_a=256, cap_b=2048, batch=True):
        """Kept lists A, B (canonical order of the build positions) and the batch of ``sel``."""
        self._ensure_lists()
        sel = np.arange(self.n, dtype=np.int64) if sel is None else np.ascontiguousarray(sel, dtype=np.int64)
        k = sel.size
        A = np.full((k, cap_a), -1, dtype=np.int32)
        na = np.zeros(k, dtype=np.int32)
        B = np.full((k, cap_b), -1, dtype=np.int32)
        nb = np.zeros(k, dtype=np.int32)
        PR = max(self.P_R, 1)
        bt = np.full((k, PR), -1, dtype=np.int32) if batch else None
        nbt = np.zeros(k, dtype=np.int32) if batch else None
        wt = np.zeros(k, dtype=np.float64) if batch else None
        st = self._c()
        bp = np.ascontiguousarray(self.build_pos)
        rc = lib().orc_lists_skin(ctypes.byref(st), _ptr(bp), _ptr(sel), k, cap_a, cap_b, _ptr(A), _ptr(na),
                                  _ptr(B), _ptr(nb), _ptr(bt), _ptr(nbt), _ptr(wt))
        if rc != 0:
            raise RuntimeError("oracle list capacity exceeded")
        out = dict(A=A, nA=na, B=B, nB=nb)
        if batch:
            out.update(batch=bt, nbatch=nbt, weight=wt)
        return out

    # ---- near field (Sec. 2.2) -------------------------------------------
    def near(self, sel=None, all_shell=False, energy=False, virial=False):
        """Uncorrected near-field force F_core + F*_shell of ``sel`` (and 1/2 pair energy,
        and the per-atom pair virial [n,6] = xx, yy, zz, xy, xz, yz); with kept lists,
        the estimator of ``orc_near_skin``."""
        sel = np.arange(self.n, dtype=np.int64) if sel is None else np.ascontiguousarray(sel, dtype=np.int64)
        F = np.zeros((sel.size, 3))
        E = np.zeros(sel.size) if energy else None
        W = np.zeros((sel.size, 6)) if virial else None
        st = self._c()
        if self.kept_lists:
            self._ensure_lists()
            bp = np.ascontiguousarray(self.build_pos)
            rc = lib().orc_near_skin(ctypes.byref(st), _ptr(bp), _ptr(sel), sel.size, int(bool(all_shell)),
                                     _ptr(F), _ptr(E), _ptr(W))
        else:
            rc = lib().orc_near(ctypes.byref(st), _ptr(sel), sel.size, int(bool(all_shell)), _ptr(F), _ptr(E),
                                _ptr(W))
        if rc != 0:
            raise RuntimeError("oracle near-field capacity exceeded")
        out = (F,) + ((E,) if energy else ()) + ((W,) if virial else ())
        return out if len(out) > 1 else F

    def pair_terms(self, si, sj, r2):
        r2 = np.ascontiguousarray(r2, dtype=np.float64).reshape(-1)
        phi = np.empty_like(r2)
        e = np.empty_like(r2)
        st = self._c()
        lib().orc_pair_terms(ctypes.byref(st), si, sj, r2.size, _ptr(r2), _ptr(phi), _ptr(e))
        return phi, e

    # ---- far field (Sec. 2.1, 2.2) -----------------------------------------
    def fhat(self, k2):
        k2 = np.ascontiguousarray(k2, dtype=np.float64).reshape(-1)
        out = np.empty_like(k2)
        st = self._c()
        lib().orc_sog_fhat(ctypes.byref(st), k2.size, _ptr(k2), _ptr(out))
        return out

    def fhat_dk2(self, k2):
        """dFhat/d(k^2) of Eq. (Fouriertransform)."""
        k2 = np.ascontiguousarray(k2, dtype=np.float64).reshape(-1)
        out = np.empty_like(k2)
        st = self._c()
        lib().orc_sog_fhat_dk2(ctypes.byref(st), k2.size, _ptr(k2), _ptr(out))
        return out

    def far_virial(self, m, c, rho):
        """Virial [6] (xx, yy, zz, xy, xz, yz) of the far-field energy estimator
        U_F* = k_e/(2V) sum_p c_p |rho_p|^2: minus its derivative under a homogeneous
        strain of positions and box.  k . r does not change, k_a -> k_a - eps_ab k_b
        and V -> V (1 + tr eps), so W_ab = delta_ab U_F* + (k_e/V) sum_p c_p
        (Fhat'/Fhat)(k_p^2) k_pa k_pb |rho_p|^2, with c_p the weight of Fhat(k_p)
        (the k-batch's importance weight or, enumerated, Fhat itself)."""
        k = self.kvec(m)
        k2 = (k ** 2).sum(1)
        g = self.fhat_dk2(k2) / self.fhat(k2)
        r2 = (np.asarray(rho) ** 2).sum(1)
        V = self.volume
        UF = KE / (2.0 * V) * float((c * r2).sum())
        wk = KE / V * c * g * r2
        W = np.zeros(6)
        for comp, (a, b) in enumerate(((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))):
            W[comp] = float((wk * k[:, a] * k[:, b]).sum()) + (UF if a == b else 0.0)
        return W

    def sampler_S(self):
        st = self._c()
        return float(lib().orc_sampler_S(ctypes.byref(st)))

    def sampler_Z(self):
        Z = np.zeros((self.M + 1, 3))
        st = self._c()
        lib().orc_sampler_Z(ctypes.byref(st), _ptr(Z))
        return Z

    def kbatch(self):
        """(m [P_F,3] int32, c [P_F] with c_p = S/(P_F |k_p|^2), S)."""
        m = np.zeros((self.P_F, 3), dtype=np.int32)
        c = np.zeros(self.P_F)
        st = self._c()
        S = lib().orc_kbatch(ctypes.byref(st), _ptr(m), _ptr(c))
        return m, c, float(S)

    def kvec(self, m):
        return 2.0 * np.pi * np.asarray(m, dtype=np.float64) / self.box

    def enumerated_modes(self, m_max):
        """All m != 0 with |m_d| <= m_max and weight c = Fhat(k) (Eq. (Long))."""
        r = np.arange(-m_max, m_max + 1)
        mm = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
        mm = mm[np.any(mm != 0, axis=1)].astype(np.int32)
        k2 = (self.kvec(mm) ** 2).sum(1)
        return np.ascontiguousarray(mm), self.fhat(k2)

    def rho(self, m):
        m = np.ascontiguousarray(m, dtype=np.int32).reshape(-1, 3)
        out = np.zeros((m.shape[0], 2))
        st = self._c()
        lib().orc_rho(ctypes.byref(st), m.shape[0], _ptr(m), _ptr(out))
        return out

    def far(self, m, c, rho=None, sel=None):
        """Far-field force of ``sel`` and U_F* for modes m with weights c."""
        m = np.ascontiguousarray(m, dtype=np.int32).reshape(-1, 3)
        c = np.ascontiguousarray(c, dtype=np.float64)
        if rho is None:
            rho = self.rho(m)
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        sel = np.arange(self.n, dtype=np.int64) if sel is None else np.ascontiguousarray(sel, dtype=np.int64)
        F = np.zeros((sel.size, 3))
        U = np.zeros(1)
        st = self._c()
        lib().orc_far(ctypes.byref(st), m.shape[0], _ptr(m), _ptr(c), _ptr(rho), _ptr(sel), sel.size,
                      _ptr(F), _ptr(U))
        return F, float(U[0])

    def self_energy(self):
        st = self._c()
        return float(lib().orc_self_energy(ctypes.byref(st)))

    # ---- full force evaluation ----------------------------------------------
    def forces(self, sel=None, energy=False, kmodes=None, all_shell=False):
        """IRBSOG force F* = F_core + F*_shell - F^corr + F*_F (Sec. 2.2).

        ``kmodes=(m, c)`` replaces the sampled k-batch (enumeration mode).
        Returns a dict with total F (of ``sel``), near (uncorrected), far, Fcorr
        and, if ``energy``, [U_N, U_F*, U_self, U_total] and the virial [6]
        (xx, yy, zz, xy, xz, yz) W = W_N + W_F* of the same estimators (F^corr,
        not a pair force, has none).
        """
        allsel = np.arange(self.n, dtype=np.int64)
        Fn_all, En, Wn = self.near(allsel, all_shell=all_shell, energy=True, virial=True)
        Fcorr = Fn_all.mean(axis=0)
        if kmodes is None:
            m, c, S = self.kbatch()
        else:
            m, c = kmodes
            S = None
        rho = self.rho(m)
        sel_ = allsel if sel is None else np.asarray(sel, dtype=np.int64)
        Ff, Uf = self.far(m, c, rho, sel_)
        Fn = Fn_all[sel_]
        out = dict(F=Fn - Fcorr + Ff, near=Fn, far=Ff, Fcorr=Fcorr, m=m, c=c, S=S, rho=rho)
        if energy:
            UN = float(En.sum())
            Us = self.self_energy()
            out["energy"] = np.array([UN, Uf, Us, UN + Uf - Us])
            out["virial"] = Wn.sum(0) + self.far_virial(m, c, rho)
            out["virial_near"] = Wn.sum(0)
        return out

    # ---- integrators (Sec. 2.3) ----------------------------------------------
    def gaussian_noise(self, step):
        """Langevin noise xi[n,3]: Box-Muller on Philox stream 2, block 0."""
        w = draw(self.seed, step, np.arange(self.n, dtype=np.uint32), 2, 0).astype(np.float64)
        u = (w + 0.5) * 2.0 ** -32
        r1 = np.sqrt(-2.0 * np.log(u[:, 0]))
        r2 = np.sqrt(-2.0 * np.log(u[:, 2]))
        return np.stack([r1 * np.cos(2.0 * np.pi * u[:, 1]), r1 * np.sin(2.0 * np.pi * u[:, 1]),
                         r2 * np.cos(2.0 * np.pi * u[:, 3])], axis=1)

    def kinetic2(self, vel):
        """sum_i m_i v_i^2 in eV."""
        return float((self.mass[self.species][:, None] * vel ** 2).sum() / FCONV)

    def kinetic_tensor(self, vel):
        """K_ab = sum_i m_i v_ia v_ib in eV, (xx, yy, zz, xy, xz, yz): the velocity
        term of the stress whose xy component enters the Green-Kubo viscosity
        of Sec. 3 (S = K + W with the virial W)."""
        v = np.asarray(vel, dtype=np.float64).reshape(-1, 3)
        m = self.mass[self.species]
        out = np.empty(6)
        for c, (a, b) in enumerate(((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))):
            out[c] = float(np.sum(m * v[:, a] * v[:, b])) / FCONV
        return out

    def run(self, vel, nsteps, dt, integrator=INTEGRATOR_LANGEVIN_BAOAB, T=1200.0, gamma=1.0,
            F=None, tdamp=0.1, nh_chain=3, kmodes=None, all_shell=False):
        """Advance (pos, vel) by ``nsteps``; returns (vel, F).  Forces at step s use
        RNG step index s; the Langevin O-step of the step s -> s+1 uses index s+1.
        ``gamma`` is the collision rate gamma/m in 1/ps (same for all species);
        Nose-Hoover: chain of ``nh_chain`` with time constant ``tdamp`` [ps], a
        half step before the first half kick and after the second.  ``kmodes`` /
        ``all_shell`` as in :meth:`forces` (the deterministic force)."""
        vel = np.array(vel, dtype=np.float64).reshape(-1, 3)
        minv = (FCONV / self.mass[self.species])[:, None]
        if F is None:
            F = self.forces(kmodes=kmodes, all_shell=all_shell)["F"]
        c1 = np.exp(-gamma * dt)
        sig = np.sqrt((1.0 - c1 * c1) * KB * T * FCONV / self.mass[self.species])[:, None]
        if integrator == INTEGRATOR_NOSE_HOOVER and getattr(self, "chain", None) is None:
            self.chain = NHChain(nh_chain, T, tdamp, 3 * self.n - 3)
        for _ in range(nsteps):
            nxt = self.step + 1
            if integrator == INTEGRATOR_NOSE_HOOVER:
                vel = vel * self.chain.half_step(self.kinetic2(vel), dt)
            vel = vel + 0.5 * dt * F * minv
            if integrator == INTEGRATOR_LANGEVIN_BAOAB:
                self.pos = self.pos + 0.5 * dt * vel
                vel = c1 * vel + sig * self.gaussian_noise(nxt)
                self.pos = self.pos + 0.5 * dt * vel
            else:
                self.pos = self.pos + dt * vel
            self.step = nxt
            if self.list_every > 0 and nxt % self.list_every == 0:
                self.build_pos = self.pos.copy()
            elif self.list_every < 0 and self.build_pos is not None:
                d = self.pos - self.build_pos
                d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
                if d2.max() > self.displacement_limit2():
                    self.build_pos = self.pos.copy()
                    self.builds += 1
            F = self.forces(kmodes=kmodes, all_shell=all_shell)["F"]
            vel = vel + 0.5 * dt * F * minv
            if integrator == INTEGRATOR_NOSE_HOOVER:
                vel = vel * self.chain.half_step(self.kinetic2(vel), dt)
        return vel, F

