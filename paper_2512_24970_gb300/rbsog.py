"""ctypes binding of ``librbsog.so`` (the C ABI declared in ``include/rbsog.h``).

Argument marshalling only: every stage of the force evaluation and MD step
runs in the library's CUDA kernels.  Host arrays are numpy (``ptr_kind`` =
HOST); device arrays are torch CUDA tensors (``ptr_kind`` = DEVICE), used for
device memory and streams only.  If the library has not been built, loading
raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os

import numpy as np

from . import build as _build

FP64 = 0
MIXED = 1
NVE_VV = 0
LANGEVIN_BAOAB = 1
NOSE_HOOVER = 2
PTR_HOST = 0
PTR_DEVICE = 1

MAX_PR = 64

ERRORS = {
    -1: "RBSOG_E_INVAL", -2: "RBSOG_E_NONNEUTRAL", -3: "RBSOG_E_BOX_TOO_SMALL",
    -4: "RBSOG_E_CAP_OVERFLOW", -5: "RBSOG_E_CUDA", -6: "RBSOG_E_TIMEOUT",
    -7: "RBSOG_E_NO_SOG_ROOT", -8: "RBSOG_E_NO_SYSTEM", -9: "RBSOG_E_SKIN",
}
MAX_CORE = 64
LISTS_AUTO = -1   # list_every: rebuild kept lists when an atom has moved by skin/2
MAX_KEPT = 512

EXPORTS = [
    "rbsog_create", "rbsog_destroy", "rbsog_set_system", "rbsog_set_velocities",
    "rbsog_compute_forces", "rbsog_step", "rbsog_get_state", "rbsog_set_state", "rbsog_sync",
    "rbsog_get_sog", "rbsog_set_core_radii", "rbsog_get_list_builds", "rbsog_get_thermostat", "rbsog_set_thermostat", "rbsog_get_kinetic_tensor",
    "rbsog_get_list_origin", "rbsog_set_list_origin", "rbsog_move_atoms", "rbsog_forces_at", "rbsog_debug_get_lists", "rbsog_debug_get_kept_lists", "rbsog_debug_get_kept_batch_used", "rbsog_debug_kept_b16", "rbsog_debug_get_kbatch", "rbsog_debug_set_kbatch",
    "rbsog_debug_get_parts", "rbsog_debug_set_whole_shell", "rbsog_debug_sincos", "rbsog_set_profiling",
    "rbsog_get_stage_times", "rbsog_get_stage_marks", "rbsog_last_error", "rbsog_structure_factor_static",
    "rbsog_ensemble_create", "rbsog_ensemble_destroy", "rbsog_ensemble_add", "rbsog_ensemble_replica",
    "rbsog_ensemble_step", "rbsog_ensemble_sync", "rbsog_ensemble_last_error",
    "rbsog_set_schedule", "rbsog_get_schedule", "rbsog_probe_peak",
    "rbsog_ensemble_set_mode", "rbsog_ensemble_get_mode", "rbsog_ensemble_set_groups",
]
ENSEMBLE_PACKED, ENSEMBLE_GRAPHS = 0, 1
PROBE_FP32, PROBE_FP32X2, PROBE_FP64, PROBE_IMAD = 0, 1, 2, 3
SF_STATIC_PMAX = 1024
NSTAGE = 9
# stages of rbsog_get_stage_times: integrator + histograms, binning, near field, the far-field
# branch on the side stream (k-batch, structure factor, its reduction, far force), F^corr, the
# closing total force + half kick after the branches join, the whole evaluation, and inside the
# far-field branch the structure-factor kernel and the far-force kernel alone
STAGES = ["prepare", "bin", "near", "far", "corr", "finish", "total", "rho", "farforce"]
NMARK = 12
# marks of rbsog_get_stage_marks (time from the start of the evaluation)
MARKS = ["start", "prepared", "binned", "near_done", "corr_done", "joined", "end",
         "side_start", "rho_start", "rho_done", "reduce_done", "far_done"]


class RbsogError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [
        ("b", ctypes.c_double), ("M", ctypes.c_int32), ("s", ctypes.c_double), ("w0", ctypes.c_double),
        ("r_core", ctypes.c_double), ("r_shell", ctypes.c_double),
        ("P_R", ctypes.c_int32), ("P_F", ctypes.c_int32), ("seed", ctypes.c_uint64),
        ("precision", ctypes.c_int32), ("integrator", ctypes.c_int32),
        ("dt", ctypes.c_double), ("T", ctypes.c_double), ("gamma", ctypes.c_double),
        ("list_every", ctypes.c_int32), ("skin", ctypes.c_double),
        ("tdamp", ctypes.c_double), ("nh_chain", ctypes.c_int32),
    ]


class Schedule(ctypes.Structure):
    """Launch shapes of the mixed far field (``rbsog_schedule``)."""
    _fields_ = [("rho_variant", ctypes.c_int32), ("rho_blocks_per_sm", ctypes.c_int32),
                ("far_atoms_per_thread", ctypes.c_int32), ("far_segments", ctypes.c_int32),
                ("far_packed", ctypes.c_int32), ("near_blocks_per_sm", ctypes.c_int32),
                ("rho_tile_atoms", ctypes.c_int32), ("near_wide", ctypes.c_int32),
                ("rho_reduce", ctypes.c_int32)]

    def as_tuple(self):
        return (self.rho_variant, self.rho_blocks_per_sm, self.far_atoms_per_thread, self.far_segments,
                self.far_packed, self.near_blocks_per_sm, self.rho_tile_atoms, self.near_wide, self.rho_reduce)


@dataclasses.dataclass
class MethodParams:
    b: float = 1.3
    M: int = 64
    s: float = 0.0          # <= 0: solve with w0 for C^1 at r_shell
    w0: float = 0.0
    r_core: float = 6.0
    r_shell: float = 12.0
    P_R: int = 20
    P_F: int = 500
    seed: int = 1
    precision: int = MIXED
    integrator: int = LANGEVIN_BAOAB
    dt: float = 0.001
    T: float = 1200.0
    gamma: float = 1.0
    list_every: int = 0     # 0: per-step lists; n >= 1: kept lists rebuilt every n steps; -1: when needed
    skin: float = 0.0       # Verlet skin of kept lists [A]
    tdamp: float = 0.1      # Nose-Hoover time constant [ps]
    nh_chain: int = 3       # Nose-Hoover chain length

    def c(self):
        p = Params()
        for f in dataclasses.fields(self):
            setattr(p, f.name, getattr(self, f.name))
        return p


_lib = None


def lib_path() -> str:
    return _build.LIB


def load():
    """Load librbsog.so (built by ``paper_2512_24970_gb300.build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError("librbsog.so is not built (%s): run paper_2512_24970_gb300.build.build()" % path)
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    I = ctypes.c_int
    I32, I64 = ctypes.c_int32, ctypes.c_int64
    L.rbsog_create.argtypes = [ctypes.POINTER(P), I, P]
    L.rbsog_destroy.argtypes = [P]
    L.rbsog_destroy.restype = None
    L.rbsog_set_system.argtypes = [P, I64, P, P, I32, P, P, P, P, ctypes.POINTER(Params), I]
    L.rbsog_set_velocities.argtypes = [P, P, I]
    L.rbsog_compute_forces.argtypes = [P, P, P, P, I]
    L.rbsog_step.argtypes = [P, I64]
    L.rbsog_get_state.argtypes = [P, P, P, P, I]
    L.rbsog_set_state.argtypes = [P, P, P, I64, I]
    L.rbsog_sync.argtypes = [P]
    L.rbsog_get_sog.argtypes = [P, P, P, P]
    L.rbsog_get_list_builds.argtypes = [P, P]
    L.rbsog_set_core_radii.argtypes = [P, P]
    L.rbsog_get_thermostat.argtypes = [P, P, P]
    L.rbsog_get_kinetic_tensor.argtypes = [P, P, I]
    L.rbsog_get_list_origin.argtypes = [P, P, I]
    L.rbsog_move_atoms.argtypes = [P, P, I64, I]
    L.rbsog_forces_at.argtypes = [P, P, I64, P, I]
    L.rbsog_set_list_origin.argtypes = [P, P, I]
    L.rbsog_set_thermostat.argtypes = [P, P, P]
    L.rbsog_debug_get_lists.argtypes = [P, P, I64, I32, I32, P, P, P, P, P, P, P]
    L.rbsog_debug_get_kept_lists.argtypes = [P, P, I64, I32, I32, P, P, P, P, P, P, P]
    L.rbsog_debug_get_kept_batch_used.argtypes = [P, P, I64, P]
    L.rbsog_debug_kept_b16.argtypes = [P, I32, P]
    L.rbsog_debug_get_kbatch.argtypes = [P, P, P]
    L.rbsog_debug_set_kbatch.argtypes = [P, I32, P, P]
    L.rbsog_debug_get_parts.argtypes = [P, P, P, P, P]
    L.rbsog_debug_set_whole_shell.argtypes = [P, I]
    L.rbsog_debug_sincos.argtypes = [P, I64, P, P, P]
    L.rbsog_set_profiling.argtypes = [P, I]
    L.rbsog_get_stage_times.argtypes = [P, P, I32]
    L.rbsog_get_stage_marks.argtypes = [P, P, I32]
    L.rbsog_structure_factor_static.argtypes = [P, I32, P, P]
    L.rbsog_ensemble_create.argtypes = [ctypes.POINTER(P), I, P, I32]
    L.rbsog_ensemble_destroy.argtypes = [P]
    L.rbsog_ensemble_destroy.restype = None
    L.rbsog_ensemble_add.argtypes = [P, I64, P, P, I32, P, P, P, P, ctypes.POINTER(Params), I,
                                     ctypes.POINTER(I32)]
    L.rbsog_ensemble_replica.argtypes = [P, I32]
    L.rbsog_ensemble_replica.restype = P
    L.rbsog_ensemble_step.argtypes = [P, I64]
    L.rbsog_ensemble_sync.argtypes = [P]
    L.rbsog_ensemble_set_mode.argtypes = [P, I32]
    L.rbsog_ensemble_get_mode.argtypes = [P, ctypes.POINTER(I32)]
    L.rbsog_ensemble_set_groups.argtypes = [P, I32]
    L.rbsog_ensemble_last_error.argtypes = [P]
    L.rbsog_ensemble_last_error.restype = ctypes.c_char_p
    L.rbsog_last_error.argtypes = [P]
    L.rbsog_last_error.restype = ctypes.c_char_p
    L.rbsog_probe_peak.argtypes = [I, I, ctypes.POINTER(ctypes.c_double)]
    L.rbsog_set_schedule.argtypes = [P, ctypes.POINTER(Schedule)]
    L.rbsog_get_schedule.argtypes = [P, ctypes.POINTER(Schedule)]
    _lib = L
    return L


def probe_peak(device: int, kind: int) -> float:
    """Measured multiply-add lane operations per second of one pipe (``rbsog_probe_peak``)."""
    L = load()
    v = ctypes.c_double()
    rc = L.rbsog_probe_peak(device, kind, ctypes.byref(v))
    if rc != 0:
        raise RbsogError(rc, "rbsog_probe_peak failed")
    return v.value


def _np_ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _ptr_kind(a):
    """(pointer, kind) of a numpy array (HOST) or a torch CUDA tensor (DEVICE)."""
    if a is None:
        return None, PTR_HOST
    if isinstance(a, np.ndarray):
        return ctypes.c_void_p(a.ctypes.data), PTR_HOST
    # torch tensor
    if a.is_cuda:
        return ctypes.c_void_p(a.data_ptr()), PTR_DEVICE
    return ctypes.c_void_p(a.data_ptr()), PTR_HOST


class Context:
    """One simulation context on one GPU (a thin owner of ``rbsog_ctx*``)."""

    def __init__(self, device: int = 0, stream: int | None = None):
        """``stream``: a cudaStream_t handle (e.g. ``torch.cuda.Stream().cuda_stream``)
        the library runs on; None/0 = a library-owned stream ordered with the
        legacy default stream."""
        self._L = load()
        if stream is None:
            stream = 0
        h = ctypes.c_void_p()
        rc = self._L.rbsog_create(ctypes.byref(h), device, ctypes.c_void_p(stream))
        if rc != 0:
            raise RbsogError(rc, "rbsog_create failed")
        self.h = h
        self.n = 0
        self.params = None

    def close(self):
        if getattr(self, "h", None):
            if getattr(self, "_owned", True):       # replica views belong to their ensemble
                self._L.rbsog_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, rc):
        if rc != 0:
            raise RbsogError(rc, self._L.rbsog_last_error(self.h).decode())

    # ------------------------------------------------------------------
    def set_system(self, pos, species, charge, mass, bmh, box, params: MethodParams):
        pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
        species = np.ascontiguousarray(species, dtype=np.int32)
        charge = np.ascontiguousarray(charge, dtype=np.float64)
        mass = np.ascontiguousarray(mass, dtype=np.float64)
        bmh = np.ascontiguousarray(bmh, dtype=np.float64)
        box = np.ascontiguousarray(box, dtype=np.float64)
        p = params.c()
        self._ck(self._L.rbsog_set_system(self.h, pos.shape[0], _np_ptr(pos), _np_ptr(species), charge.size,
                                          _np_ptr(charge), _np_ptr(mass), _np_ptr(bmh), _np_ptr(box),
                                          ctypes.byref(p), PTR_HOST))
        self.n = pos.shape[0]
        self.params = params
        return self

    def set_workload(self, w, params: MethodParams):
        self.set_system(w.pos, w.species, w.charge, w.mass, w.bmh, w.box, params)
        if w.vel is not None:
            self.set_velocities(w.vel)
        return self

    def set_velocities(self, vel):
        if isinstance(vel, np.ndarray):
            vel = np.ascontiguousarray(vel, dtype=np.float64)
        ptr, kind = _ptr_kind(vel)
        self._ck(self._L.rbsog_set_velocities(self.h, ptr, kind))

    def compute_forces(self, forces=None, energy=False, virial=False):
        """Forces [n,3] FP64 (numpy unless ``forces`` is a CUDA tensor to fill)
        and, if asked, the energy 4-vector and the virial 6-vector
        (xx, yy, zz, xy, xz, yz): returns F, (F, E), (F, W) or (F, E, W)."""
        out = np.zeros((self.n, 3)) if forces is None else forces
        ptr, kind = _ptr_kind(out)
        if (energy or virial) and kind == PTR_DEVICE:
            raise ValueError("energy or virial output with device forces: call again with host arrays")
        e = np.zeros(4) if energy else None
        wv = np.zeros(6) if virial else None
        self._ck(self._L.rbsog_compute_forces(self.h, ptr, _np_ptr(e), _np_ptr(wv), kind))
        res = (out,) + ((e,) if energy else ()) + ((wv,) if virial else ())
        return res if len(res) > 1 else out

    def step(self, nsteps: int):
        self._ck(self._L.rbsog_step(self.h, int(nsteps)))

    def get_state(self, pos=None, vel=None):
        pos = np.zeros((self.n, 3)) if pos is None else pos
        vel = np.zeros((self.n, 3)) if vel is None else vel
        pp, kind = _ptr_kind(pos)
        vp, _ = _ptr_kind(vel)
        st = ctypes.c_int64()
        self._ck(self._L.rbsog_get_state(self.h, pp, vp, ctypes.byref(st), kind))
        return pos, vel, st.value

    def set_state(self, pos=None, vel=None, step=0):
        if isinstance(pos, np.ndarray):
            pos = np.ascontiguousarray(pos, dtype=np.float64)
        if isinstance(vel, np.ndarray):
            vel = np.ascontiguousarray(vel, dtype=np.float64)
        pp, kind = _ptr_kind(pos)
        vp, kind2 = _ptr_kind(vel)
        if pos is None:
            kind = kind2
        self._ck(self._L.rbsog_set_state(self.h, pp, vp, int(step), kind))

    def sync(self):
        self._ck(self._L.rbsog_sync(self.h))

    def sog(self):
        M = self.params.M
        s = ctypes.c_double()
        S = ctypes.c_double()
        w = np.zeros(M + 1)
        self._ck(self._L.rbsog_get_sog(self.h, ctypes.byref(s), _np_ptr(w), ctypes.byref(S)))
        return s.value, w, S.value

    def move_atoms(self, pos, step):
        """Positions [n, 3] (numpy or CUDA tensor) and step counter, keeping the
        velocities and the kept lists (rebuilt by the device check when needed)."""
        if isinstance(pos, np.ndarray):
            pos = np.ascontiguousarray(pos, dtype=np.float64)
        pp, kind = _ptr_kind(pos)
        self._ck(self._L.rbsog_move_atoms(self.h, pp, int(step), kind))

    def forces_at(self, pos, step, forces=None):
        """move_atoms(pos, step) and the force-only compute_forces in one call
        (one synchronization for host arrays): forces [n, 3] FP64 at the
        positions pos [n, 3].  pos and forces both numpy (host) or both CUDA
        tensors of this context's device (asynchronous on its stream)."""
        if isinstance(pos, np.ndarray):
            pos = np.ascontiguousarray(pos, dtype=np.float64)
        out = np.zeros((self.n, 3)) if forces is None else forces
        for a in (pos, out):
            n3 = a.size if isinstance(a, np.ndarray) else a.numel()
            f64 = a.dtype == np.float64 if isinstance(a, np.ndarray) else str(a.dtype) == "torch.float64"
            contig = a.flags["C_CONTIGUOUS"] if isinstance(a, np.ndarray) else a.is_contiguous()
            if n3 != 3 * self.n or not f64 or not contig:
                raise ValueError("pos and forces must be contiguous float64 arrays of shape [n, 3]")
        pp, kind = _ptr_kind(pos)
        fp, fkind = _ptr_kind(out)
        if fkind != kind:
            raise ValueError("pos and forces must both be host arrays or both device tensors")
        self._ck(self._L.rbsog_forces_at(self.h, pp, int(step), fp, kind))
        return out

    def list_origin(self):
        """Kept lists: the positions [n, 3] of their last build (with get_state, what a restore needs)."""
        out = np.zeros((self.n, 3))
        self._ck(self._L.rbsog_get_list_origin(self.h, _np_ptr(out), PTR_HOST))
        return out

    def set_list_origin(self, pos_b):
        """Kept lists: build the next evaluation's lists from the positions pos_b [n, 3]."""
        a = np.ascontiguousarray(pos_b, dtype=np.float64).reshape(-1, 3)
        self._ck(self._L.rbsog_set_list_origin(self.h, _np_ptr(a), PTR_HOST))

    def kinetic_tensor(self, out=None):
        """K_ab = sum_i m_i v_ia v_ib [eV], (xx, yy, zz, xy, xz, yz), of the current
        velocities; with the virial W of compute_forces the stress is S = K + W.
        ``out``: a CUDA float64 tensor of 6 to receive it on the device (no sync)."""
        if out is not None:
            self._ck(self._L.rbsog_get_kinetic_tensor(self.h, ctypes.c_void_p(out.data_ptr()), PTR_DEVICE))
            return out
        K = np.zeros(6)
        self._ck(self._L.rbsog_get_kinetic_tensor(self.h, _np_ptr(K), PTR_HOST))
        return K

    def thermostat(self):
        """Nose-Hoover chain (eta, v_eta) between steps."""
        M = self.params.nh_chain
        eta, ve = np.zeros(M), np.zeros(M)
        self._ck(self._L.rbsog_get_thermostat(self.h, _np_ptr(eta), _np_ptr(ve)))
        return eta, ve

    def set_thermostat(self, eta, v_eta):
        eta = np.ascontiguousarray(eta, dtype=np.float64)
        ve = np.ascontiguousarray(v_eta, dtype=np.float64)
        self._ck(self._L.rbsog_set_thermostat(self.h, _np_ptr(eta), _np_ptr(ve)))

    def checkpoint(self, path=None):
        """What a bit-for-bit restart needs: positions, velocities and step
        counter, the kept lists' build positions (kept lists, once evaluated)
        and the Nose-Hoover chain (Nose-Hoover runs).  Returns a dict; with
        ``path`` also writes it with numpy.savez."""
        pos, vel, step = self.get_state()
        ck = {"pos": pos, "vel": vel, "step": np.int64(step)}
        if self.params.list_every != 0:
            try:
                ck["list_origin"] = self.list_origin()
            except RbsogError:          # no lists yet: a restore builds at the restored positions, as this would
                pass
        if self.params.integrator == NOSE_HOOVER:
            ck["nh_eta"], ck["nh_v"] = self.thermostat()
        if path is not None:
            np.savez(path, **ck)
        return ck

    def restore(self, ck):
        """Resume from checkpoint() (its dict or the .npz it wrote) on a context
        with the same system and parameters."""
        if not isinstance(ck, dict):
            with np.load(ck) as f:
                ck = {k: f[k] for k in f.files}
        self.set_state(ck["pos"], ck["vel"], int(ck["step"]))
        if "list_origin" in ck:
            self.set_list_origin(ck["list_origin"])
        if "nh_eta" in ck:
            self.set_thermostat(ck["nh_eta"], ck["nh_v"])

    def set_core_radii(self, r_core_pair=None):
        """Species-dependent core radii [ns][ns] (None: the single r_core)."""
        t = None if r_core_pair is None else np.ascontiguousarray(r_core_pair, dtype=np.float64)
        self._ck(self._L.rbsog_set_core_radii(self.h, _np_ptr(t)))

    def list_builds(self) -> int:
        """Builds of the kept random batch lists since set_system."""
        b = np.zeros(1, dtype=np.int64)
        self._ck(self._L.rbsog_get_list_builds(self.h, _np_ptr(b)))
        return int(b[0])

    # ---- parity hooks -----------------------------------------------------
    def debug_lists(self, sel, cap_core=128, cap_shell=512, batch=True):
        sel = np.ascontiguousarray(sel, dtype=np.int64)
        k = sel.size
        core = np.full((k, cap_core), -1, dtype=np.int32)
        ncore = np.zeros(k, dtype=np.int32)
        shell = np.full((k, cap_shell), -1, dtype=np.int32)
        nshell = np.zeros(k, dtype=np.int32)
        PR = self.params.P_R
        bt = np.full((k, PR), -1, dtype=np.int32) if batch else None
        nb = np.zeros(k, dtype=np.int32) if batch else None
        wt = np.zeros(k) if batch else None
        self._ck(self._L.rbsog_debug_get_lists(self.h, _np_ptr(sel), k, cap_core, cap_shell, _np_ptr(core),
                                               _np_ptr(ncore), _np_ptr(shell), _np_ptr(nshell), _np_ptr(bt),
                                               _np_ptr(nb), _np_ptr(wt)))
        out = dict(core=core, ncore=ncore, shell=shell, nshell=nshell)
        if batch:
            out.update(batch=bt, nbatch=nb, weight=wt)
        return out

    def debug_kept_lists(self, sel, cap_a=MAX_CORE, cap_b=MAX_KEPT, batch=True):
        """Kept lists A, B (caller ids, canonical order of the build) and the batch of ``sel``."""
        sel = np.ascontiguousarray(sel, dtype=np.int64)
        k = sel.size
        A = np.full((k, cap_a), -1, dtype=np.int32)
        nA = np.zeros(k, dtype=np.int32)
        B = np.full((k, cap_b), -1, dtype=np.int32)
        nB = np.zeros(k, dtype=np.int32)
        PR = self.params.P_R
        bt = np.full((k, PR), -1, dtype=np.int32) if batch else None
        nb = np.zeros(k, dtype=np.int32) if batch else None
        wt = np.zeros(k) if batch else None
        self._ck(self._L.rbsog_debug_get_kept_lists(self.h, _np_ptr(sel), k, cap_a, cap_b, _np_ptr(A), _np_ptr(nA),
                                                    _np_ptr(B), _np_ptr(nB), _np_ptr(bt), _np_ptr(nb), _np_ptr(wt)))
        out = dict(A=A, nA=nA, B=B, nB=nB)
        if batch:
            out.update(batch=bt, nbatch=nb, weight=wt)
        return out

    def debug_kept_batch_used(self, sel):
        """The shell batch the last evaluation's pair sums read (caller ids, draw order; -1 rows: all of B)."""
        sel = np.ascontiguousarray(sel, dtype=np.int64)
        bt = np.full((sel.size, self.params.P_R), -1, dtype=np.int32)
        self._ck(self._L.rbsog_debug_get_kept_batch_used(self.h, _np_ptr(sel), sel.size, _np_ptr(bt)))
        return bt

    def debug_kept_b16(self, force_wide=False):
        """Read B's 32-bit rows always (force_wide) or the 16-bit ones where they fit; returns
        whether the last build's offsets all fit 16 bits."""
        f = np.zeros(1, dtype=np.int32)
        self._ck(self._L.rbsog_debug_kept_b16(self.h, 1 if force_wide else 0, _np_ptr(f)))
        return bool(f[0])

    def debug_kbatch(self, P=None):
        P = self.params.P_F if P is None else P
        m = np.zeros((P, 3), dtype=np.int32)
        c = np.zeros(P)
        self._ck(self._L.rbsog_debug_get_kbatch(self.h, _np_ptr(m), _np_ptr(c)))
        return m, c

    def debug_set_kbatch(self, m=None, c=None):
        if m is None:
            self._ck(self._L.rbsog_debug_set_kbatch(self.h, 0, None, None))
            return
        m = np.ascontiguousarray(m, dtype=np.int32).reshape(-1, 3)
        c = np.ascontiguousarray(c, dtype=np.float64)
        self._ck(self._L.rbsog_debug_set_kbatch(self.h, m.shape[0], _np_ptr(m), _np_ptr(c)))

    def debug_parts(self, P=None):
        P = self.params.P_F if P is None else P
        near = np.zeros((self.n, 3))
        far = np.zeros((self.n, 3))
        fc = np.zeros(3)
        rho = np.zeros((P, 2))
        self._ck(self._L.rbsog_debug_get_parts(self.h, _np_ptr(near), _np_ptr(far), _np_ptr(fc), _np_ptr(rho)))
        return dict(near=near, far=far, Fcorr=fc, rho=rho)

    def set_schedule(self, rho_variant: int, rho_blocks_per_sm: int, far_atoms_per_thread: int,
                     far_segments: int, far_packed: int = 1, near_blocks_per_sm: int = 0,
                     rho_tile_atoms: int = 0, near_wide: int = 0, rho_reduce: int = 0):
        """Launch shapes of the mixed far field and the kept near field (the step
        graph is captured again)."""
        q = Schedule(rho_variant, rho_blocks_per_sm, far_atoms_per_thread, far_segments, far_packed,
                     near_blocks_per_sm, rho_tile_atoms, near_wide, rho_reduce)
        self._ck(self._L.rbsog_set_schedule(self.h, ctypes.byref(q)))

    def schedule(self):
        q = Schedule()
        self._ck(self._L.rbsog_get_schedule(self.h, ctypes.byref(q)))
        return q.as_tuple()

    def set_profiling(self, on: bool):
        self._ck(self._L.rbsog_set_profiling(self.h, 1 if on else 0))

    def stage_times(self):
        ms = np.zeros(NSTAGE, dtype=np.float32)
        self._ck(self._L.rbsog_get_stage_times(self.h, _np_ptr(ms), NSTAGE))
        return ms

    def stage_marks(self):
        """Times [ms] of the stage marks (``MARKS``) of the latest evaluation, from its start."""
        ms = np.zeros(NMARK, dtype=np.float32)
        self._ck(self._L.rbsog_get_stage_marks(self.h, _np_ptr(ms), NMARK))
        return ms

    def debug_sincos(self, th):
        th = np.ascontiguousarray(th, dtype=np.uint32)
        s = np.zeros(th.size, dtype=np.float32)
        c = np.zeros(th.size, dtype=np.float32)
        self._ck(self._L.rbsog_debug_sincos(self.h, th.size, _np_ptr(th), _np_ptr(s), _np_ptr(c)))
        return s, c

    def structure_factor_static(self, m, rho=None):
        """rho(k_p) [P, 2] FP64 of the current positions for modes ``m`` [P, 3]
        (torch int32 CUDA tensor), through the allocation-free entry point;
        ``rho`` (torch float64 CUDA tensor) is written and returned."""
        import torch
        if rho is None:
            rho = torch.empty((m.shape[0], 2), dtype=torch.float64, device=m.device)
        assert m.is_cuda and m.dtype == torch.int32 and m.is_contiguous()
        assert rho.is_cuda and rho.dtype == torch.float64 and rho.is_contiguous()
        self._ck(self._L.rbsog_structure_factor_static(self.h, m.shape[0], ctypes.c_void_p(m.data_ptr()),
                                                        ctypes.c_void_p(rho.data_ptr())))
        return rho

    def debug_whole_shell(self, flag: bool):
        self._ck(self._L.rbsog_debug_set_whole_shell(self.h, 1 if flag else 0))


class Ensemble:
    """Independent replicas of uneven size stepped together on one GPU
    (``rbsog_ensemble_*``): each replica is a full context on its own stream."""

    def __init__(self, device: int = 0, stream: int | None = None, max_replicas: int = 64):
        self._L = load()
        h = ctypes.c_void_p()
        rc = self._L.rbsog_ensemble_create(ctypes.byref(h), device, ctypes.c_void_p(stream or 0), max_replicas)
        if rc != 0:
            raise RbsogError(rc, "rbsog_ensemble_create failed")
        self.h = h
        self.replicas = []

    def _ck(self, rc):
        if rc != 0:
            raise RbsogError(rc, self._L.rbsog_ensemble_last_error(self.h).decode())

    def add(self, pos, species, charge, mass, bmh, box, params: MethodParams):
        """Add a replica (arguments as Context.set_system); returns its Context view."""
        pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
        species = np.ascontiguousarray(species, dtype=np.int32)
        charge = np.ascontiguousarray(charge, dtype=np.float64)
        mass = np.ascontiguousarray(mass, dtype=np.float64)
        bmh = np.ascontiguousarray(bmh, dtype=np.float64)
        box = np.ascontiguousarray(box, dtype=np.float64)
        prm = params.c()
        r = ctypes.c_int32()
        self._ck(self._L.rbsog_ensemble_add(self.h, pos.shape[0], _np_ptr(pos), _np_ptr(species), charge.size,
                                            _np_ptr(charge), _np_ptr(mass), _np_ptr(bmh), _np_ptr(box),
                                            ctypes.byref(prm), PTR_HOST, ctypes.byref(r)))
        ctx = Context.__new__(Context)      # a non-owning view of the replica's context
        ctx._L = self._L
        ctx.h = ctypes.c_void_p(self._L.rbsog_ensemble_replica(self.h, r.value))
        ctx.n = pos.shape[0]
        ctx.params = params
        ctx._owned = False
        self.replicas.append(ctx)
        return ctx

    def add_workload(self, w, params: MethodParams):
        return self.add(w.pos, w.species, w.charge, w.mass, w.bmh, w.box, params)

    def step(self, nsteps: int):
        self._ck(self._L.rbsog_ensemble_step(self.h, int(nsteps)))

    def set_mode(self, mode: int):
        """ENSEMBLE_PACKED (one launch per stage over all replicas, where they
        allow it) or ENSEMBLE_GRAPHS (the replicas' own step graphs as child
        nodes of one graph)."""
        self._ck(self._L.rbsog_ensemble_set_mode(self.h, int(mode)))

    def set_groups(self, groups: int):
        """Packed mode: replicas dealt into this many groups of about equal
        atoms, the groups' packed launches as parallel graph branches."""
        self._ck(self._L.rbsog_ensemble_set_groups(self.h, int(groups)))
        self._groups = int(groups)

    def used_mode(self) -> int:
        m = ctypes.c_int32()
        self._ck(self._L.rbsog_ensemble_get_mode(self.h, ctypes.byref(m)))
        return m.value

    def launch_kind(self):
        m = self.used_mode()
        if m == ENSEMBLE_PACKED:
            g = getattr(self, "_groups", 1)
            return ("packed: one CUDA graph per ensemble step; the replicas in %d group(s) of about equal atoms, "
                    "each stage of a group one kernel launch over its replicas' blocks, the groups as parallel "
                    "branches" % g)
        if m == ENSEMBLE_GRAPHS:
            return "one CUDA graph per ensemble step (every replica's step graph a child node)"
        return "not stepped yet"

    def sync(self):
        self._ck(self._L.rbsog_ensemble_sync(self.h))

    def close(self):
        if getattr(self, "h", None):
            for c in self.replicas:
                c.h = None
            self._L.rbsog_ensemble_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

