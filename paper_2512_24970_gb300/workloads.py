"""Seeded synthetic inputs: molten alkali-halide configurations.

This module holds none of the method's arithmetic.  It builds the inputs
that both the CUDA path and the FP64 oracle consume: rock-salt lattices with
Gaussian jitter, seed-shuffled cation species for mixtures, Maxwell-Boltzmann
velocities, and the BMH parameter tables printed in the paper (Table 1 for
NaCl, Table 3 for LiCl-NaCl).  Random numbers come from numpy's Philox bit
generator keyed by the workload seed.

Recipe (the paper's workloads are lattices of this shape):
  conventional rock-salt cell a = 6.3 Angstrom (8 ions, 0.0320 ions/A^3),
  cations on fcc sites, Cl- offset by (a/2, 0, 0), jitter sigma = 0.25 A per
  component, charges +-1 e, masses Li 6.941, Na 22.98977, Cl 35.453 amu.
"""
from __future__ import annotations

import dataclasses
import numpy as np

KB = 8.617333262e-5         # eV / K
FCONV = 9648.53321          # (eV/Angstrom)/amu -> Angstrom/ps^2

A_CELL = 6.3

# Table 1 (Tosi-Fumi NaCl): pairs Na-Na, Na-Cl, Cl-Cl; rows A [eV], sigma [A],
# C [eV A^6], D [eV A^8], rho [A].
_T1 = {
    ("Na", "Na"): (0.303, 2.340, 1.049, 0.499, 0.317),
    ("Na", "Cl"): (0.242, 2.755, 6.991, 8.676, 0.317),
    ("Cl", "Cl"): (0.182, 3.170, 72.40, 145.427, 0.317),
}
# Table 3 (LiCl-NaCl): same column order (A, sigma, C, D, rho).
_T3 = {
    ("Li", "Li"): (0.4225, 1.632, 0.045625, 0.01875, 0.3170),
    ("Li", "Na"): (0.334, 1.986, 0.218875, 0.0968, 0.3185),
    ("Na", "Na"): (0.2640625, 2.340, 1.05, 0.50, 0.3200),
    ("Li", "Cl"): (0.29046875, 2.401, 1.25, 1.50, 0.3215),
    ("Na", "Cl"): (0.21125, 2.755, 7.00, 8.6875, 0.3230),
    ("Cl", "Cl"): (0.1584375, 3.170, 71.328, 143.281, 0.3261),
}
MASS = {"Li": 6.941, "Na": 22.98977, "Cl": 35.453}
CHARGE = {"Li": 1.0, "Na": 1.0, "Cl": -1.0}


def bmh_table(names, table):
    """[ns][ns][5] array in ABI order (A, sigma, rho, C, D)."""
    ns = len(names)
    out = np.zeros((ns, ns, 5))
    for i, a in enumerate(names):
        for j, b in enumerate(names):
            key = (a, b) if (a, b) in table else (b, a)
            A, sig, C, D, rho = table[key]
            out[i, j] = (A, sig, rho, C, D)
    return out


def nacl_params():
    names = ["Na", "Cl"]
    return names, bmh_table(names, _T1)


def licl_nacl_params():
    names = ["Li", "Na", "Cl"]
    return names, bmh_table(names, _T3)


@dataclasses.dataclass
class Workload:
    name: str
    pos: np.ndarray        # [n,3] FP64
    species: np.ndarray    # [n] int32
    names: list
    charge: np.ndarray     # [ns]
    mass: np.ndarray       # [ns]
    bmh: np.ndarray        # [ns][ns][5]
    box: np.ndarray        # [3]
    seed: int
    vel: np.ndarray | None = None

    @property
    def n(self):
        return self.pos.shape[0]


def rock_salt(cells, a=A_CELL, jitter=0.25, seed=1, composition="NaCl", li_fraction=0.59):
    """Rock-salt lattice of cells=(nx,ny,nz) conventional cells with jitter.

    composition: "NaCl", "LiCl" or "LiCl-NaCl" (cations shuffled by seed with
    the given Li fraction of the cation sites).
    """
    nx, ny, nz = cells
    fcc = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]])
    cat = []
    an = []
    for iz in range(nz):
        for iy in range(ny):
            for ix in range(nx):
                o = np.array([ix, iy, iz], dtype=np.float64)
                cat.append((o + fcc) * a)
                an.append((o + fcc + np.array([.5, 0, 0])) * a)
    cat = np.concatenate(cat)
    an = np.concatenate(an)
    ncat = cat.shape[0]
    rng = np.random.Generator(np.random.Philox(seed))
    if composition == "NaCl":
        names, bmh = nacl_params()
        cat_sp = np.zeros(ncat, dtype=np.int32)
        cl = 1
    elif composition == "LiCl":
        names, bmh = licl_nacl_params()
        cat_sp = np.zeros(ncat, dtype=np.int32)
        cl = 2
    elif composition == "LiCl-NaCl":
        names, bmh = licl_nacl_params()
        nli = int(round(li_fraction * ncat))
        cat_sp = np.ones(ncat, dtype=np.int32)
        cat_sp[:nli] = 0
        cat_sp = rng.permutation(cat_sp).astype(np.int32)
        cl = 2
    else:
        raise ValueError(composition)
    pos = np.concatenate([cat, an])
    species = np.concatenate([cat_sp, np.full(an.shape[0], cl, dtype=np.int32)])
    pos = pos + rng.normal(0.0, jitter, size=pos.shape) if jitter > 0 else pos
    box = np.array([nx * a, ny * a, nz * a], dtype=np.float64)
    charge = np.array([CHARGE[s] for s in names])
    mass = np.array([MASS[s] for s in names])
    return Workload(name=f"{composition} {nx}x{ny}x{nz}", pos=np.ascontiguousarray(pos),
                    species=species, names=names, charge=charge, mass=mass, bmh=bmh,
                    box=box, seed=seed)


def maxwell_boltzmann(w: Workload, T, seed=None):
    """Velocities [n,3] in Angstrom/ps at temperature T, zero total momentum."""
    rng = np.random.Generator(np.random.Philox(1000 + (w.seed if seed is None else seed)))
    m = w.mass[w.species]
    v = rng.normal(size=(w.n, 3)) * np.sqrt(KB * T * FCONV / m)[:, None]
    p = (v * m[:, None]).sum(0) / m.sum()
    return v - p[None, :]


# --------------------------------------------------------------------------
# The five workload shapes (seeds 1..5).

@dataclasses.dataclass
class Config:
    key: str
    description: str
    cells: tuple
    composition: str
    seed: int
    P_R: int
    P_F: int
    T: float
    steps: int
    integrator: str        # "nve" | "langevin"
    list_every: int = -1   # kept random batch lists, rebuilt when an atom has moved by skin/2 ...
    skin: float = 1.0      # ... with this skin [A]
    gamma: float = 1.0     # Langevin friction [1/ps]


CONFIGS = {
    "nacl_1k": Config("nacl_1k", "molten NaCl N=1000, 5^3 cells, L=31.5 A, NVE dt=1 fs",
                      (5, 5, 5), "NaCl", 1, 20, 200, 1200.0, 100, "nve"),
    "nacl_64k": Config("nacl_64k", "molten NaCl N=64000, 20^3 cells, L=126 A, Langevin 1200 K dt=1 fs",
                       (20, 20, 20), "NaCl", 2, 20, 500, 1200.0, 1000, "langevin"),
    "liclnacl_216k": Config("liclnacl_216k", "LiCl-NaCl 59:41 N=216000, 30^3 cells, L=189 A, Langevin 1100 K",
                            (30, 30, 30), "LiCl-NaCl", 3, 30, 1000, 1100.0, 500, "langevin"),
    "nacl_1m": Config("nacl_1m", "molten NaCl N=1024000, 40x40x80 cells, 252x252x504 A, Langevin 1200 K",
                      (40, 40, 80), "NaCl", 4, 20, 1000, 1200.0, 200, "langevin"),
}


def make(key, **over):
    c = CONFIGS[key]
    w = rock_salt(c.cells, seed=c.seed, composition=c.composition)
    w.vel = maxwell_boltzmann(w, c.T)
    return w, dataclasses.replace(c, **over)


def ensemble(n_rep=64, seed=5):
    """Replica shapes of the batched ensemble: N ~ U[512, 32768] rounded to
    8 n^3 with n in [4, 16]; composition uniform over NaCl, LiCl, LiCl-NaCl;
    T ~ U[1100, 1300] K.  (LiCl and LiCl-NaCl use Table 3; no K+ parameters
    are printed in the paper.)"""
    rng = np.random.Generator(np.random.Philox(seed))
    comps = ["NaCl", "LiCl", "LiCl-NaCl"]
    reps = []
    for r in range(n_rep):
        nd = rng.uniform(512, 32768)
        n = int(np.clip(round((nd / 8.0) ** (1.0 / 3.0)), 4, 16))
        comp = comps[int(rng.integers(0, 3))]
        T = float(rng.uniform(1100.0, 1300.0))
        w = rock_salt((n, n, n), seed=seed * 1000 + r, composition=comp)
        w.vel = maxwell_boltzmann(w, T)
        reps.append((w, T))
    return reps


def core_radii_from_sigma(bmh, r_core=6.0):
    """Species-dependent core radii (the adaptive cutoff named in Sec. 1 has no
    printed rule; this is the example rule used here): r_core scaled by each
    pair's BMH size parameter sigma_ab relative to the largest, so pairs of
    small ions keep a smaller exact core.  Symmetric [ns][ns] table."""
    sig = np.asarray(bmh, dtype=np.float64)[..., 1]
    return r_core * sig / sig.max()
