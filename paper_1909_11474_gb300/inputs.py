"""Seeded synthetic inputs for the minimal Tersoff hot path.

This module only draws random numbers and lays out diamond-silicon geometry; it holds none of the
potential's arithmetic. Both the CUDA path (through the binding) and the FP64 CPU oracle receive
exactly the arrays built here.

The paper's training data are DFT calculations on 64-atom periodic diamond cells, strained cells and
thermal snapshots (Sec. III.A); those data are not available, so seeded cells with the same shapes
stand in for them:

* diamond Si, conventional 8-atom cubic basis, lattice a = 5.431 A, m_x x m_y x m_z supercells;
* a random symmetric strain eps with all six independent components ~ U(-s, s), applied as
  x -> (I + eps) x to positions and lattice rows;
* i.i.d. Gaussian displacements per Cartesian component;
* optional vacancies (random atoms removed);
* a population of parameter sets drawn gene-wise: gene ~ U[0, 1] mapped linearly to
  [value - 30%|value|, value + 30%|value|] around the Table 2 values (the paper's real-valued
  chromosome, Sec. III.B; the +-30% range is this workload's choice).

Every workload is seeded with numpy's PCG64 from SeedSequence(20191125 + workload id).
"""
from __future__ import annotations

import dataclasses

import numpy as np

# Table 2 of the paper: optimised minimal-Tersoff parameters, in the gene order of Eq. 16
# x = [D0 (eV), alpha (1/A), r0 (A), beta, n, h], and the hand-chosen cutoffs R1, R2 (A).
TABLE2_PARAMS = np.array([3.21481, 1.43134, 2.23801, 0.282818, 0.602568, -0.641048], dtype=np.float64)
TABLE2_R1 = 2.8
TABLE2_R2 = 3.2
PARAM_NAMES = ("D0", "alpha", "r0", "beta", "n", "h")

LATTICE_A = 5.431  # A, conventional cubic lattice constant of the synthetic cells
SEED_BASE = 20191125

# Conventional diamond basis in fractional coordinates: fcc sites plus the (1/4,1/4,1/4) copy.
_FCC = np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])
DIAMOND_BASIS = np.concatenate([_FCC, _FCC + 0.25], axis=0)


def rng_for(workload_id: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(SEED_BASE + workload_id)))


def diamond_supercell(reps=(2, 2, 2), a: float = LATTICE_A):
    """Perfect diamond supercell: positions [N][3] and box [3][3] (rows are lattice vectors)."""
    mx, my, mz = reps
    cells = np.array([[i, j, k] for i in range(mx) for j in range(my) for k in range(mz)], dtype=np.float64)
    frac = (cells[:, None, :] + DIAMOND_BASIS[None, :, :]).reshape(-1, 3)
    pos = frac * a
    box = np.diag([mx * a, my * a, mz * a]).astype(np.float64)
    return pos, box


def random_strain(rng: np.random.Generator, s: float) -> np.ndarray:
    """Symmetric strain tensor, six independent components ~ U(-s, s)."""
    e = rng.uniform(-s, s, size=6)
    return np.array([[e[0], e[3], e[5]], [e[3], e[1], e[4]], [e[5], e[4], e[2]]], dtype=np.float64)


def thermal_velocities(rng: np.random.Generator, mass: np.ndarray, T: float) -> np.ndarray:
    """Maxwell-Boltzmann velocities (A/fs) at temperature T (K) for masses in amu, with the
    centre-of-mass velocity removed. Each component has variance kB T / m; kB T / m in eV/amu is
    converted with 1 eV/amu = 9.648533215665e-3 A^2/fs^2 (CODATA 2018)."""
    mass = np.asarray(mass, dtype=np.float64)
    sd = np.sqrt(8.617333262e-5 * T / mass * 9.648533215665e-3)
    v = rng.normal(0.0, 1.0, size=(len(mass), 3)) * sd[:, None]
    v -= (mass[:, None] * v).sum(0) / mass.sum()
    return v


SI_MASS = 28.0855   # amu, standard atomic weight of Si


def apply_strain(pos: np.ndarray, box: np.ndarray, eps: np.ndarray):
    m = np.eye(3) + eps
    return pos @ m.T, box @ m.T


@dataclasses.dataclass
class ConfigSet:
    """A batch of periodic configurations laid out for the C-ABI.

    pos      [Ntot][3] float64, atoms of config c are rows atom_off[c] .. atom_off[c+1]-1
    box      [C][3][3] float64, row k is lattice vector k of config c
    atom_off [C+1]     int32
    """
    pos: np.ndarray
    box: np.ndarray
    atom_off: np.ndarray

    @property
    def C(self) -> int:
        return len(self.atom_off) - 1

    @property
    def natoms(self) -> np.ndarray:
        return np.diff(self.atom_off)

    @property
    def Ntot(self) -> int:
        return int(self.atom_off[-1])

    def config(self, c: int):
        a, b = int(self.atom_off[c]), int(self.atom_off[c + 1])
        return self.pos[a:b], self.box[c]


def pack_configs(pos_list, box_list) -> ConfigSet:
    off = np.zeros(len(pos_list) + 1, dtype=np.int32)
    off[1:] = np.cumsum([len(p) for p in pos_list])
    return ConfigSet(np.ascontiguousarray(np.concatenate(pos_list, axis=0), dtype=np.float64),
                     np.ascontiguousarray(np.stack(box_list), dtype=np.float64), off)


def make_cells(rng, C, reps_fn, strain_fn, sigma_fn, vac_fn) -> ConfigSet:
    pos_list, box_list = [], []
    for _ in range(C):
        reps = reps_fn()
        pos, box = diamond_supercell(reps)
        nvac = vac_fn()
        if nvac > 0:
            keep = np.sort(rng.choice(len(pos), size=len(pos) - nvac, replace=False))
            pos = pos[keep]
        eps = strain_fn()
        pos, box = apply_strain(pos, box, eps)
        sigma = sigma_fn()
        pos = pos + rng.normal(0.0, sigma, size=pos.shape)
        pos_list.append(pos)
        box_list.append(box)
    return pack_configs(pos_list, box_list)


def population(rng, P: int, center=TABLE2_PARAMS, rel: float = 0.30):
    """P parameter sets: genes ~ U[0,1], mapped to [center - rel|center|, center + rel|center|]."""
    genes = rng.uniform(0.0, 1.0, size=(P, 6))
    lo = center - rel * np.abs(center)
    hi = center + rel * np.abs(center)
    return np.ascontiguousarray(lo + genes * (hi - lo)), genes


def target_noise(rng, C: int, natoms: np.ndarray, e_sigma=1e-3, w_sigma=5e-3, f_sigma=0.02):
    """Gaussian noise for targets: E per atom (eV), W per atom (6 comps, eV), F (eV/A)."""
    ne = rng.normal(0.0, e_sigma, size=C)
    nw = rng.normal(0.0, w_sigma, size=(C, 6))
    nf = rng.normal(0.0, f_sigma, size=(int(np.sum(natoms)), 3))
    return ne, nw, nf


# ----------------------------------------------------------------------------------------------
# The five workloads.  Each returns a dict of numpy arrays; sizes can be scaled down for tests.
# ----------------------------------------------------------------------------------------------

def workload_single_cell():
    """One 2x2x2 (64-atom) cell, displacements sigma = 0.05 A, Table 2 parameters."""
    rng = rng_for(1)
    cs = make_cells(rng, 1, lambda: (2, 2, 2), lambda: np.zeros((3, 3)), lambda: 0.05, lambda: 0)
    return {"configs": cs, "params": TABLE2_PARAMS[None, :].copy()}


def workload_ga_batch(P: int = 200, C: int = 300):
    """GA fitness batch: P random parameter sets x C 64-atom cells, strain +-2 %, sigma = 0.1 A."""
    rng = rng_for(2)
    cs = make_cells(rng, C, lambda: (2, 2, 2), lambda: random_strain(rng, 0.02), lambda: 0.1, lambda: 0)
    params, genes = population(rng, P)
    noise = target_noise(rng, C, cs.natoms)
    return {"configs": cs, "params": params, "genes": genes, "noise": noise, "hidden": TABLE2_PARAMS.copy()}


def workload_uneven(P: int = 1000, C: int = 500):
    """Uneven batch: supercells 1..4 per axis (8..512 atoms), 0-2 vacancies, strain +-3 %,
    sigma ~ U(0.05, 0.2) A."""
    rng = rng_for(3)
    cs = make_cells(rng, C,
                    lambda: tuple(int(v) for v in rng.integers(1, 5, size=3)),
                    lambda: random_strain(rng, 0.03),
                    lambda: float(rng.uniform(0.05, 0.2)),
                    lambda: int(rng.integers(0, 3)))
    params, genes = population(rng, P)
    noise = target_noise(rng, C, cs.natoms)
    return {"configs": cs, "params": params, "genes": genes, "noise": noise, "hidden": TABLE2_PARAMS.copy()}


def workload_adjoint(P: int = 64, C: int = 100):
    """Adjoint workload: P parameter sets x C 64-atom cells of the GA-batch distribution."""
    rng = rng_for(4)
    cs = make_cells(rng, C, lambda: (2, 2, 2), lambda: random_strain(rng, 0.02), lambda: 0.1, lambda: 0)
    params, genes = population(rng, P)
    noise = target_noise(rng, C, cs.natoms)
    return {"configs": cs, "params": params, "genes": genes, "noise": noise, "hidden": TABLE2_PARAMS.copy()}


def workload_md(reps: int = 40, sigma: float = 0.08):
    """MD-scale force call: reps^3 conventional cells (512,000 atoms at reps = 40), sigma = 0.08 A."""
    rng = rng_for(5)
    cs = make_cells(rng, 1, lambda: (reps, reps, reps), lambda: np.zeros((3, 3)), lambda: sigma, lambda: 0)
    return {"configs": cs, "params": TABLE2_PARAMS[None, :].copy()}


def with_targets(w: dict, clean_E, clean_W, clean_F, mask=None):
    """Attach targets = clean values (per-atom E and W, forces) + the workload's noise draw."""
    ne, nw, nf = w["noise"]
    C = w["configs"].C
    t = {
        "E": np.ascontiguousarray(clean_E + ne, dtype=np.float64),
        "W": np.ascontiguousarray(clean_W + nw, dtype=np.float64),
        "F": np.ascontiguousarray(clean_F + nf, dtype=np.float64),
        "mask": np.full(C, 7, dtype=np.uint8) if mask is None else np.asarray(mask, dtype=np.uint8),
    }
    return t
