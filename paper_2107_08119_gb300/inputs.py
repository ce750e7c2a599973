"""Seeded synthetic inputs shaped like the paper's workloads.

This module builds positions, boxes, velocities, parameter vectors and
training structures only; it holds none of the method's arithmetic.  Both the
CUDA path's tests and the FP64 oracle's tests draw their inputs from here.

The paper's DFT training sets (general Si, silicene, PbTe) are not available;
diamond-lattice silicon-like structures stand in for them (the general-Si
model of Table I uses a 5 A cutoff on the same material).

Units: Angstrom, fs, amu, eV, K.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 2107081190
A_SI = 5.43            # cubic diamond lattice constant of Si (Angstrom)
MASS_SI = 28.0         # amu
KB_EV = 8.617333262e-5  # Boltzmann constant (eV/K)
# 1 amu A^2/fs^2 in eV, from the CODATA 2018 atomic mass constant and elementary charge
AMU_A2_FS2_EV = 1.66053906660e-27 * 1.0e-20 / 1.0e-30 / 1.602176634e-19

# PbTe-like two-species rocksalt (the paper's PbTe model, Table I: r_c^R = 8 A,
# n_max^R = 12, r_c^A = 4 A, n_max^A = 6, l_max = 4, 40 neurons, 41 descriptors)
A_PBTE = 6.46           # rocksalt PbTe lattice constant (Angstrom)
Z_PB, Z_TE = 82.0, 52.0  # atomic numbers: the multicomponent weights sqrt(Z_i Z_j)
MASS_PBTE = 167.4       # amu: the mean of Pb (207.2) and Te (127.6); the MD here takes one mass
PBTE_HYPER = dict(n_max_R=12, n_max_A=6, l_max=4, n_neu=40, rc_R=8.0, rc_A=4.0)

_ROCKSALT_CATION = np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])

_DIAMOND_BASIS = np.array([
    [0.00, 0.00, 0.00], [0.00, 0.50, 0.50], [0.50, 0.00, 0.50], [0.50, 0.50, 0.00],
    [0.25, 0.25, 0.25], [0.25, 0.75, 0.75], [0.75, 0.25, 0.75], [0.75, 0.75, 0.25],
])


def rng_for(config: int, stream: int = 0) -> np.random.Generator:
    return np.random.default_rng([BASE_SEED + config, stream])


def diamond(n1: int, n2: int, n3: int, a: float = A_SI):
    """Perfect cubic-diamond supercell: positions (8 n1 n2 n3, 3), box (3, 3).
    Atoms are ordered cell by cell (x slowest), basis atoms innermost."""
    ii, jj, kk = np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij")
    cells = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1).astype(np.float64)
    pos = (cells[:, None, :] + _DIAMOND_BASIS[None, :, :]).reshape(-1, 3) * a
    box = np.diag([n1 * a, n2 * a, n3 * a]).astype(np.float64)
    return pos, box


def rocksalt(n1: int, n2: int, n3: int, a: float = A_PBTE):
    """Rocksalt supercell: positions (8 n1 n2 n3, 3), species numbers (Pb on
    the fcc sites, Te shifted by a/2 along x), box (3, 3)."""
    ii, jj, kk = np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij")
    cells = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1).astype(np.float64)
    basis = np.concatenate([_ROCKSALT_CATION, _ROCKSALT_CATION + [0.5, 0.0, 0.0]])
    pos = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a
    Z = np.tile(np.array([Z_PB] * 4 + [Z_TE] * 4), len(cells))
    box = np.diag([n1 * a, n2 * a, n3 * a]).astype(np.float64)
    return pos, Z, box


def displace(pos, sigma: float, rng: np.random.Generator):
    return pos + rng.normal(0.0, sigma, size=pos.shape)


def random_z(n_par: int, rng: np.random.Generator, low: float = -0.5, high: float = 0.5):
    """Parameter vector drawn uniformly, as the paper initialises the SNES mean."""
    return rng.uniform(low, high, size=n_par)


def maxwell_boltzmann(n: int, temperature: float, mass: float, rng: np.random.Generator):
    """Velocities (n, 3) in A/fs at exactly `temperature` with 3n - 3 degrees of
    freedom after removing the centre-of-mass velocity."""
    sd = np.sqrt(KB_EV * temperature / (mass * AMU_A2_FS2_EV))
    v = rng.normal(0.0, sd, size=(n, 3))
    v -= v.mean(axis=0)
    ek = 0.5 * mass * AMU_A2_FS2_EV * np.sum(v * v)
    t_now = 2.0 * ek / ((3 * n - 3) * KB_EV)
    return v * np.sqrt(temperature / t_now)


def remove_sites(pos, n_remove: int, rng: np.random.Generator):
    """Vacancies: drop `n_remove` sites chosen by a seeded permutation; the
    remaining atoms keep their original order."""
    keep = np.sort(rng.permutation(pos.shape[0])[n_remove:])
    return pos[keep]


# ---------------------------------------------------------------- workloads
def config1(n_par: int = 1021):
    """512-atom diamond (4x4x4 cells), sigma = 0.1 A, weights U(-1/2, 1/2)."""
    rng = rng_for(1)
    pos, box = diamond(4, 4, 4)
    pos = displace(pos, 0.1, rng)
    z = random_z(n_par, rng)
    return pos, box, z


def config2(n_cells: int = 25, n_par: int = 1021, temperature: float = 300.0):
    """NVE MD: n_cells^3 diamond cells (125,000 atoms at 25), sigma = 0.1 A,
    Maxwell-Boltzmann velocities at 300 K, mass 28 amu."""
    rng = rng_for(2)
    pos, box = diamond(n_cells, n_cells, n_cells)
    pos = displace(pos, 0.1, rng)
    vel = maxwell_boltzmann(pos.shape[0], temperature, MASS_SI, rng)
    z = random_z(n_par, rng)
    return pos, vel, box, z


def config3(cells=(40, 40, 80), vacancy_fraction: float = 0.1, n_par: int = 1021,
            temperature: float = 300.0):
    """Heat-transport MD: diamond cells with 10 % of sites removed at random,
    sigma = 0.15 A, 300 K.  cells=(4, 4, 4) gives the 512-site replica."""
    rng = rng_for(3, stream=int(np.prod(cells)))
    pos, box = diamond(*cells)
    n_vac = int(round(vacancy_fraction * pos.shape[0]))
    pos = remove_sites(pos, n_vac, rng)
    pos = displace(pos, 0.15, rng)
    vel = maxwell_boltzmann(pos.shape[0], temperature, MASS_SI, rng)
    z = random_z(n_par, rng)
    return pos, vel, box, z


def config_pbte(cells=(4, 4, 4), sigma: float = 0.1, temperature: float = 300.0):
    """PbTe-like two-species workload for the split-hyperparameter model:
    rocksalt cells (a = 6.46 A), seeded displacements sigma = 0.1 A,
    Maxwell-Boltzmann velocities at 300 K with the one mass MASS_PBTE, and a
    parameter vector of the 41-40-1 network drawn U(-1/2, 1/2) with the
    input-layer weights matched to the scale of the weighted descriptors:
    the weights sqrt(Z_i Z_j) (atomic numbers 82 and 52) make the radial
    descriptors ~Zbar and the angular ones ~Zbar^2 times larger than for one
    species of weight 1 (Zbar = sqrt(82 x 52)), so the columns of w1 for the
    13 radial descriptors are divided by Zbar and those for the 28 angular
    ones by Zbar^2 (a trained potential's weights match its inputs; random
    U(-1/2, 1/2) weights on descriptors of ~1e3 would saturate the network).
    Returns (pos, vel, box, z, Z) with Z the atomic number of every atom."""
    rng = rng_for(6, stream=int(np.prod(cells)))
    pos, Z, box = rocksalt(*cells)
    pos = displace(pos, sigma, rng)
    vel = maxwell_boltzmann(pos.shape[0], temperature, MASS_PBTE, rng)
    n_r = PBTE_HYPER["n_max_R"] + 1
    n_des = n_r + (PBTE_HYPER["n_max_A"] + 1) * PBTE_HYPER["l_max"]
    n_neu = PBTE_HYPER["n_neu"]
    z = random_z((n_des + 2) * n_neu + 1, rng)
    zbar = np.sqrt(Z_PB * Z_TE)
    w1 = z[:n_neu * n_des].reshape(n_neu, n_des)
    w1[:, :n_r] /= zbar
    w1[:, n_r:] /= zbar ** 2
    return pos, vel, box, z, Z


def training_structures(n_struct: int = 200, seed_stream: int = 0):
    """Periodic training cells of uneven size: 8 n1 n2 n3 atoms in [32, 256],
    lattice constant 5.43 (1 + d)^(-1/3) with d ~ U(-0.1, 0.1) (density +-10 %),
    displacements with sigma ~ U(0.1, 0.3) A."""
    rng = rng_for(4, stream=seed_stream)
    shapes = [(a, b, c) for a in range(1, 5) for b in range(1, 5) for c in range(1, 5) if 4 <= a * b * c <= 32]
    out = []
    for _ in range(n_struct):
        n1, n2, n3 = shapes[rng.integers(len(shapes))]
        d = rng.uniform(-0.1, 0.1)
        a = A_SI * (1.0 + d) ** (-1.0 / 3.0)
        pos, box = diamond(n1, n2, n3, a)
        sigma = rng.uniform(0.1, 0.3)
        pos = displace(pos, sigma, rng)
        out.append({"pos": pos, "box": box})
    return out


def config4(n_struct: int = 200, n_pop: int = 50, n_par: int = 1021):
    """SNES generation: training structures, a teacher parameter vector
    (labels are computed from it by whichever NEP evaluator the caller uses)
    and a population z_k ~ N(0, 0.1^2) (mean 0, step 0.1)."""
    structures = training_structures(n_struct)
    rng = rng_for(4, stream=1)
    teacher = random_z(n_par, rng)
    pop = rng.normal(0.0, 0.1, size=(n_pop, n_par))
    return structures, teacher, pop


def config5(n_par: int = 1021):
    """64-atom (2x2x2 cells) check structure for gradients, sigma = 0.15 A,
    a teacher and a student parameter vector."""
    rng = rng_for(5)
    pos, box = diamond(2, 2, 2)
    pos = displace(pos, 0.15, rng)
    teacher = random_z(n_par, rng)
    student = random_z(n_par, rng)
    return pos, box, teacher, student
