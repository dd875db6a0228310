"""Seeded synthetic inputs shared by the tests, the benchmark and ``smoke()``.

This module holds no arithmetic of the method: it only builds lattices,
species, masses, potential parameters and random-initialised MLP weights with
numpy's seeded generator.  The paper's systems (FCC copper, bulk water, LGPS,
alanine peptides) and its pretrained MLIPs (UMA, Orb, EMT, GFF) are not
available; these synthetic systems stand in for them with the same structure:
dense periodic atomic systems of 32 to 32,768 atoms with a cheap pair-potential
draft and a costlier many-body target.

Configurations (window length K is the lookahead L of Alg. 1):

1. 32 atoms, one species (39.95 amu), 12 A box, FCC 2x2x2 (a = 6 A); target =
   LJ (eps 0.0104 eV, sigma 3.4 A, cutoff 8.5 A) + 0.05 eV tanh(MLP 17->64->64->1)
   on 16 radial basis functions at 5 A; draft = LJ; dt 2 fs, gamma 0.01/fs,
   300 K, K = 8.
2. 256 atoms, two species (12, 16 amu) alternating, 20 A box, FCC 4x4x4;
   MLP 50->128x3->1 on 2x16 radial + 16 angular + 2 one-hot, FP32; LJ draft
   with per-species eps/sigma; dt 1 fs, 300 K, K = 16.
3. configuration 1 with a learned draft: LJ + MLP 9->32->1 on 8 radial basis
   functions, linear head, BF16 inference.
4. 4,096 atoms, three species (1, 12, 16 amu) cycled, rho = 0.1/A^3, simple
   cubic 16^3, cutoffs 6 A; MLP 67->256x4->1 in BF16; dt 0.5 fs, 350 K, K = 32.
5. 32,768 atoms, three species, 70 A box, simple cubic 32^3; MLP 67->256x4->1
   in FP8; K = 64.

Positions get a uniform jitter of +-0.05 nearest-neighbour spacings (seed 0),
momenta are Maxwell-Boltzmann at T (seed 2), MLP weights are N(0, 1/fan_in)
(seed 1), biases 0, rounded to float32 so that every consumer sees the same
numbers.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

# physical constants used only to draw initial momenta (CODATA 2018)
_KB_EV = 1.380649e-23 / 1.602176634e-19
_KAPPA = (1.602176634e-19 / 1e-10) / (1.66053906660e-27 * 1e-10 / 1e-30)


@dataclass
class System:
    positions: np.ndarray          # [N, 3] float64, Angstrom (unwrapped)
    momenta: np.ndarray            # [N, 3] float64, amu*Angstrom/fs
    species: np.ndarray            # [N] int32
    masses: np.ndarray             # [S] float64, amu
    box: np.ndarray                # [3] float64, Angstrom
    seed: int = 12345              # Philox key of the dynamics

    @property
    def n_atoms(self) -> int:
        return int(self.positions.shape[0])

    @property
    def n_species(self) -> int:
        return int(self.masses.shape[0])


@dataclass
class Potential:
    lj_eps: Optional[np.ndarray] = None
    lj_sigma: Optional[np.ndarray] = None
    lj_cutoff: float = 0.0
    n_rbf: int = 0
    n_ang: int = 0
    n_layers: int = 0
    width: int = 0
    desc_cutoff: float = 0.0
    head: str = "tanh"             # "tanh": head_scale*tanh(y) per atom; "linear": y per atom
    head_scale: float = 0.05
    weights: Optional[np.ndarray] = None   # packed float32 values stored as float64
    precision: str = "fp32"        # arithmetic of the MLP on the GPU: fp32 | bf16 | fp8
    k_harm: float = 0.0
    q_ref: Optional[np.ndarray] = None
    shear: float = 0.0


@dataclass
class Integrator:
    dt: float
    gamma: float
    temperature: float
    K: int
    scheme: str = "aboba"   # "aboba" (Eq. 2) or "obabo" (the staggered frame of App. E)


@dataclass
class Workload:
    name: str
    system: System
    draft: Potential
    target: Potential
    integ: Integrator
    n_steps: int
    notes: str = ""


def input_dim(n_species: int, n_rbf: int, n_ang: int) -> int:
    return n_species * n_rbf + n_ang + n_species


def n_weights(d0: int, n_layers: int, width: int) -> int:
    if n_layers <= 0:
        return 0
    return width * d0 + width + (n_layers - 1) * (width * width + width) + width + 1


def mlp_weights(d0: int, n_layers: int, width: int, seed: int, col_scale=None) -> np.ndarray:
    """W ~ N(0, 1/fan_in) in the packed order (layer, row, column), biases 0, rounded to float32.
    col_scale (optional, length d0) multiplies the columns of the first layer."""
    rng = np.random.default_rng(seed)
    parts = []
    din = d0
    for li in range(n_layers):
        w = rng.standard_normal((width, din)) / np.sqrt(din)
        if li == 0 and col_scale is not None:
            w = w * np.asarray(col_scale, dtype=np.float64)[None, :]
        parts.append(w)
        parts.append(np.zeros(width))
        din = width
    parts.append(rng.standard_normal(width) / np.sqrt(width))
    parts.append(np.zeros(1))
    w = np.concatenate([p.ravel() for p in parts]).astype(np.float32).astype(np.float64)
    assert w.size == n_weights(d0, n_layers, width)
    return w


def dense_input_scale(n_species: int, n_rbf: int = 16, n_ang: int = 16, angular: float = 1.0 / 40.0):
    """First-layer column scale for the dense (rho = 0.1/A^3, 6 A cutoff) systems: with ~90 neighbours the 16
    angular sums reach ~1e2 and unscaled N(0, 1/fan_in) weights saturate the tanh head (no MLP force at all);
    their columns are scaled by 1/40 so first-layer pre-activations are O(1).  Radial and one-hot columns: 1."""
    return np.concatenate([np.ones(n_species * n_rbf), np.full(n_ang, angular), np.ones(n_species)])


def fcc(cells: int, a: float) -> np.ndarray:
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    g = np.stack(np.meshgrid(*[np.arange(cells)] * 3, indexing="ij"), -1).reshape(-1, 3)
    return ((g[:, None, :] + basis[None]) * a).reshape(-1, 3)


def simple_cubic(cells: int, a: float) -> np.ndarray:
    g = np.stack(np.meshgrid(*[np.arange(cells)] * 3, indexing="ij"), -1).reshape(-1, 3)
    return (g + 0.5) * a


def jitter(pos: np.ndarray, spacing: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return pos + rng.uniform(-0.05 * spacing, 0.05 * spacing, size=pos.shape)


def mb_momenta(masses_per_atom: np.ndarray, temperature: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    sd = np.sqrt(masses_per_atom * _KB_EV * temperature * _KAPPA)
    return rng.standard_normal((masses_per_atom.size, 3)) * sd[:, None]


def _system(pos, species, masses, L, temperature, seed=12345):
    masses = np.asarray(masses, dtype=np.float64)
    species = np.asarray(species, dtype=np.int32)
    mom = mb_momenta(masses[species], temperature, seed=2)
    return System(positions=pos.astype(np.float64), momenta=mom, species=species, masses=masses,
                  box=np.array([L, L, L], dtype=np.float64), seed=seed)


def config1(K: int = 8) -> Workload:
    pos = jitter(fcc(2, 6.0), 6.0 / np.sqrt(2.0), seed=0)
    sysm = _system(pos, np.zeros(32), [39.95], 12.0, 300.0)
    lj = dict(lj_eps=np.array([0.0104]), lj_sigma=np.array([3.4]), lj_cutoff=8.5)
    d0 = input_dim(1, 16, 0)
    target = Potential(**lj, n_rbf=16, n_ang=0, n_layers=2, width=64, desc_cutoff=5.0, head="tanh", head_scale=0.05,
                       weights=mlp_weights(d0, 2, 64, seed=1), precision="fp32")
    draft = Potential(**lj)
    return Workload("lj_mlp_32atoms_K%d" % K, sysm, draft, target, Integrator(2.0, 0.01, 300.0, K), 1000)


def config2(K: int = 16) -> Workload:
    pos = jitter(fcc(4, 5.0), 5.0 / np.sqrt(2.0), seed=0)
    species = np.arange(256) % 2
    sysm = _system(pos, species, [12.0, 16.0], 20.0, 300.0)
    lj = dict(lj_eps=np.array([0.0104, 0.0067]), lj_sigma=np.array([3.0, 2.8]), lj_cutoff=8.5)
    d0 = input_dim(2, 16, 16)
    target = Potential(**lj, n_rbf=16, n_ang=16, n_layers=3, width=128, desc_cutoff=5.0, head="tanh",
                       head_scale=0.05, weights=mlp_weights(d0, 3, 128, seed=1), precision="fp32")
    draft = Potential(**lj)
    return Workload("lj_mlp_angular_256atoms_K%d" % K, sysm, draft, target, Integrator(1.0, 0.01, 300.0, K), 10000)


def learned_draft(base: Potential, n_species: int, seed: int = 3, precision: str = "bf16") -> Potential:
    """LJ + per-atom MLP 9->32->1 on 8 radial basis functions (linear head), starting from small random weights."""
    d0 = input_dim(n_species, 8, 0)
    w = mlp_weights(d0, 1, 32, seed=seed)
    # start near the pure pair draft: scale the output row down
    nw = w.size
    w[nw - 33:nw - 1] *= 1e-2
    w = w.astype(np.float32).astype(np.float64)
    return Potential(lj_eps=base.lj_eps, lj_sigma=base.lj_sigma, lj_cutoff=base.lj_cutoff, n_rbf=8, n_ang=0,
                     n_layers=1, width=32, desc_cutoff=base.desc_cutoff or 5.0, head="linear", head_scale=1.0,
                     weights=w, precision=precision)


def config3(K: int = 8) -> Workload:
    w = config1(K)
    w.draft = learned_draft(w.target, 1)
    w.name = "learned_draft_32atoms_K%d" % K
    w.n_steps = 10000
    return w


def _config_large(cells: int, L: float, K: int, precision: str, dt: float, T: float) -> Workload:
    spacing = L / cells
    pos = jitter(simple_cubic(cells, spacing), spacing, seed=0)
    n = pos.shape[0]
    species = np.arange(n) % 3
    sysm = _system(pos, species, [1.0, 12.0, 16.0], L, T)
    lj = dict(lj_eps=np.array([0.002, 0.004, 0.006]), lj_sigma=np.array([1.6, 2.2, 2.0]), lj_cutoff=6.0)
    d0 = input_dim(3, 16, 16)
    target = Potential(**lj, n_rbf=16, n_ang=16, n_layers=4, width=256, desc_cutoff=6.0, head="tanh",
                       head_scale=0.05, weights=mlp_weights(d0, 4, 256, seed=1, col_scale=dense_input_scale(3)),
                       precision=precision)
    draft = Potential(**lj)
    return Workload("bf16_mlp_%datoms_K%d" % (n, K), sysm, draft, target, Integrator(dt, 0.01, T, K), 2000)


def config4(K: int = 32) -> Workload:
    L = (4096 / 0.1) ** (1.0 / 3.0)
    return _config_large(16, L, K, "bf16", 0.5, 350.0)


def config5(K: int = 64) -> Workload:
    w = _config_large(32, 70.0, K, "fp8", 0.5, 350.0)
    w.name = "fp8_mlp_32768atoms_K%d" % K
    w.n_steps = 100000
    return w


def small_system(n_cells: int = 1, a: float = 5.0, n_species: int = 2, seed: int = 0, L: Optional[float] = None,
                 temperature: float = 300.0) -> System:
    """A tiny FCC system for brute-force and finite-difference checks."""
    pos = jitter(fcc(n_cells, a), a / np.sqrt(2.0), seed=seed)
    n = pos.shape[0]
    species = np.arange(n) % n_species
    masses = np.array([12.0, 16.0, 1.0][:n_species])
    return _system(pos, species, masses, L if L is not None else n_cells * a, temperature)


CONFIGS = {1: config1, 2: config2, 3: config3, 4: config4, 5: config5}


def replace(obj, **kw):
    return dataclasses.replace(obj, **kw)
