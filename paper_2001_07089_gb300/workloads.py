"""Seeded synthetic inputs for the Kob-Andersen workloads.

This module only produces inputs: interaction parameters as the paper states
them, box sizes from the density, seeded type assignments and replica
mixes. It holds none of the method's arithmetic (no forces, no integration,
no thermostat), so both the CUDA path and the CPU oracle can take their
inputs from here without sharing any computation.

Sources of the numbers:
* Kob-Andersen parameters: eps_AA = 1, eps_AB = 1.5, eps_BB = 0.5,
  sigma_AA = 1, sigma_AB = 0.8, sigma_BB = 0.88, m = 1, cutoff 2.5 sigma_ab
  (Sec. "Model", Eqs. (VKALJ) and (VshiftedKALJ)).
* 80:20 A:B mixture (Sec. "Model"); B particles are placed at seeded random
  indices, which has the same distribution as the paper's random swap of each
  B with an A (Sec. "Initialization of positions").
* Density 1.2 and the workload sizes are those of the benchmark
  configurations (N = 1000, 32 000, 10^6, 8*10^6, and a 512-replica mix).
* The two-dimensional variant (Sec. "Suggested problems"): N = 1000 at
  N/L^2 = 1.204 (L = 28.82) with A:B = 65:35.
"""
from __future__ import annotations

import dataclasses

import numpy as np

KA_EPS = np.array([[1.0, 1.5], [1.5, 0.5]])
KA_SIG = np.array([[1.0, 0.8], [0.8, 0.88]])
KA_RC = 2.5 * KA_SIG
KA_MASS = 1.0
DENSITY = 1.2
# the two-dimensional problem (Sec. "Suggested problems"): N/L^2 = 1.204, A:B = 65:35
DENSITY_2D = 1.204
FRAC_B_2D = 0.35
SKIN = 0.3
DT = 0.005


def box_length(n: int, density: float = DENSITY) -> float:
    """Edge of the cubic box holding n particles at the given number density."""
    return float((n / density) ** (1.0 / 3.0))


def box_length_2d(n: int, density: float = DENSITY_2D) -> float:
    """Edge of the square box holding n particles at the given areal density (two dimensions)."""
    return float(np.sqrt(n / density))


def ka_types(n: int, seed: int, frac_b: float = 0.2) -> np.ndarray:
    """uint8 types: round(frac_b*n) B particles (type 1) at seeded random indices."""
    nb = int(round(frac_b * n))
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x4B41]))
    t = np.zeros(n, dtype=np.uint8)
    if nb:
        t[rng.choice(n, size=nb, replace=False)] = 1
    return t


def uniform_positions(n: int, L: float, seed: int) -> np.ndarray:
    """n x 3 positions uniform in [0, L) (an ideal-gas configuration)."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x5550]))
    return rng.uniform(0.0, L, size=(n, 3))


def gaussian_velocities(n: int, T: float, seed: int) -> np.ndarray:
    """n x 3 velocities with independent N(0, T) components (no centring)."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x5645]))
    return rng.normal(0.0, np.sqrt(T), size=(n, 3))


ENSEMBLE_SIZES = (250, 500, 1000, 2000, 4000, 8000)


@dataclasses.dataclass
class EnsembleSpec:
    n: np.ndarray       # int64 particles per replica
    T: np.ndarray       # float64 bath temperature per replica
    L: np.ndarray       # float64 box edge per replica
    types: list         # uint8 array per replica

    @property
    def total(self) -> int:
        return int(self.n.sum())


def ensemble(nrep: int = 512, seed: int = 4, sizes=ENSEMBLE_SIZES, t_lo: float = 0.45,
             t_hi: float = 2.0) -> EnsembleSpec:
    """Replica mix: N uniform over `sizes`, T uniform in [t_lo, t_hi], density 1.2."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x454E]))
    n = rng.choice(np.asarray(sizes, dtype=np.int64), size=nrep)
    T = rng.uniform(t_lo, t_hi, size=nrep)
    L = np.array([box_length(int(k)) for k in n])
    types = [ka_types(int(k), seed * 100003 + r) for r, k in enumerate(n)]
    return EnsembleSpec(n=n.astype(np.int64), T=T, L=L, types=types)


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    n: int
    seed: int
    T0: float
    description: str

    @property
    def L(self) -> float:
        return box_length(self.n)


WORKLOADS = {
    "ka1k": Workload("ka1k", 1000, 1, 2.0,
                     "KA 80:20, N=1000, rho=1.2, 10^3 lattice + 0.05 jitter, MB T=2.0, NVE dt=0.005, FP64"),
    "ka32k": Workload("ka32k", 32000, 2, 2.0,
                      "KA 80:20, N=32000, rho=1.2, cell + Verlet list skin 0.3, NVT T=0.8 then NVE dt=0.005"),
    "ka1m": Workload("ka1m", 1_000_000, 3, 0.5,
                     "KA 80:20, N=10^6, rho=1.2, 100^3 lattice, NVT T=0.5, dt=0.005, mixed"),
    "ka8m": Workload("ka8m", 8_000_000, 5, 2.0,
                     "KA 80:20, N=8*10^6, rho=1.2, 200^3 lattice, quench 2.0 -> 0.45 then NVE"),
}
