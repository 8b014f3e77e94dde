"""Seeded synthetic inputs (no method arithmetic lives here).

Both the CUDA path's callers and the oracle-based tests draw their inputs from
this module, so the two sides see identical EPI tables, compositions,
temperatures and lattice shapes.  Nothing here computes an energy, a
probability or a trajectory.

The trained EPI parameters of the paper are not published, so effective pair
interactions are drawn from a normal distribution of the stated width and
quantised to int32 in 0.01 meV units (the paper's models are per-shell
species-pair tables; Method, Eq. Linear_EPI and Eq. Total_EPI).
"""
from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np

BCC, FCC = 0, 1
INT8, PACKED4 = 0, 1


def epi_gaussian(K: int, M: int, sigma_mev: float, seed: int) -> np.ndarray:
    """Symmetric int32 [K][M][M] table in 0.01 meV units.

    Upper triangle including the diagonal is drawn from N(0, sigma_mev) with
    numpy's default_rng(seed) in row-major (k, p <= q) order, scaled by 100 and
    rounded half away from zero; the lower triangle mirrors it.
    """
    rng = np.random.default_rng(seed)
    V = np.zeros((K, M, M), np.int32)
    for k in range(K):
        for p in range(M):
            for q in range(p, M):
                x = rng.normal(0.0, sigma_mev) * 100.0
                r = int(np.sign(x) * np.floor(abs(x) + 0.5))
                V[k, p, q] = r
                V[k, q, p] = r
    return V


def equiatomic(M: int) -> List[float]:
    return [1.0 / M] * M


def random_species(n: int, M: int, seed: int) -> np.ndarray:
    """Uniform random int8 species ids (not composition-exact)."""
    return np.random.default_rng(seed).integers(0, M, n).astype(np.int8)


def log_temperatures(R: int, t_lo: float = 300.0, t_hi: float = 3000.0) -> np.ndarray:
    """T_r = t_lo * (t_hi/t_lo)^(r/(R-1)), r = 0..R-1."""
    if R == 1:
        return np.array([t_lo])
    return t_lo * (t_hi / t_lo) ** (np.arange(R) / (R - 1))


def batched_edges(R: int = 64, lo: int = 24, hi: int = 96, seed: int = 1) -> np.ndarray:
    """Per-replica cubic edge lengths drawn uniformly from {lo..hi}."""
    return np.random.default_rng(seed).integers(lo, hi + 1, R)


@dataclass
class Workload:
    name: str
    kind: int
    dims: Tuple[int, int, int]
    M: int
    K: int
    comp: List[float]
    sigma_mev: float
    epi_seed: int
    init_seed: int
    storage: int
    temperatures: List[float] = field(default_factory=list)
    sweeps: int = 1
    seed: int = 1

    @property
    def sites(self) -> int:
        m = 2 if self.kind == BCC else 4
        return self.dims[0] * self.dims[1] * self.dims[2] * m

    def epi(self) -> np.ndarray:
        return epi_gaussian(self.K, self.M, self.sigma_mev, self.epi_seed)


# Oracle-sized BCC 16^3 quaternary, 4-shell EPI, 1000 K, 100 sweeps.
ORACLE_BCC16 = Workload("bcc16_q4_k4_int8", BCC, (16, 16, 16), 4, 4, equiatomic(4), 20.0,
                        1, 1, INT8, [1000.0], 100, 1)
# Throughput BCC 256^3 (33.5M sites), int8.
THROUGHPUT_BCC256 = Workload("bcc256_q4_k4_int8", BCC, (256, 256, 256), 4, 4, equiatomic(4),
                             20.0, 1, 1, INT8, [2500.0, 1500.0, 800.0], 1000, 1)
# Scale: BCC 800^3 (1.024B sites) packed 4-bit at 1200 K.
SCALE_BCC800 = Workload("bcc800_q4_k4_packed4", BCC, (800, 800, 800), 4, 4, equiatomic(4),
                        20.0, 1, 1, PACKED4, [1200.0], 200, 1)
# Scale: FCC 400^3 (256M sites), 5 species 0.3/0.25/0.2/0.15/0.1, 3 shells, N(0,30 meV).
SCALE_FCC400 = Workload("fcc400_q5_k3_packed4", FCC, (400, 400, 400), 5, 3,
                        [0.3, 0.25, 0.2, 0.15, 0.1], 30.0, 1, 1, PACKED4, [1200.0], 200, 1)
