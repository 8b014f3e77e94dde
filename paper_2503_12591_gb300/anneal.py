"""Simulated annealing and the specific heat from energy fluctuations.

The paper anneals from 2000 K downwards in 50 K steps, discards the first
sweeps at each temperature and records the following ones to compute C_V
(Method "MC simulation"; Results "Energy model", Fig. CV).  The specific heat
is the textbook canonical fluctuation formula C_V = (<E^2> - <E>^2) / (k_B T^2).

The energy after every sweep comes from smcx_sweep_energies: the library
accumulates the exact sum of the accepted energy changes, so E(t) = E(0) +
(dsum(t) - dsum(0)), recorded on the device after each sweep and read once.
Every number here is computed by the CUDA library; this module only
schedules calls and sums the int64 energies it returns (FP64 moments).
"""
from dataclasses import dataclass, field
from typing import List

import numpy as np

KB_MEV = 8.617333262e-2  # meV / K


@dataclass
class AnnealStep:
    T: float
    sweeps_discarded: int
    sweeps_recorded: int
    mean_E: float          # 0.01 meV
    var_E: float           # (0.01 meV)^2
    cv_per_site: float     # k_B units per site: C_V / (N k_B)
    accept_rate: float
    energies: List[int] = field(default_factory=list)


def energy_trace(lat, T: float, n: int, seed: int):
    """Sweep n times at T; return the exact energy after each sweep."""
    return [int(e) for e in lat.sweep_energies(T, n, seed)]


def specific_heat(energies, T: float, n_sites: int) -> float:
    """C_V / (N k_B) = (<E^2> - <E>^2) / (N (k_B T)^2), E in 0.01 meV."""
    e = np.asarray(energies, np.float64) * 0.01  # meV
    return float(e.var() / (n_sites * (KB_MEV * T) ** 2))


def anneal(lat, temperatures, discard: int, record: int, seed: int, keep_energies=False):
    """Run the annealing schedule; return one AnnealStep per temperature."""
    steps = []
    for T in temperatures:
        st0 = lat.state()[1].copy()
        if discard:
            lat.sweep(T, discard, seed)
        E = energy_trace(lat, T, record, seed)
        st1 = lat.state()[1]
        trials = max(1, int(st1[0] - st0[0]))
        e = np.asarray(E, np.float64)
        steps.append(AnnealStep(T=float(T), sweeps_discarded=discard, sweeps_recorded=record,
                                mean_E=float(e.mean()), var_E=float(e.var()),
                                cv_per_site=specific_heat(E, T, lat.N),
                                accept_rate=float(st1[1] - st0[1]) / trials,
                                energies=list(E) if keep_energies else []))
    return steps


def paper_schedule(t_hi=2000.0, t_lo=1000.0, step=50.0):
    """2000 K down to t_lo in 50 K steps."""
    n = int(round((t_hi - t_lo) / step))
    return [t_hi - i * step for i in range(n + 1)]
