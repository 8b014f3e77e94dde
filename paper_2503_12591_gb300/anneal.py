"""Simulated annealing and the specific heat from energy fluctuations.

The paper anneals from 2000 K downwards in 50 K steps, discards the first
sweeps at each temperature and records the following ones to compute C_V
(Method "MC simulation"; Results "Energy model", Fig. CV).  The specific heat
is the canonical fluctuation formula C_V = (<E^2> - <E>^2) / (k_B T^2).

This module only schedules library calls.  smcx_sweep_cv sweeps, records the
exact energy after every sweep on the device (E(0) plus the accepted energy
changes) and reduces that trace on the device in FP64 to <E>, Var(E) and
C_V / (N k_B); the acceptance rate comes from the library's counters.
"""
from dataclasses import dataclass, field
from typing import List


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


def anneal(lat, temperatures, discard: int, record: int, seed: int, keep_energies=False):
    """Run the annealing schedule; return one AnnealStep per temperature."""
    steps = []
    for T in temperatures:
        st0 = lat.state()[1].copy()
        if discard:
            lat.sweep(T, discard, seed)
        E, mean, var, cv = lat.sweep_cv(T, record, seed, want_trace=keep_energies)
        st1 = lat.state()[1]
        trials = max(1, int(st1[0] - st0[0]))
        steps.append(AnnealStep(T=float(T), sweeps_discarded=discard, sweeps_recorded=record,
                                mean_E=mean, var_E=var, cv_per_site=cv,
                                accept_rate=float(st1[1] - st0[1]) / trials,
                                energies=[int(e) for e in E] if keep_energies else []))
    return steps


def paper_schedule(t_hi=2000.0, t_lo=1000.0, step=50.0):
    """2000 K down to t_lo in 50 K steps."""
    n = int(round((t_hi - t_lo) / step))
    return [t_hi - i * step for i in range(n + 1)]
