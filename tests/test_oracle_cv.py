"""Pins of the oracle's specific heat (Results, Fig. C_V; Method "MC
simulation"): C_V / (N k_B) = Var(E) / (N (k_B T)^2) from energy
fluctuations.

The fluctuation form is checked against the definition C_V = d<E>/dT: on the
16-site BCC box (binary 8/8, 12,870 states, Supplementary "Statistical
mechanics" for the canonical average) the oracle, given the enumerated
energies with Boltzmann weights, must equal a central finite difference of
the exactly enumerated <E>(T), divided by N k_B.  A wrong k_B unit, a missing
0.01 meV factor, a per-site slip or a standard deviation in place of the
variance fails it.  A two-level system checks the closed form of the Schottky
anomaly, and a recorded trace (unit weights) checks the time-average form.
"""
import itertools

import numpy as np
import pytest

import oracle as O
from paper_2503_12591_gb300.inputs import epi_gaussian

KB = 8.617333262e-2  # meV/K (exact SI definition)


def _enumerated_energies():
    dims, K = (2, 2, 2), 4
    V = epi_gaussian(K, 2, 20.0, 11)
    E = []
    for ones in itertools.combinations(range(16), 8):
        s = np.zeros(16, np.int8)
        s[list(ones)] = 1
        E.append(O.energy(O.BCC, dims, 2, K, V, s))
    return np.array(E, np.int64)


def _boltzmann(E, T):
    e = E.astype(np.float64) * 0.01  # meV
    return np.exp(-(e - e.min()) / (KB * T))


def _mean_energy_mev(E, T):
    w = _boltzmann(E, T)
    return float((w * E.astype(np.float64) * 0.01).sum() / w.sum())


@pytest.mark.parametrize("T", [300.0, 1000.0, 2500.0])
def test_fluctuation_equals_derivative_of_mean_energy(T):
    E = _enumerated_energies()
    assert E.size == 12870
    N = 16
    mean, var, cv = O.specific_heat(E, N, T, w=_boltzmann(E, T))
    h = 1e-3 * T
    dEdT = (_mean_energy_mev(E, T + h) - _mean_energy_mev(E, T - h)) / (2 * h)  # meV / K
    assert cv == pytest.approx(dEdT / (N * KB), rel=1e-6)
    assert mean * 0.01 == pytest.approx(_mean_energy_mev(E, T), rel=1e-12)
    assert cv > 0.0


@pytest.mark.parametrize("g0,g1,delta_mev,T", [(1, 1, 50.0, 600.0), (2, 5, 120.0, 900.0), (3, 1, 10.0, 3000.0)])
def test_two_level_closed_form(g0, g1, delta_mev, T):
    # two levels 0 and delta with degeneracies g0, g1, one site:
    # C / k_B = g0 g1 x^2 e^x / (g0 e^x + g1)^2 with x = delta / (k_B T)
    x = delta_mev / (KB * T)
    want = g0 * g1 * x * x * np.exp(x) / (g0 * np.exp(x) + g1) ** 2
    E = np.array([0, int(round(delta_mev * 100))], np.int64)
    w = np.array([g0, g1 * np.exp(-x)])
    _, _, cv = O.specific_heat(E, 1, T, w=w)
    assert cv == pytest.approx(want, rel=1e-12)


def test_trace_average_and_shift_invariance():
    # a trace alternating between two energies a, b has Var = (b - a)^2 / 4
    a, b, N, T = -123456789, -123400000, 1000, 1500.0
    E = np.array([a, b] * 50, np.int64)
    mean, var, cv = O.specific_heat(E, N, T)
    assert mean == pytest.approx((a + b) / 2, rel=1e-15)
    assert var == pytest.approx((b - a) ** 2 / 4, rel=1e-12)
    assert cv == pytest.approx(((b - a) * 0.01) ** 2 / 4 / (N * (KB * T) ** 2), rel=1e-12)
    # shifting every energy leaves the fluctuation unchanged
    _, var2, cv2 = O.specific_heat(E + 987654321, N, T)
    assert var2 == pytest.approx(var, rel=1e-12) and cv2 == pytest.approx(cv, rel=1e-12)
    # a constant trace has no fluctuation
    assert O.specific_heat(np.full(7, a, np.int64), N, T)[2] == 0.0
    with pytest.raises(ValueError):
        O.specific_heat(E, N, 0.0)
