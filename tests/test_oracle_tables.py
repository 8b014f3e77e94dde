"""Oracle acceptance-table pins (Supplementary "Monte Carlo Simulation
Algorithms", Metropolis acceptance: 1 for dE <= 0, exp(-beta dE) otherwise).

The table realises the acceptance as u < thr(dE) for a 32-bit uniform u; the
pins compare thr with the closed form 2^32 exp(-beta dE) computed here with
numpy, and check its limits T -> 0 and T -> infinity.
"""
import numpy as np
import pytest

import oracle as O

KB = 8.617333262e-2  # meV/K


@pytest.mark.parametrize("T", [300.0, 800.0, 1000.0, 1200.0, 2500.0, 3000.0])
def test_threshold_closed_form(T):
    A, nA, B = O.threshold_tables(T)
    beta = 0.01 / (KB * T)  # per 0.01 meV unit
    assert A[0] == 2 ** 32 - 1 and B[0] == 2 ** 32 - 1
    assert nA == O.NA_MAX or A[nA] == 0
    assert A[nA - 1] > 0
    assert (np.diff(A[:nA].astype(np.int64)) <= 0).all()
    assert (np.diff(B.astype(np.int64)) <= 0).all()
    rng = np.random.default_rng(int(T))
    ds = np.concatenate([np.arange(1, 3000), rng.integers(1, nA * 1024 + 5000, 3000)])
    for d in ds:
        want = 2.0 ** 32 * np.exp(-beta * float(d))
        got = O.threshold(A, nA, B, int(d))
        assert abs(got - want) <= 4.0 + 1e-9 * want, (d, got, want)
    # beyond the table the threshold is exactly 0 and so is the closed form (< 1)
    assert O.threshold(A, nA, B, nA * 1024 + 7) == 0
    assert 2.0 ** 32 * np.exp(-beta * nA * 1024) < 1.0 or nA == O.NA_MAX


def test_threshold_limits():
    A, nA, B = O.threshold_tables(1e-3)  # T -> 0: only dE <= 0 accepted
    assert nA == 1
    assert all(O.threshold(A, nA, B, d) == 0 for d in [1, 2, 100, 1023, 1024, 10 ** 6])
    A, nA, B = O.threshold_tables(1e12)  # T -> infinity: everything accepted
    assert nA == O.NA_MAX
    beta = 0.01 / (KB * 1e12)
    for d in [1, 1000, 10 ** 5, 10 ** 6]:
        assert O.threshold(A, nA, B, d) >= 2.0 ** 32 * np.exp(-beta * d) - 4
        assert O.threshold(A, nA, B, d) >= 0.999 * 2 ** 32
    # dE <= 0 never reaches the table: it is accepted outright
