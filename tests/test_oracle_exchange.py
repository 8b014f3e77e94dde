"""Oracle pins for replica exchange between temperature slots (Supplementary
"Parallelization opportunities": configurations at different temperatures
are exchanged by a rule that keeps detailed balance).

The rule pinned here is the textbook parallel-tempering Metropolis step: the
swap of configurations a (slot t, inverse temperature beta_t) and c (slot
t+1) is accepted with probability min(1, exp((beta_t - beta_{t+1})(E_a -
E_c))), and even rounds pair slots (0,1), (2,3), ..., odd rounds (1,2),
(3,4), ...
"""
import numpy as np

import oracle as O

KB = 8.617333262e-2  # meV / K


def test_pairing_schedule_equal_temperatures():
    # equal temperatures: every proposed pair swaps (x = 0)
    R = 5
    T = [1000.0] * R
    E = np.arange(R, dtype=np.int64) * 1000
    rep = np.arange(R, dtype=np.int32)
    acc = np.zeros(R - 1, np.int64)
    O.exchange_round(T, E, rep, 0, 1, acc)
    assert rep.tolist() == [1, 0, 3, 2, 4]
    O.exchange_round(T, E, rep, 1, 1, acc)
    assert rep.tolist() == [1, 3, 0, 4, 2]
    assert acc.tolist() == [1, 1, 1, 1]


def test_sign_cold_slot_takes_lower_energy():
    # slot 0 is the colder one; it holds the higher-energy replica 0, so the
    # swap raises the joint weight and is always accepted
    T = [300.0, 600.0]
    for seed in range(20):
        rep = np.array([0, 1], np.int32)
        O.exchange_round(T, [100_000, 0], rep, 0, seed)
        assert rep.tolist() == [1, 0]
    # the reverse, with a gap of 1000 meV: exp(-19.3) ~ 4e-9, never seen in 200 tries
    for seed in range(200):
        rep = np.array([0, 1], np.int32)
        O.exchange_round(T, [0, 100_000], rep, 0, seed)
        assert rep.tolist() == [0, 1]


def test_odd_round_leaves_two_slots_alone():
    rep = np.array([0, 1], np.int32)
    O.exchange_round([300.0, 300.0], [0, 0], rep, 1, 3)
    assert rep.tolist() == [0, 1]


def test_acceptance_rate_is_boltzmann_ratio():
    T = np.array([800.0, 1000.0])
    b = 1.0 / (KB * T)
    for dE_mev in (-20.0, -60.0):
        E = np.array([0, int(round(-dE_mev * 100))], np.int64)  # E_a - E_c = dE_mev
        x = (b[0] - b[1]) * dE_mev
        p = np.exp(x)
        n = 20000
        hits = 0
        for i in range(n):
            rep = np.array([0, 1], np.int32)
            O.exchange_round(T, E, rep, 2 * i, 11)
            hits += rep[0] == 1
        sigma = np.sqrt(p * (1 - p) / n)
        assert abs(hits / n - p) < 4 * sigma, (dE_mev, hits / n, p)


def test_detailed_balance_two_replica_enumeration():
    """Two replicas on a three-level system: the joint Boltzmann weight is
    stationary under the exchange step (probabilities estimated from many
    rounds, then checked against the balance condition)."""
    T = np.array([700.0, 1400.0])
    b = 1.0 / (KB * T)
    levels = np.array([0, 3000, 9000], np.int64)  # 0, 30, 90 meV
    # swap probability for each ordered pair of levels, estimated
    n = 4000
    P = np.zeros((3, 3))
    for i in range(3):
        for j in range(3):
            hits = 0
            for k in range(n):
                rep = np.array([0, 1], np.int32)
                O.exchange_round(T, [levels[i], levels[j]], rep, 2 * k, 5 + 3 * i + j)
                hits += rep[0] == 1
            P[i, j] = hits / n
    w = lambda i, j: np.exp(-b[0] * levels[i] * 0.01 - b[1] * levels[j] * 0.01)
    for i in range(3):
        for j in range(3):
            lhs = w(i, j) * P[i, j]
            rhs = w(j, i) * P[j, i]
            tol = 4 * np.sqrt(max(P[i, j], P[j, i]) / n) * max(w(i, j), w(j, i)) + 1e-12
            assert abs(lhs - rhs) < tol, (i, j, lhs, rhs)
