"""Oracle sampler pins (Supplementary "Statistical mechanics" and "Monte Carlo
Simulation Algorithms"; canonical swap trials, Metropolis acceptance).

- Exact enumeration: on a 2x2x2-cell BCC box (16 sites, binary 8/8, 12,870
  states) the Boltzmann distribution of the energy levels is computed exactly
  and compared with the oracle chain's energy histogram (chi-square).
- Invariants: composition conservation, split-sweep identity
  sweep(a); sweep(b) == sweep(a + b), attempt counting, V = 0 and T -> 0
  limits.
- Order independence: a Python re-run of the tiled schedule that visits the
  tiles and sites of every phase in a random order must reproduce the
  oracle's trajectory exactly (the LIZ rule makes the order irrelevant).
"""
import itertools

import numpy as np
import pytest
from scipy import stats

import oracle as O
from paper_2503_12591_gb300.inputs import epi_gaussian

KB = 8.617333262e-2


def _exact_levels(V, T):
    dims = (2, 2, 2)
    N = 16
    E = []
    for ones in itertools.combinations(range(N), 8):
        s = np.zeros(N, np.int8)
        s[list(ones)] = 1
        E.append(O.energy(O.BCC, dims, 2, 4, V, s))
    E = np.array(E)
    lev, inv = np.unique(E, return_inverse=True)
    w = np.exp(-(lev - lev.min()) * 0.01 / (KB * T))
    g = np.bincount(inv)
    p = g * w
    return lev, p / p.sum()


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5])
def test_exact_enumeration_chi2(seed):
    V = epi_gaussian(4, 2, 5.0, 100 + seed)
    T = 2000.0
    lev, p = _exact_levels(V, T)
    dims = (2, 2, 2)
    sig = O.init_config(O.BCC, dims, 2, [0.5, 0.5], seed)
    O.sweep(O.BCC, dims, 2, 4, V, sig, T, 200, seed)  # burn-in
    n, thin = 6000, 6
    idx = {int(e): i for i, e in enumerate(lev)}
    hist = np.zeros(len(lev))
    sw = 200
    for _ in range(n):
        O.sweep(O.BCC, dims, 2, 4, V, sig, T, thin, seed, sweep0=sw)
        sw += thin
        hist[idx[O.energy(O.BCC, dims, 2, 4, V, sig)]] += 1
    exp = p * n
    # merge low-expectation levels into one bin
    keep = exp >= 5
    obs = np.concatenate([hist[keep], [hist[~keep].sum()]])
    ex = np.concatenate([exp[keep], [exp[~keep].sum()]])
    if ex[-1] < 5:
        obs[-2] += obs[-1]
        ex[-2] += ex[-1]
        obs, ex = obs[:-1], ex[:-1]
    chi2 = ((obs - ex) ** 2 / ex).sum()
    pval = stats.chi2.sf(chi2, len(ex) - 1)
    assert pval > 1e-3, (chi2, len(ex), pval)


def test_enumeration_detects_wrong_temperature():
    # sensitivity: a chain run at 1.5x the temperature must fail the same test
    V = epi_gaussian(4, 2, 5.0, 101)
    lev, p = _exact_levels(V, 2000.0)
    dims = (2, 2, 2)
    sig = O.init_config(O.BCC, dims, 2, [0.5, 0.5], 1)
    idx = {int(e): i for i, e in enumerate(lev)}
    hist = np.zeros(len(lev))
    for i in range(4000):
        O.sweep(O.BCC, dims, 2, 4, V, sig, 3000.0, 6, 1, sweep0=6 * i)
        hist[idx[O.energy(O.BCC, dims, 2, 4, V, sig)]] += 1
    exp = p * 4000
    keep = exp >= 5
    chi2 = ((hist[keep] - exp[keep]) ** 2 / exp[keep]).sum()
    assert stats.chi2.sf(chi2, keep.sum() - 1) < 1e-6


@pytest.mark.parametrize("kind,K,dims,L,nt", [
    (O.BCC, 4, (12, 12, 12), 3, (4, 4, 4)),
    (O.BCC, 4, (12, 12, 12), 3, (1, 1, 1)),
    (O.FCC, 3, (8, 8, 8), 3, (2, 2, 2)),
])
def test_composition_split_and_counts(kind, K, dims, L, nt):
    M = 4
    V = epi_gaussian(K, M, 20.0, 3)
    sig = O.init_config(kind, dims, M, [0.25] * 4, 7)
    N = sig.size
    c0 = np.bincount(sig, minlength=M)
    a = sig.copy()
    st1 = O.sweep(kind, dims, M, K, V, a, 1000.0, 3, 42, 0, 0, L, nt)
    st2 = O.sweep(kind, dims, M, K, V, a, 1000.0, 2, 42, 3, 0, L, nt)
    b = sig.copy()
    st = O.sweep(kind, dims, M, K, V, b, 1000.0, 5, 42, 0, 0, L, nt)
    assert (a == b).all()
    assert (st1 + st2 == st).all()
    assert st[0] == 5 * N
    assert (np.bincount(b, minlength=M) == c0).all()
    assert 0 < st[1] < st[0] - st[2]
    # a different seed or replica id gives a different trajectory
    c = sig.copy()
    O.sweep(kind, dims, M, K, V, c, 1000.0, 5, 43, 0, 0, L, nt)
    assert (c != b).any()
    d = sig.copy()
    O.sweep(kind, dims, M, K, V, d, 1000.0, 5, 42, 0, 1, L, nt)
    assert (d != b).any()


def test_limits_zero_epi_and_zero_temperature():
    dims, K, M = (6, 6, 6), 4, 4
    sig = O.init_config(O.BCC, dims, M, [0.25] * 4, 3)
    st = O.sweep(O.BCC, dims, M, K, np.zeros((K, M, M), np.int32), sig.copy(), 500.0, 3, 1, L=3)
    assert st[1] == st[0] - st[2]  # V = 0: every distinct-species proposal accepted
    V = epi_gaussian(K, M, 20.0, 5)
    s = sig.copy()
    E = O.energy(O.BCC, dims, M, K, V, s)
    for i in range(5):
        O.sweep(O.BCC, dims, M, K, V, s, 1e-6, 1, 1, sweep0=i, L=3)
        E2 = O.energy(O.BCC, dims, M, K, V, s)
        assert E2 <= E
        E = E2


def _python_sweep(kind, dims, M, K, V, sig, T, seed, sweep, L, nt, rng):
    """Same trials as the oracle, phases in order, but tiles and sites inside a
    phase visited in a random order."""
    z, v = O.shells(kind, K)
    A, nA, B = O.threshold_tables(T)
    m = O.sites_per_cell(kind)
    N = sig.size
    phases = {}
    for s in range(N):
        ph, _ = O.phase_of(kind, dims, L, nt, s)
        phases.setdefault(ph, []).append(s)
    for ph in sorted(phases):
        sites = list(phases[ph])
        rng.shuffle(sites)
        for s in sites:
            rd, ru = O.attempt_words(seed, sweep, 0, s)
            d = (rd * int(z[0])) >> 32
            sp = O.neighbour(kind, dims, s, v[d])
            if sig[s] == sig[sp]:
                continue
            dE = O.delta_e(kind, dims, M, K, V, sig, s, d)
            if dE <= 0 or ru < O.threshold(A, nA, B, dE):
                sig[s], sig[sp] = sig[sp], sig[s]
    return m


@pytest.mark.parametrize("kind,K,dims,L,nt", [
    (O.BCC, 4, (6, 6, 8), 3, (2, 2, 2)),
    (O.FCC, 3, (6, 6, 6), 3, (1, 2, 2)),
])
def test_phase_order_independence(kind, K, dims, L, nt):
    M = 4
    V = epi_gaussian(K, M, 30.0, 11)
    sig = O.init_config(kind, dims, M, [0.25] * 4, 2)
    a = sig.copy()
    O.sweep(kind, dims, M, K, V, a, 1500.0, 2, 5, 0, 0, L, nt)
    b = sig.copy()
    rng = np.random.default_rng(0)
    for sw in range(2):
        _python_sweep(kind, dims, M, K, V, b, 1500.0, 5, sw, L, nt, rng)
    assert (a == b).all()


def test_shared_direction_enumeration_chi2():
    """Shared-direction proposals sample the same canonical distribution:
    nearest-neighbour EPI (K = 1) on the 16-site box with the link-cell
    schedule L = 2 (every phase holds one site), exact enumeration chi^2."""
    dims, K = (2, 2, 2), 1
    V = epi_gaussian(K, 2, 20.0, 31)
    T = 1500.0
    E = []
    for ones in itertools.combinations(range(16), 8):
        s = np.zeros(16, np.int8)
        s[list(ones)] = 1
        E.append(O.energy(O.BCC, dims, 2, K, V, s))
    E = np.array(E)
    lev, inv = np.unique(E, return_inverse=True)
    p = np.bincount(inv) * np.exp(-(lev - lev.min()) * 0.01 / (KB * T))
    p /= p.sum()
    sig = O.init_config(O.BCC, dims, 2, [0.5, 0.5], 3)
    idx = {int(e): i for i, e in enumerate(lev)}
    hist = np.zeros(len(lev))
    n, thin = 5000, 4
    for i in range(n):
        O.sweep(O.BCC, dims, 2, K, V, sig, T, thin, 9, sweep0=thin * i, L=2, proposal=1)
        hist[idx[O.energy(O.BCC, dims, 2, K, V, sig)]] += 1
    exp = p * n
    keep = exp >= 5
    obs = np.concatenate([hist[keep], [hist[~keep].sum()]])
    ex = np.concatenate([exp[keep], [exp[~keep].sum()]])
    if ex[-1] < 5:
        obs, ex = obs[:-1], ex[:-1]
    chi2 = ((obs - ex) ** 2 / ex).sum()
    assert stats.chi2.sf(chi2, len(ex) - 1) > 1e-3


def test_shared_direction_differs_and_is_uniform():
    z1 = 8
    counts = np.zeros(z1, np.int64)
    for t in range(50):
        for ic in range(128):
            counts[O.phase_direction(5, 3, 0, t, ic, z1)] += 1
    exp = counts.sum() / z1
    assert ((counts - exp) ** 2 / exp).sum() < 30.0
    dims, K, M = (12, 12, 12), 4, 4
    V = epi_gaussian(K, M, 20.0, 3)
    a = O.init_config(O.BCC, dims, M, [0.25] * 4, 2)
    b = a.copy()
    O.sweep(O.BCC, dims, M, K, V, a, 1000.0, 2, 1, L=4, nt=(2, 2, 2), proposal=0)
    st = O.sweep(O.BCC, dims, M, K, V, b, 1000.0, 2, 1, L=4, nt=(2, 2, 2), proposal=1)
    assert (a != b).any()
    assert (np.bincount(b, minlength=M) == np.bincount(a, minlength=M)).all()
    assert st[0] == 2 * b.size


def test_block_direction_enumeration_chi2():
    """Block-shared proposals (one direction per tile colour, block of two
    tiles and phase) sample the canonical distribution: nearest-neighbour EPI
    on the 16-site box, link-cell schedule L = 2, exact enumeration chi^2."""
    dims, K = (2, 2, 2), 1
    V = epi_gaussian(K, 2, 20.0, 33)
    T = 1500.0
    E = []
    for ones in itertools.combinations(range(16), 8):
        s = np.zeros(16, np.int8)
        s[list(ones)] = 1
        E.append(O.energy(O.BCC, dims, 2, K, V, s))
    E = np.array(E)
    lev, inv = np.unique(E, return_inverse=True)
    p = np.bincount(inv) * np.exp(-(lev - lev.min()) * 0.01 / (KB * T))
    p /= p.sum()
    sig = O.init_config(O.BCC, dims, 2, [0.5, 0.5], 5)
    idx = {int(e): i for i, e in enumerate(lev)}
    hist = np.zeros(len(lev))
    n, thin = 5000, 4
    for i in range(n):
        O.sweep(O.BCC, dims, 2, K, V, sig, T, thin, 13, sweep0=thin * i, L=2, proposal=2)
        hist[idx[O.energy(O.BCC, dims, 2, K, V, sig)]] += 1
    exp = p * n
    keep = exp >= 5
    obs = np.concatenate([hist[keep], [hist[~keep].sum()]])
    ex = np.concatenate([exp[keep], [exp[~keep].sum()]])
    if ex[-1] < 5:
        obs, ex = obs[:-1], ex[:-1]
    chi2 = ((obs - ex) ** 2 / ex).sum()
    assert stats.chi2.sf(chi2, len(ex) - 1) > 1e-3


def test_block_direction_shared_by_pairs_and_uniform():
    """Mode 2 directions are uniform over the 8 shell-1 directions; on a
    lattice with two blocks per colour the trajectory differs from mode 1's,
    conserves the composition, attempts every site once per sweep, and the
    OpenMP oracle follows it exactly."""
    z1 = 8
    counts = np.zeros(z1, np.int64)
    for blk in range(40):
        for tc in range(8):
            for ic in range(54):
                counts[O.block_direction(5, 3, 0, tc, blk, ic, z1)] += 1
    exp = counts.sum() / z1
    assert ((counts - exp) ** 2 / exp).sum() < 30.0
    dims, K, M = (12, 12, 12), 4, 4
    V = epi_gaussian(K, M, 20.0, 3)
    a = O.init_config(O.BCC, dims, M, [0.25] * 4, 2)
    b, c = a.copy(), a.copy()
    O.sweep(O.BCC, dims, M, K, V, a, 1000.0, 2, 1, L=3, nt=(4, 2, 2), proposal=1)
    st = O.sweep(O.BCC, dims, M, K, V, b, 1000.0, 2, 1, L=3, nt=(4, 2, 2), proposal=2)
    O.sweep_parallel(O.BCC, dims, M, K, V, c, 1000.0, 2, 1, L=3, nt=(4, 2, 2), threads=4, proposal=2)
    assert (a != b).any()
    assert (b == c).all()  # the OpenMP oracle follows the same trajectory
    assert (np.bincount(b, minlength=M) == np.bincount(a, minlength=M)).all()
    assert st[0] == 2 * b.size
