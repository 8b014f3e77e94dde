"""Oracle pins for the qSRO model (Method "The EPI and qSRO model", Eq.
quadratic_local_SRO), integer form:

    E = pair energy + sum_i sum_k W[k][s_i] n_k(i)^2,

n_k(i) = number of shell-k neighbours of site i with i's own species (the
same-element pair fraction times z_k; W carries the 1/z_k^2), W in 0.01 meV.

- Closed forms for pure elements, B2 and L1_2 (hand-counted same-species
  neighbours).
- Local energy change = brute-force E(after) - E(before), every site and
  direction, including a 2x2x2 box where shell vectors alias.
- Exact enumeration of the 12,870-state binary box: chi-square of the
  chain's energy histogram against the Boltzmann weights of the model.
- Schedule: the qSRO read reach (R1 + 2 R_K) makes FCC with 3 shells need
  link cells of 4 (the paper's 4x4x4 for FeCoNiAlTi qSRO); brute-force
  independence with the larger read set, and L = 3 must show violations.
"""
import itertools

import numpy as np
import pytest
from scipy import stats

import oracle as O
from paper_2503_12591_gb300.inputs import epi_gaussian

KB = 8.617333262e-2


def _w(K, M, seed, scale=300):
    return np.random.default_rng(seed).integers(-scale, scale + 1, (K, M)).astype(np.int32)


def test_pure_element():
    dims = (3, 4, 3)
    V = epi_gaussian(4, 3, 20.0, 1)
    W = _w(4, 3, 2)
    N = O.n_sites(O.BCC, dims)
    sig = np.full(N, 1, np.int8)
    z = [8, 6, 12, 24]
    want = O.energy(O.BCC, dims, 3, 4, V, sig) + N * sum(int(W[k, 1]) * z[k] ** 2 for k in range(4))
    assert O.energy_qsro(O.BCC, dims, 3, 4, V, W, sig) == want


def test_b2():
    dims = (4, 3, 5)
    V = epi_gaussian(4, 2, 20.0, 3)
    W = _w(4, 2, 4)
    N = O.n_sites(O.BCC, dims)
    sig = np.tile(np.array([0, 1], np.int8), N // 2)
    # shells 1 and 4 join the two sublattices (no same-species neighbours);
    # shells 2 (6) and 3 (12) stay on a sublattice (all same species)
    q = sum(int(W[1, p]) * 36 + int(W[2, p]) * 144 for p in (0, 1)) * (N // 2)
    assert O.energy_qsro(O.BCC, dims, 2, 4, V, W, sig) == O.energy(O.BCC, dims, 2, 4, V, sig) + q


def test_l12():
    dims = (3, 3, 4)
    V = epi_gaussian(3, 2, 30.0, 5)
    W = _w(3, 2, 6)
    N = O.n_sites(O.FCC, dims)
    sig = np.tile(np.array([1, 0, 0, 0], np.int8), N // 4)  # B (1) on the corners
    # B: no B in shell 1, 6 B in shell 2, none in shell 3
    # A: 8 A of 12 in shell 1, 6 of 6 in shell 2, 16 of 24 in shell 3
    qB = 36 * int(W[1, 1])
    qA = 64 * int(W[0, 0]) + 36 * int(W[1, 0]) + 256 * int(W[2, 0])
    want = O.energy(O.FCC, dims, 2, 3, V, sig) + (N // 4) * qB + (3 * N // 4) * qA
    assert O.energy_qsro(O.FCC, dims, 2, 3, V, W, sig) == want


@pytest.mark.parametrize("kind,dims,M,K", [
    (O.BCC, (3, 3, 3), 3, 4),
    (O.BCC, (2, 2, 2), 2, 4),   # aliasing shell vectors
    (O.FCC, (3, 2, 3), 4, 3),
    (O.FCC, (2, 2, 2), 3, 2),
])
def test_delta_e_brute_force(kind, dims, M, K):
    N = O.n_sites(kind, dims)
    z, _ = O.shells(kind, K)
    V = epi_gaussian(K, M, 20.0, 7)
    W = _w(K, M, 8)
    rng = np.random.default_rng(9)
    for trial in range(2):
        sig = rng.integers(0, M, N).astype(np.int8)
        e0 = O.energy_qsro(kind, dims, M, K, V, W, sig)
        for s in range(N):
            for d in range(z[0]):
                _, vecs = O.shells(kind, 1)
                t = O.neighbour(kind, dims, s, vecs[d])
                got = O.delta_e_qsro(kind, dims, M, K, V, W, sig, s, d)
                b = sig.copy()
                b[s], b[t] = sig[t], sig[s]
                assert got == O.energy_qsro(kind, dims, M, K, V, W, b) - e0, (s, d)


def _exact_levels(V, W, T):
    dims = (2, 2, 2)
    E = []
    for ones in itertools.combinations(range(16), 8):
        s = np.zeros(16, np.int8)
        s[list(ones)] = 1
        E.append(O.energy_qsro(O.BCC, dims, 2, 4, V, W, s))
    E = np.array(E)
    lev, inv = np.unique(E, return_inverse=True)
    p = np.bincount(inv) * np.exp(-(lev - lev.min()) * 0.01 / (KB * T))
    return lev, p / p.sum()


@pytest.mark.parametrize("seed", [1, 2])
def test_exact_enumeration_chi2(seed):
    V = epi_gaussian(4, 2, 5.0, 200 + seed)
    W = _w(4, 2, 300 + seed, scale=40)
    T = 2000.0
    lev, p = _exact_levels(V, W, T)
    dims = (2, 2, 2)
    sig = O.init_config(O.BCC, dims, 2, [0.5, 0.5], seed)
    O.sweep_qsro(O.BCC, dims, 2, 4, V, W, sig, T, 100, seed)
    n, thin = 2500, 4
    idx = {int(e): i for i, e in enumerate(lev)}
    hist = np.zeros(len(lev))
    sw = 100
    for _ in range(n):
        O.sweep_qsro(O.BCC, dims, 2, 4, V, W, sig, T, thin, seed, sweep0=sw)
        sw += thin
        hist[idx[O.energy_qsro(O.BCC, dims, 2, 4, V, W, sig)]] += 1
    ex = p * n
    keep = ex >= 5
    obs = np.concatenate([hist[keep], [hist[~keep].sum()]])
    exv = np.concatenate([ex[keep], [ex[~keep].sum()]])
    if exv[-1] < 5:
        obs[-2] += obs[-1]
        exv[-2] += exv[-1]
        obs, exv = obs[:-1], exv[:-1]
    chi2 = ((obs - exv) ** 2 / exv).sum()
    assert stats.chi2.sf(chi2, len(exv) - 1) > 1e-3


def test_enumeration_sees_the_quadratic_term():
    """Control: the chain of the qSRO model is not distributed like the pair
    model alone when W is large."""
    V = epi_gaussian(4, 2, 5.0, 201)
    W = _w(4, 2, 301, scale=60)
    T = 2000.0
    lev_0, p_0 = _exact_levels(V, np.zeros_like(W), T)
    dims = (2, 2, 2)
    sig = O.init_config(O.BCC, dims, 2, [0.5, 0.5], 1)
    n = 1000
    E0 = []
    sw = 0
    for _ in range(n):
        O.sweep_qsro(O.BCC, dims, 2, 4, V, W, sig, T, 4, 1, sweep0=sw)
        sw += 4
        E0.append(O.energy(O.BCC, dims, 2, 4, V, sig))
    # mean pair energy under the qSRO chain vs under the pair model
    mean_pair_model = float((lev_0 * p_0).sum())
    assert abs(np.mean(E0) - mean_pair_model) > 5 * np.std(E0) / np.sqrt(n / 10)


def _neighbours(kind, dims, K):
    z, v = O.shells(kind, K)
    N = O.n_sites(kind, dims)
    return z, np.array([[O.neighbour(kind, dims, s, vec) for vec in v] for s in range(N)], np.int64)


def _violations_qsro(kind, dims, K, L, nt):
    z, nb = _neighbours(kind, dims, K)
    N = nb.shape[0]
    n1 = nb[:, :z[0]]
    ph = np.zeros(N, np.int64)
    tile = np.zeros((N, 3), np.int64)
    for s in range(N):
        p, t = O.phase_of(kind, dims, L, nt, s)
        ph[s] = p
        tile[s] = t
    nA = L ** 3 * O.sites_per_cell(kind)
    tc, ic = ph // nA, ph % nA
    bad = 0
    for s2 in range(N):
        # sites whose local energy a trial at s2 may change, for any partner
        U = np.unique(np.concatenate([[s2], n1[s2], nb[s2], nb[n1[s2]].ravel()]))
        # ... and every site their local energies read
        R = np.unique(np.concatenate([U, nb[U].ravel()]))
        X = np.unique(np.concatenate([R, n1[R].ravel()]))
        X = X[X != s2]
        conc = (tc[X] == tc[s2]) & ((tile[X] != tile[s2]).any(1) | (ic[X] == ic[s2]))
        bad += int(conc.sum())
    return bad


@pytest.mark.parametrize("dims,L,nt", [
    ((8, 8, 8), 4, (1, 1, 1)),     # the paper's 4x4x4 link cell
    ((12, 8, 8), 4, (4, 2, 2)),    # thinnest tiles the qSRO reach allows (3 cells)
])
def test_fcc_qsro_schedule_independent(dims, L, nt):
    assert O.schedule_check_model(O.FCC, dims, 3, L, nt, 1) == 0
    assert _violations_qsro(O.FCC, dims, 3, L, nt) == 0


def test_fcc_qsro_needs_larger_link_cell():
    dims = (9, 9, 9)
    assert O.schedule_check_model(O.FCC, dims, 3, 3, (1, 1, 1), 0) == 0   # fine for the pair model
    assert O.schedule_check_model(O.FCC, dims, 3, 3, (1, 1, 1), 1) != 0   # not for qSRO
    assert _violations_qsro(O.FCC, dims, 3, 3, (1, 1, 1)) > 0
    assert O.schedule_check_model(O.FCC, (12, 8, 8), 3, 4, (6, 2, 2), 1) != 0  # tiles of 2 cells


def test_qsro_tile_passes_compose_to_sweep():
    """Every tile of colour 0, then 1, ... through the single-tile pass equals
    the qSRO sweep (the single-tile pass is the sweep restricted to a tile)."""
    kind, K, dims, L, nt, M = O.FCC, 3, (12, 8, 8), 4, (4, 2, 2), 3
    V = epi_gaussian(K, M, 20.0, 6)
    W = _w(K, M, 7)
    sig = O.init_config(kind, dims, M, [1 / 3] * 3, 8)
    a, b = sig.copy(), sig.copy()
    st = O.sweep_qsro(kind, dims, M, K, V, W, a, 1100.0, 1, 3, sweep0=5, replica=2, L=L, nt=nt)
    tot = np.zeros(4, np.int64)
    for tc in range(8):
        for z in range(nt[2]):
            for y in range(nt[1]):
                for x in range(nt[0]):
                    if (x & 1) | ((y & 1) << 1) | ((z & 1) << 2) == tc:
                        tot += O.tile_pass_qsro(kind, dims, M, K, V, W, b, 1100.0, 3, 5, 2, L, nt, (x, y, z))
    assert (a == b).all()
    assert tot.tolist() == st.tolist()


def test_qsro_local_energy_sum_rule_and_l12():
    dims = (3, 3, 4)
    V = epi_gaussian(3, 2, 30.0, 5)
    W = _w(3, 2, 6)
    N = O.n_sites(O.FCC, dims)
    sig = np.tile(np.array([1, 0, 0, 0], np.int8), N // 4)
    e2 = O.local_energy2_qsro(O.FCC, dims, 2, 3, V, W, sig)
    pair = O.local_energy2(O.FCC, dims, 2, 3, V, sig)
    assert (e2[0::4] - pair[0::4] == 2 * 36 * int(W[1, 1])).all()
    assert (e2[1::4] - pair[1::4] == 2 * (64 * int(W[0, 0]) + 36 * int(W[1, 0]) + 256 * int(W[2, 0]))).all()
    rnd = np.random.default_rng(3).integers(0, 2, N).astype(np.int8)
    assert O.local_energy2_qsro(O.FCC, dims, 2, 3, V, W, rnd).sum() == 2 * O.energy_qsro(O.FCC, dims, 2, 3, V, W, rnd)
